/*
 * CPU oracle for the BLINK dirty-imaging hot path (arXiv 2505.15204).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code, header or constant with the CUDA library.
 *
 * It is a plain, slow statement of what the method computes, one function per step, in exact integer
 * arithmetic for the correlation and in FP64 for everything else:
 *
 *   correlate   Eq. 2 and Sec. 5.2.2: S_ij^pq = sum_{t, ch} x_i^p conj(x_j^q) over the N_s samples of an
 *               integration and the c fine channels of an output channel; lower triangle i >= j.
 *   uvw         Sec. 5.2.3-5.2.4: (u, v, w) = (r_i - r_j) * nu / c for every baseline and channel.
 *   cells       Sec. 5.2.4 (gridding "based on the (u, v) coordinates", nearest cell, no kernel).
 *   phase       Sec. 5.2.3 (geometric corrections: the phase centre set to a pointing direction, with the
 *               (u, v, w) of that direction): V' = V exp(+2 pi i w), (u, v) in the tangent plane at it.
 *   gains       Sec. 5.2.3 (calibration and cable-length corrections): per-tile, per-polarisation complex
 *               gains g, V_ij^pq = g_i^p S_ij^pq conj(g_j^q) (a diagonal Jones matrix per tile).
 *   grid        Sec. 5.2.4: natural weighting, every visibility and its Hermitian mirror weight 1.
 *   fft2        Eq. 4 / Sec. 5.2.4: unnormalised inverse 2D transform, own radix-2 FFT for powers of
 *               two and a mixed-radix Cooley-Tukey recursion for other sides; direct DFT for small sides.
 *   image       Sec. 5.2.4: real part / sum of weights, shifted so the phase centre is the middle pixel.
 *   grid_kb     Sec. 5.2.4 and 8 (gridding with a convolution kernel, in progress in the paper): each
 *               visibility spread over W x W cells of a grid twice the image side by a separable
 *               Kaiser-Bessel kernel; the image is the central half of the transform, divided by the
 *               kernel's Fourier transform (grid correction).
 *   dedisperse  Sec. 2 and 7 (the FRB search that follows imaging): incoherent dedispersion of the image cube,
 *               out[t] = (1/F) sum_f img[t + d_f][f] with per-channel delays d_f in integrations.
 *
 * Readings where the paper is silent (stated in the design notes): Stokes I = (S_XX + S_YY) / (2K);
 * uv cell default = u_max / (N/2 - 1); cell = floor(u / du + 1/2); autos gridded at (0, 0); grid DC at
 * [0][0], row = v, column = u; image row = y (m), column = x (l), pixel (N/2, N/2) = phase centre.
 *
 * Compiled with -ffp-contract=off so each FP64 operation rounds once, in the order written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_C_LIGHT 299792458.0
#define ORC_TWO_PI 6.283185307179586476925286766559

enum { ORC_POL_I = 0, ORC_POL_XX = 1 };

/* ---- packed 4-bit complex sample: re = low nibble, im = high nibble, two's complement ---- */
static int orc_lo(uint8_t b) { int v = b & 0xF; return v >= 8 ? v - 16 : v; }
static int orc_hi(uint8_t b) { int v = (b >> 4) & 0xF; return v >= 8 ? v - 16 : v; }

int64_t oracle_n_baselines(int n_tiles) { return (int64_t)n_tiles * (n_tiles + 1) / 2; }

/*
 * Correlation of one integration `tau` and one output channel `f` (Eq. 2; Sec. 5.2.2: lower triangle per
 * integration and channel).  `volt` points at sample 0 of the set's first fine channel; consecutive
 * samples are `fine_stride * n_tiles * 2` bytes apart and consecutive fine channels `n_tiles * 2`.
 * S is int64 [B][4][2] (re, im) with b = i(i+1)/2 + j and polarisation index 2p + q (XX, XY, YX, YY).
 * Pairs with a flagged tile stay 0.
 */
void oracle_correlate_one(const uint8_t* volt, int64_t fine_stride, int n_tiles, int ns, int c, int tau, int f,
                          const uint8_t* flags, int64_t* S)
{
    int64_t B = oracle_n_baselines(n_tiles);
    memset(S, 0, (size_t)B * 8 * sizeof(int64_t));
    int64_t sample_stride = fine_stride * n_tiles * 2;
    for (int t = tau * ns; t < (tau + 1) * ns; t++) {
        for (int ch = f * c; ch < (f + 1) * c; ch++) {
            const uint8_t* x = volt + (int64_t)t * sample_stride + (int64_t)ch * n_tiles * 2;
            for (int i = 0; i < n_tiles; i++) {
                for (int j = 0; j <= i; j++) {
                    if (flags && (flags[i] || flags[j])) continue;
                    int64_t b = (int64_t)i * (i + 1) / 2 + j;
                    for (int p = 0; p < 2; p++) {
                        for (int q = 0; q < 2; q++) {
                            int64_t ar = orc_lo(x[2 * i + p]), ai = orc_hi(x[2 * i + p]);
                            int64_t br = orc_lo(x[2 * j + q]), bi = orc_hi(x[2 * j + q]);
                            /* (ar + i ai) * conj(br + i bi) */
                            S[(b * 4 + 2 * p + q) * 2 + 0] += ar * br + ai * bi;
                            S[(b * 4 + 2 * p + q) * 2 + 1] += ai * br - ar * bi;
                        }
                    }
                }
            }
        }
    }
}

/* All integrations and output channels: S int64 [T][F][B][4][2], T = n_samples / ns, F = n_fine / c. */
void oracle_correlate(const uint8_t* volt, int64_t fine_stride, int n_tiles, int n_fine, int c, int ns,
                      int n_samples, const uint8_t* flags, int64_t* S)
{
    int T = n_samples / ns, F = n_fine / c;
    int64_t per = oracle_n_baselines(n_tiles) * 8;
    for (int tau = 0; tau < T; tau++)
        for (int f = 0; f < F; f++)
            oracle_correlate_one(volt, fine_stride, n_tiles, ns, c, tau, f, flags, S + ((int64_t)tau * F + f) * per);
}

/*
 * Calibration of one integration and channel (Sec. 5.2.3, corrections applied to the visibilities): with a
 * diagonal Jones matrix diag(g_i^X, g_i^Y) per tile, V_ij^pq = g_i^p S_ij^pq conj(g_j^q).  g is complex
 * double [n_tiles][2 pol][2] (re, im); S int64 [B][4][2]; V complex double [B][4][2] (raw sums, not / K).
 */
void oracle_apply_gains(const int64_t* S, int n_tiles, const double* g, double* V)
{
    for (int i = 0; i < n_tiles; i++) {
        for (int j = 0; j <= i; j++) {
            int64_t b = (int64_t)i * (i + 1) / 2 + j;
            for (int p = 0; p < 2; p++) {
                for (int q = 0; q < 2; q++) {
                    double sr = (double)S[(b * 4 + 2 * p + q) * 2 + 0], si = (double)S[(b * 4 + 2 * p + q) * 2 + 1];
                    double gr = g[(i * 2 + p) * 2 + 0], gi = g[(i * 2 + p) * 2 + 1];
                    double hr = g[(j * 2 + q) * 2 + 0], hi = -g[(j * 2 + q) * 2 + 1];   /* conj(g_j^q) */
                    /* (gr + i gi)(sr + i si) */
                    double tr = gr * sr - gi * si, ti = gr * si + gi * sr;
                    /* (tr + i ti)(hr + i hi) */
                    V[(b * 4 + 2 * p + q) * 2 + 0] = tr * hr - ti * hi;
                    V[(b * 4 + 2 * p + q) * 2 + 1] = tr * hi + ti * hr;
                }
            }
        }
    }
}

/*
 * Full calibration (Sec. 5.2.3) with a 2x2 Jones matrix per tile: V_ij = J_i S_ij J_j^H, i.e.
 * V_ij^pq = sum_{r,s} J_i[p][r] S_ij^rs conj(J_j[q][s]).  J is complex double [n_tiles][2][2][2]
 * (J[p][r] re, im); S int64 [B][4][2]; V complex double [B][4][2].  A diagonal J is oracle_apply_gains.
 */
void oracle_apply_jones(const int64_t* S, int n_tiles, const double* J, double* V)
{
    for (int i = 0; i < n_tiles; i++) {
        for (int j = 0; j <= i; j++) {
            int64_t b = (int64_t)i * (i + 1) / 2 + j;
            for (int p = 0; p < 2; p++) {
                for (int q = 0; q < 2; q++) {
                    double vr = 0.0, vi = 0.0;
                    for (int r = 0; r < 2; r++) {
                        for (int s2 = 0; s2 < 2; s2++) {
                            double sr = (double)S[(b * 4 + 2 * r + s2) * 2 + 0];
                            double si = (double)S[(b * 4 + 2 * r + s2) * 2 + 1];
                            double ar = J[((i * 2 + p) * 2 + r) * 2 + 0], ai = J[((i * 2 + p) * 2 + r) * 2 + 1];
                            double cr = J[((j * 2 + q) * 2 + s2) * 2 + 0], ci = -J[((j * 2 + q) * 2 + s2) * 2 + 1];
                            double tr = ar * sr - ai * si, ti = ar * si + ai * sr;   /* J_i[p][r] S^rs */
                            vr += tr * cr - ti * ci;                                  /* * conj(J_j[q][s]) */
                            vi += tr * ci + ti * cr;
                        }
                    }
                    V[(b * 4 + 2 * p + q) * 2 + 0] = vr;
                    V[(b * 4 + 2 * p + q) * 2 + 1] = vi;
                }
            }
        }
    }
}

/* Output-channel centre frequency = mean of its c fine-channel centres (summed in order, then / c). */
void oracle_output_freqs(const double* fine, int n_fine, int c, double* out)
{
    for (int f = 0; f < n_fine / c; f++) {
        double s = 0.0;
        for (int k = 0; k < c; k++) s += fine[f * c + k];
        out[f] = s / (double)c;
    }
}

/* Baseline coordinates in wavelengths (Sec. 5.2.3-5.2.4): b = r_i - r_j (E, N, U metres),
 * (u, v, w) = b * (nu / c).  uvw is [B][3]. */
void oracle_uvw(const double* enu, int n_tiles, double nu, double* uvw)
{
    double inv_lambda = nu / ORC_C_LIGHT;
    for (int i = 0; i < n_tiles; i++)
        for (int j = 0; j <= i; j++) {
            int64_t b = (int64_t)i * (i + 1) / 2 + j;
            for (int d = 0; d < 3; d++) uvw[b * 3 + d] = (enu[i * 3 + d] - enu[j * 3 + d]) * inv_lambda;
        }
}

/*
 * Phase centre (Sec. 5.2.3: geometric corrections set the phase centre to a pointing direction, and the
 * imager computes (u, v, w) for it).  The pointing s0 = (l0, m0, n0) is given by direction cosines in the
 * local (E, N, Up) frame, n0 = sqrt(1 - l0^2 - m0^2).  The image plane's axes (e_l, e_m) are E and N carried
 * to s0 by the rotation about Up x s0 that takes Up to s0 (Rodrigues' formula; the identity at zenith):
 * with r = sqrt(l0^2 + m0^2) and k = (-m0, l0, 0) / r,
 *     e_l = (n0 + kx^2 (1 - n0),  kx ky (1 - n0),      -ky r)
 *     e_m = (kx ky (1 - n0),      n0 + ky^2 (1 - n0),   kx r).
 * Returns -1 unless l0^2 + m0^2 < 1.
 */
int oracle_phase_basis(double l0, double m0, double* el, double* em, double* s0)
{
    double r2 = l0 * l0 + m0 * m0;
    if (!(r2 < 1.0)) return -1;
    double n0 = sqrt(1.0 - r2);
    s0[0] = l0;
    s0[1] = m0;
    s0[2] = n0;
    if (r2 == 0.0) {
        el[0] = 1.0; el[1] = 0.0; el[2] = 0.0;
        em[0] = 0.0; em[1] = 1.0; em[2] = 0.0;
        return 0;
    }
    double r = sqrt(r2), kx = -m0 / r, ky = l0 / r, c1 = 1.0 - n0;
    el[0] = n0 + kx * kx * c1;
    el[1] = kx * ky * c1;
    el[2] = -ky * r;
    em[0] = kx * ky * c1;
    em[1] = n0 + ky * ky * c1;
    em[2] = kx * r;
    return 0;
}

/* (u, v, w) of every baseline for the pointing (l0, m0): u = b.e_l nu/c, v = b.e_m nu/c, w = b.s0 nu/c,
 * b = r_i - r_j.  At zenith this is oracle_uvw exactly.  Returns -1 for an invalid pointing. */
int oracle_uvw_phased(const double* enu, int n_tiles, double nu, double l0, double m0, double* uvw)
{
    double el[3], em[3], s0[3];
    if (oracle_phase_basis(l0, m0, el, em, s0)) return -1;
    double inv_lambda = nu / ORC_C_LIGHT;
    for (int i = 0; i < n_tiles; i++)
        for (int j = 0; j <= i; j++) {
            int64_t b = (int64_t)i * (i + 1) / 2 + j;
            double d[3];
            for (int k = 0; k < 3; k++) d[k] = enu[i * 3 + k] - enu[j * 3 + k];
            uvw[b * 3 + 0] = (d[0] * el[0] + d[1] * el[1] + d[2] * el[2]) * inv_lambda;
            uvw[b * 3 + 1] = (d[0] * em[0] + d[1] * em[1] + d[2] * em[2]) * inv_lambda;
            uvw[b * 3 + 2] = (d[0] * s0[0] + d[1] * s0[1] + d[2] * s0[2]) * inv_lambda;
        }
    return 0;
}

/* V <- V exp(+2 pi i w) for every baseline and polarisation product (V complex double [B][4][2]); the
 * phase is taken from w's fractional part (w - round(w) is exact), so large w lose no precision. */
void oracle_apply_phase(double* V, const double* uvw, int64_t n_baselines)
{
    for (int64_t b = 0; b < n_baselines; b++) {
        double w = uvw[b * 3 + 2], fr = w - nearbyint(w);
        double c = cos(ORC_TWO_PI * fr), sn = sin(ORC_TWO_PI * fr);
        for (int p = 0; p < 4; p++) {
            double* z = V + (b * 4 + p) * 2;
            double re = z[0] * c - z[1] * sn, im = z[0] * sn + z[1] * c;
            z[0] = re;
            z[1] = im;
        }
    }
}

/* Default uv cell (wavelengths): the longest unflagged projected baseline at the highest frequency lands
 * in the outermost usable cell, du = u_max / (N/2 - 1); u_max = max |(b_E, b_N)| * (nu_max / c).  With a
 * convolution kernel of W >= 2 cells the grid side is 2N and the support must stay inside it too:
 * du = u_max / (N - 1 - W/2), which keeps the image's pixel scale within a fraction of a percent of the
 * nearest-cell one.  The projection is onto the image plane of the pointing (l0, m0) (oracle_phase_basis):
 * (b_E, b_N) at zenith, (b.e_l, b.e_m) elsewhere.
 * Degenerate arrays (no unflagged baseline of non-zero length) and invalid pointings get du = 1. */
double oracle_default_cell(const double* enu, int n_tiles, const uint8_t* flags, double nu_max, int n_pix,
                           int support, double l0, double m0)
{
    double el[3], em[3], s0[3];
    if (oracle_phase_basis(l0, m0, el, em, s0)) return 1.0;
    double dmax = 0.0;
    for (int i = 0; i < n_tiles; i++)
        for (int j = 0; j < i; j++) {
            if (flags && (flags[i] || flags[j])) continue;
            double b[3];
            for (int k = 0; k < 3; k++) b[k] = enu[i * 3 + k] - enu[j * 3 + k];
            double be = b[0] * el[0] + b[1] * el[1] + b[2] * el[2];
            double bn = b[0] * em[0] + b[1] * em[1] + b[2] * em[2];
            double d = sqrt(be * be + bn * bn);
            if (d > dmax) dmax = d;
        }
    double umax = dmax * (nu_max / ORC_C_LIGHT);
    if (!(umax > 0.0)) return 1.0;
    if (support >= 2) return umax / ((double)(n_pix - 1) - 0.5 * (double)support);
    return umax / (double)(n_pix / 2 - 1);
}

/* Nearest grid cell: iu = floor(u / du + 1/2), iv = floor(v / du + 1/2); kept iff |iu|, |iv| < N/2. */
void oracle_cells(const double* uvw, int64_t n_baselines, double du, int n_pix, int32_t* iu, int32_t* iv,
                  uint8_t* keep)
{
    int h = n_pix / 2;
    for (int64_t b = 0; b < n_baselines; b++) {
        double x = floor(uvw[b * 3 + 0] / du + 0.5);
        double y = floor(uvw[b * 3 + 1] / du + 0.5);
        int ok = fabs(x) < (double)h && fabs(y) < (double)h;
        iu[b] = ok ? (int32_t)x : 0;
        iv[b] = ok ? (int32_t)y : 0;
        keep[b] = (uint8_t)ok;
    }
}

/*
 * Gridding of one image (Sec. 5.2.4): natural weighting, nearest cell, no convolution kernel.
 * Visibility of baseline (i, j): Stokes I = (S_XX + S_YY) / (2K), or XX = S_XX / K.
 * Cross baselines (i > j, kept): G[v][u] += I and G[-v][-u] += conj(I), weight 2.
 * Autocorrelations (i == j, when `autos`): G[0][0] += I, weight 1.
 * G is complex double [N][N] (re, im interleaved), row = v, column = u, indices modulo N.
 * Returns W, the sum of weights.
 */
double oracle_grid(const int64_t* S, int n_tiles, const uint8_t* flags, int K, int pol, int autos,
                   const int32_t* iu, const int32_t* iv, const uint8_t* keep, int n_pix, double* G)
{
    int n = n_pix;
    memset(G, 0, (size_t)n * n * 2 * sizeof(double));
    double W = 0.0;
    for (int i = 0; i < n_tiles; i++) {
        for (int j = 0; j <= i; j++) {
            if (flags && (flags[i] || flags[j])) continue;
            int64_t b = (int64_t)i * (i + 1) / 2 + j;
            const int64_t* s = S + b * 8;
            double re, im;
            if (pol == ORC_POL_I) {
                re = (double)(s[0] + s[6]) / (2.0 * (double)K);
                im = (double)(s[1] + s[7]) / (2.0 * (double)K);
            } else {
                re = (double)s[0] / (double)K;
                im = (double)s[1] / (double)K;
            }
            if (i == j) {
                if (!autos) continue;
                G[0] += re;
                G[1] += im;
                W += 1.0;
                continue;
            }
            if (!keep[b]) continue;
            int u = ((iu[b] % n) + n) % n, v = ((iv[b] % n) + n) % n;
            int um = ((-iu[b] % n) + n) % n, vm = ((-iv[b] % n) + n) % n;
            G[((int64_t)v * n + u) * 2 + 0] += re;
            G[((int64_t)v * n + u) * 2 + 1] += im;
            G[((int64_t)vm * n + um) * 2 + 0] += re;
            G[((int64_t)vm * n + um) * 2 + 1] -= im;
            W += 2.0;
        }
    }
    return W;
}

/* oracle_grid for calibrated visibilities V (complex double [B][4][2], raw sums as from oracle_apply_gains):
 * the same cells, weights and order of additions. */
double oracle_grid_v(const double* V, int n_tiles, const uint8_t* flags, int K, int pol, int autos,
                     const int32_t* iu, const int32_t* iv, const uint8_t* keep, int n_pix, double* G)
{
    int n = n_pix;
    memset(G, 0, (size_t)n * n * 2 * sizeof(double));
    double W = 0.0;
    for (int i = 0; i < n_tiles; i++) {
        for (int j = 0; j <= i; j++) {
            if (flags && (flags[i] || flags[j])) continue;
            int64_t b = (int64_t)i * (i + 1) / 2 + j;
            const double* s = V + b * 8;
            double re, im;
            if (pol == ORC_POL_I) {
                re = (s[0] + s[6]) / (2.0 * (double)K);
                im = (s[1] + s[7]) / (2.0 * (double)K);
            } else {
                re = s[0] / (double)K;
                im = s[1] / (double)K;
            }
            if (i == j) {
                if (!autos) continue;
                G[0] += re;
                G[1] += im;
                W += 1.0;
                continue;
            }
            if (!keep[b]) continue;
            int u = ((iu[b] % n) + n) % n, v = ((iv[b] % n) + n) % n;
            int um = ((-iu[b] % n) + n) % n, vm = ((-iv[b] % n) + n) % n;
            G[((int64_t)v * n + u) * 2 + 0] += re;
            G[((int64_t)v * n + u) * 2 + 1] += im;
            G[((int64_t)vm * n + um) * 2 + 0] += re;
            G[((int64_t)vm * n + um) * 2 + 1] -= im;
            W += 2.0;
        }
    }
    return W;
}

/*
 * Gridding with a convolution kernel (Sec. 5.2.4; Sec. 8 lists kernels as work in progress).  The kernel is
 * not specified by the paper; this is a separable Kaiser-Bessel kernel of W cells,
 *     C(t) = I0(beta sqrt(1 - (2t / W)^2)) / Z  for |t| < W/2, else 0,
 * normalised to unit integral (Z = W sinh(beta) / beta), on a grid oversampled by alpha = 2 (grid side
 * twice the image side), with beta = pi sqrt((W / alpha)^2 (alpha - 1/2)^2 - 0.8), the value Beatty,
 * Nishimura and Pauly (IEEE TMI 2005) give for that oversampling.
 */

/* I0(x), the modified Bessel function of the first kind of order 0, from its power series
 * sum_k ((x/2)^k / k!)^2 (all terms positive, summed until they stop changing the sum). */
double oracle_i0(double x)
{
    double q = 0.25 * x * x, term = 1.0, sum = 1.0;
    for (int k = 1; k < 1000; k++) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term <= 1e-17 * sum) break;
    }
    return sum;
}

double oracle_kb_beta(int support)
{
    return 3.14159265358979323846 * sqrt(0.5625 * (double)support * (double)support - 0.8);
}

double oracle_kb(double t, int support, double beta)
{
    double h = 0.5 * (double)support;
    if (!(fabs(t) < h)) return 0.0;
    double r = t / h;
    return oracle_i0(beta * sqrt(1.0 - r * r)) * beta / ((double)support * sinh(beta));
}

/* The kernel's Fourier transform c(nu) = integral C(t) exp(-2 pi i nu t) dt (nu in cycles per cell).  With
 * a = pi W nu, the integral of I0(beta sqrt(1 - x^2)) cos(a x) over [-1, 1] is 2 sinh(r) / r for
 * r = sqrt(beta^2 - a^2) (2 sin(r) / r with r = sqrt(a^2 - beta^2) beyond a = beta), so
 * c(nu) = (sinh(r) / r) / (sinh(beta) / beta), c(0) = 1. */
double oracle_kb_ft(double nu, int support, double beta)
{
    double a = 3.14159265358979323846 * (double)support * nu;
    double d = beta * beta - a * a, s;
    if (d > 0.0) {
        double r = sqrt(d);
        s = sinh(r) / r;
    } else if (d < 0.0) {
        double r = sqrt(-d);
        s = sin(r) / r;
    } else {
        s = 1.0;
    }
    return s * beta / sinh(beta);
}

/* Spread value (re, im) at continuous cell position (gu, gv) over the cells (cu, cv) with |cu - gu| < W/2
 * and |cv - gv| < W/2 with weights C(cu - gu) C(cv - gv); with `mirror` also (re, -im) at (-cu, -cv).
 * Cell indices are taken modulo N. */
static void orc_spread(double* G, int n, double gu, double gv, double re, double im, int mirror, int support,
                       double beta)
{
    double h = 0.5 * (double)support;
    for (int cv = (int)floor(gv - h); cv <= (int)ceil(gv + h); cv++) {
        if (!(fabs((double)cv - gv) < h)) continue;
        double wv = oracle_kb((double)cv - gv, support, beta);
        for (int cu = (int)floor(gu - h); cu <= (int)ceil(gu + h); cu++) {
            if (!(fabs((double)cu - gu) < h)) continue;
            double w = oracle_kb((double)cu - gu, support, beta) * wv;
            int u = ((cu % n) + n) % n, v = ((cv % n) + n) % n;
            G[((int64_t)v * n + u) * 2 + 0] += w * re;
            G[((int64_t)v * n + u) * 2 + 1] += w * im;
            if (mirror) {
                int um = ((-cu % n) + n) % n, vm = ((-cv % n) + n) % n;
                G[((int64_t)vm * n + um) * 2 + 0] += w * re;
                G[((int64_t)vm * n + um) * 2 + 1] -= w * im;
            }
        }
    }
}

/*
 * Convolutional gridding of one image onto a grid of side n_grid.  V: raw sums complex double [B][4][2]
 * (integer sums, or calibrated ones), K the samples per visibility; the visibility of (i, j) is that of
 * oracle_grid.  A cross visibility at g = (u / du, v / du) is kept iff its whole support lies within
 * |c| <= n_grid/2 - 1 on both axes, i.e. |gu|, |gv| <= n_grid/2 - W/2; it and its mirror are spread with
 * weight 2 in W.  Autocorrelations sit at g = 0 (no mirror, weight 1).  G: complex double
 * [n_grid][n_grid], zeroed here.  Returns W.
 */
double oracle_grid_kb(const double* V, int n_tiles, const uint8_t* flags, int K, int pol, int autos,
                      const double* uvw, double du, int support, int n_grid, double* G)
{
    int n = n_grid;
    double beta = oracle_kb_beta(support), lim = 0.5 * (double)n_grid - 0.5 * (double)support;
    memset(G, 0, (size_t)n * n * 2 * sizeof(double));
    double W = 0.0;
    for (int i = 0; i < n_tiles; i++) {
        for (int j = 0; j <= i; j++) {
            if (flags && (flags[i] || flags[j])) continue;
            int64_t b = (int64_t)i * (i + 1) / 2 + j;
            const double* s = V + b * 8;
            double re, im;
            if (pol == ORC_POL_I) {
                re = (s[0] + s[6]) / (2.0 * (double)K);
                im = (s[1] + s[7]) / (2.0 * (double)K);
            } else {
                re = s[0] / (double)K;
                im = s[1] / (double)K;
            }
            if (i == j) {
                if (!autos) continue;
                orc_spread(G, n, 0.0, 0.0, re, im, 0, support, beta);
                W += 1.0;
                continue;
            }
            double gu = uvw[b * 3 + 0] / du, gv = uvw[b * 3 + 1] / du;
            if (!(fabs(gu) <= lim && fabs(gv) <= lim)) continue;
            orc_spread(G, n, gu, gv, re, im, 1, support, beta);
            W += 2.0;
        }
    }
    return W;
}

/* The N x N image from the shifted image `full` of the 2N grid: its central half (full pixel (x + N/2,
 * y + N/2)), divided by c((x - N/2) / 2N) c((y - N/2) / 2N) to undo the kernel's taper (grid correction;
 * |nu| <= 1/4 cycle per cell). */
void oracle_kb_crop_correct(const double* full, int n, int support, double* img)
{
    double beta = oracle_kb_beta(support);
    for (int y = 0; y < n; y++) {
        double cy = oracle_kb_ft((double)(y - n / 2) / (double)(2 * n), support, beta);
        for (int x = 0; x < n; x++) {
            double cx = oracle_kb_ft((double)(x - n / 2) / (double)(2 * n), support, beta);
            img[(int64_t)y * n + x] = full[(int64_t)(y + n / 2) * 2 * n + (x + n / 2)] / (cx * cy);
        }
    }
}

/* In-place unnormalised inverse DFT of n (a power of two) complex values spaced `stride` complex elements
 * apart: X[k] <- sum_m X[m] exp(+2 pi i k m / n).  Iterative radix-2 Cooley-Tukey: bit-reversal
 * permutation, then log2(n) butterfly stages; twiddles from libm cos/sin. */
static void orc_ifft_1d(double* x, int n, int64_t stride)
{
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double* a = x + (int64_t)i * stride * 2;
            double* b = x + (int64_t)j * stride * 2;
            double tr = a[0], ti = a[1];
            a[0] = b[0]; a[1] = b[1];
            b[0] = tr; b[1] = ti;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int k = 0; k < half; k++) {
            double ang = ORC_TWO_PI * (double)k / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int i = 0; i < n; i += len) {
                double* a = x + (int64_t)(i + k) * stride * 2;
                double* b = x + (int64_t)(i + k + half) * stride * 2;
                double tr = b[0] * wr - b[1] * wi;
                double ti = b[0] * wi + b[1] * wr;
                b[0] = a[0] - tr; b[1] = a[1] - ti;
                a[0] = a[0] + tr; a[1] = a[1] + ti;
            }
        }
    }
}

/* The same transform for any length n >= 1 (sides that are not powers of two): recursive Cooley-Tukey
 * decimation in time on the smallest prime factor p of n.  With q = n / p, the q-point transforms
 * X_r[k] = sum_j x[j p + r] w_q^(j k) of the p interleaved subsequences give
 * X[k] = sum_{r < p} w_n^(r k) X_r[k mod q]; a prime length is summed directly.  root[e] = w_N^e for the
 * top-level length N, and w_n^e = root[e * (N / n)] with the exponent reduced modulo n in integers.
 * x: n complex values `stride` complex elements apart; out: n contiguous complex values. */
static void orc_idft_any(const double* x, int64_t stride, int n, const double* root, int N, double* out)
{
    int p = n;
    for (int d = 2; d * d <= n; d++)
        if (n % d == 0) { p = d; break; }
    int64_t step = N / n;                 /* w_n^e = w_N^(e step) */
    if (p == n) {
        for (int k = 0; k < n; k++) {
            double sr = 0.0, si = 0.0;
            for (int m = 0; m < n; m++) {
                int64_t e = ((int64_t)k * m) % n;
                double c = root[2 * e * step], s = root[2 * e * step + 1];
                double xr = x[(int64_t)m * stride * 2], xi = x[(int64_t)m * stride * 2 + 1];
                sr += xr * c - xi * s;
                si += xr * s + xi * c;
            }
            out[2 * k] = sr;
            out[2 * k + 1] = si;
        }
        return;
    }
    int q = n / p;
    double* sub = (double*)malloc(sizeof(double) * 2 * (size_t)n);      /* [p][q] sub-transforms */
    for (int r = 0; r < p; r++)
        orc_idft_any(x + (int64_t)r * stride * 2, stride * p, q, root, N, sub + (int64_t)r * q * 2);
    for (int k = 0; k < n; k++) {
        double sr = 0.0, si = 0.0;
        for (int r = 0; r < p; r++) {
            int64_t e = ((int64_t)r * k) % n;
            double c = root[2 * e * step], s = root[2 * e * step + 1];
            double yr = sub[((int64_t)r * q + k % q) * 2], yi = sub[((int64_t)r * q + k % q) * 2 + 1];
            sr += yr * c - yi * s;
            si += yr * s + yi * c;
        }
        out[2 * k] = sr;
        out[2 * k + 1] = si;
    }
    free(sub);
}

/* Unnormalised inverse 2D transform in place (Eq. 4): a[y][x] = sum_{v,u} G[v][u] exp(+2 pi i (u x + v y) / n).
 * Rows (u -> x) first, then columns (v -> y): the radix-2 transform above for a power of two, the
 * mixed-radix recursion for any other n.  Returns 0, or -1 for n < 1. */
int oracle_ifft2(double* a, int n)
{
    if (n <= 0) return -1;
    if ((n & (n - 1)) == 0) {
        for (int r = 0; r < n; r++) orc_ifft_1d(a + (int64_t)r * n * 2, n, 1);
        for (int col = 0; col < n; col++) orc_ifft_1d(a + (int64_t)col * 2, n, n);
        return 0;
    }
    double* root = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    double* line = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    for (int e = 0; e < n; e++) {
        double ang = ORC_TWO_PI * (double)e / (double)n;
        root[2 * e] = cos(ang);
        root[2 * e + 1] = sin(ang);
    }
    for (int r = 0; r < n; r++) {
        orc_idft_any(a + (int64_t)r * n * 2, 1, n, root, n, line);
        memcpy(a + (int64_t)r * n * 2, line, sizeof(double) * 2 * (size_t)n);
    }
    for (int col = 0; col < n; col++) {
        orc_idft_any(a + (int64_t)col * 2, n, n, root, n, line);
        for (int y = 0; y < n; y++) {
            a[((int64_t)y * n + col) * 2] = line[2 * y];
            a[((int64_t)y * n + col) * 2 + 1] = line[2 * y + 1];
        }
    }
    free(root);
    free(line);
    return 0;
}

/* The same transform as a direct sum (any n; O(n^4), for small sides).  The phase index (u x + v y) is
 * reduced modulo n in integers before the angle is formed. */
void oracle_idft2(const double* G, int n, double* a)
{
    for (int y = 0; y < n; y++)
        for (int x = 0; x < n; x++) {
            double sr = 0.0, si = 0.0;
            for (int v = 0; v < n; v++)
                for (int u = 0; u < n; u++) {
                    int64_t k = ((int64_t)u * x + (int64_t)v * y) % n;
                    double ang = ORC_TWO_PI * (double)k / (double)n;
                    double c = cos(ang), s = sin(ang);
                    double gr = G[((int64_t)v * n + u) * 2], gi = G[((int64_t)v * n + u) * 2 + 1];
                    sr += gr * c - gi * s;
                    si += gr * s + gi * c;
                }
            a[((int64_t)y * n + x) * 2] = sr;
            a[((int64_t)y * n + x) * 2 + 1] = si;
        }
}

/* Selected pixels of the dirty image of a grid, summed directly (Eq. 4 and the shift of oracle_image):
 * out[i] = Re a[(y_i + n/2) mod n][(x_i + n/2) mod n] / W with a[Y][X] = sum G[v][u] exp(+2 pi i (u X + v Y) / n),
 * the sum taken over the grid's nonzero cells only (a gridded image has few), the phase index reduced
 * modulo n in integers.  G: complex double [n][n]; yx: int32 [n_px][2] (y, x). */
void oracle_image_pixels(const double* G, int n, double W, const int32_t* yx, int64_t n_px, double* out)
{
    int64_t nz = 0;
    for (int64_t c = 0; c < (int64_t)n * n; c++)
        if (G[2 * c] != 0.0 || G[2 * c + 1] != 0.0) nz++;
    int32_t* cu = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nz > 0 ? nz : 1));
    int32_t* cv = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nz > 0 ? nz : 1));
    int64_t k = 0;
    for (int v = 0; v < n; v++)
        for (int u = 0; u < n; u++)
            if (G[((int64_t)v * n + u) * 2] != 0.0 || G[((int64_t)v * n + u) * 2 + 1] != 0.0) {
                cu[k] = u;
                cv[k] = v;
                k++;
            }
    int h = n / 2;
    for (int64_t i = 0; i < n_px; i++) {
        int64_t X = (yx[2 * i + 1] + h) % n, Y = (yx[2 * i] + h) % n;
        double sr = 0.0;
        for (int64_t c = 0; c < nz; c++) {
            int64_t e = ((int64_t)cu[c] * X + (int64_t)cv[c] * Y) % n;
            double ang = ORC_TWO_PI * (double)e / (double)n;
            const double* g = G + ((int64_t)cv[c] * n + cu[c]) * 2;
            sr += g[0] * cos(ang) - g[1] * sin(ang);
        }
        out[i] = sr / W;
    }
    free(cu);
    free(cv);
}

/* Dirty image (Sec. 5.2.4): img[y][x] = Re a[(y + N/2) mod N][(x + N/2) mod N] / W, which puts the phase
 * centre (l = m = 0) at pixel (N/2, N/2).  Returns max |Im a| / W, which is zero up to rounding for a
 * Hermitian grid. */
double oracle_image(const double* a, int n, double W, double* img)
{
    int h = n / 2;
    double mx = 0.0;
    for (int y = 0; y < n; y++)
        for (int x = 0; x < n; x++) {
            const double* s = a + ((int64_t)((y + h) % n) * n + (x + h) % n) * 2;
            img[(int64_t)y * n + x] = s[0] / W;
            double m = fabs(s[1]) / W;
            if (m > mx) mx = m;
        }
    return mx;
}

/*
 * The whole path for a list of images of one set (one flag vector, one image side): for each image id
 * (= tau * F + f) correlate, compute uvw and cells at the output channel's frequency, grid, transform and
 * form the image.  cell_lambda <= 0 selects the default cell over the set's highest output frequency.
 * support >= 2 (at most 16) grids with the Kaiser-Bessel kernel of that many cells on a grid of side 2N
 * (oracle_grid_kb; `grids` then holds [n_ids][2N][2N][2]) and keeps the corrected central N x N image
 * (oracle_kb_crop_correct); 0 or 1 grids to the nearest cell.  (phase_l, phase_m) != (0, 0) phase-centres
 * the sums on that pointing (oracle_uvw_phased, oracle_apply_phase) before gridding.
 * gains (or NULL): complex double [F][n_tiles][2 pol][2], applied to the sums before gridding; with
 * full_jones, complex double [F][n_tiles][2][2][2] full Jones matrices instead.
 * Optional outputs (NULL to skip): grids [n_ids][N][N][2], images [n_ids][N][N], W [n_ids],
 * max|Im|/W [n_ids].  Images are independent, so they are spread over `n_threads` OpenMP threads.
 * Returns 0, or -1 on bad arguments.
 */
int oracle_pipeline(const uint8_t* volt, int64_t fine_stride, int n_tiles, int n_fine, int c, int ns,
                    const double* enu, const double* fine_freq, const uint8_t* flags,
                    int n_pix, double cell_lambda, int pol, int autos, int support, double phase_l,
                    double phase_m, const double* gains, int full_jones,
                    const int64_t* ids, int64_t n_ids, int n_threads,
                    double* grids, double* imgs, double* W_out, double* maxim_out)
{
    if (n_pix <= 2 || (n_pix & 1) || c <= 0 || ns <= 0 || n_fine % c) return -1;
    if (!(phase_l * phase_l + phase_m * phase_m < 1.0)) return -1;
    int phased = phase_l != 0.0 || phase_m != 0.0;
    if (support >= 2 && (support > 16 || (double)(n_pix - 1) - 0.5 * (double)support <= 0.0)) return -1;
    int ng = support >= 2 ? 2 * n_pix : n_pix;      /* grid side */
    int F = n_fine / c;
    double* fout = (double*)malloc(sizeof(double) * F);
    oracle_output_freqs(fine_freq, n_fine, c, fout);
    double numax = fout[0];
    for (int f = 1; f < F; f++) if (fout[f] > numax) numax = fout[f];
    double du = cell_lambda > 0.0 ? cell_lambda
                                  : oracle_default_cell(enu, n_tiles, flags, numax, n_pix, support, phase_l, phase_m);
    int64_t B = oracle_n_baselines(n_tiles);
    int K = ns * c;
    int bad = 0;
#pragma omp parallel for num_threads(n_threads) schedule(dynamic, 1)
    for (int64_t q = 0; q < n_ids; q++) {
        int tau = (int)(ids[q] / F), f = (int)(ids[q] % F);
        int64_t* S = (int64_t*)malloc(sizeof(int64_t) * B * 8);
        double* uvw = (double*)malloc(sizeof(double) * B * 3);
        int32_t* iu = (int32_t*)malloc(sizeof(int32_t) * B);
        int32_t* iv = (int32_t*)malloc(sizeof(int32_t) * B);
        uint8_t* keep = (uint8_t*)malloc(B);
        double* G = (double*)malloc(sizeof(double) * 2 * ng * ng);
        double* im = (double*)malloc(sizeof(double) * ng * ng);
        oracle_correlate_one(volt, fine_stride, n_tiles, ns, c, tau, f, flags, S);
        if (phased)
            oracle_uvw_phased(enu, n_tiles, fout[f], phase_l, phase_m, uvw);
        else
            oracle_uvw(enu, n_tiles, fout[f], uvw);
        oracle_cells(uvw, B, du, n_pix, iu, iv, keep);
        double W;
        /* the sums as complex doubles when anything changes them: calibration, then the phase rotation */
        double* V = NULL;
        if (gains || phased || support >= 2) {
            V = (double*)malloc(sizeof(double) * B * 8);
            if (gains && full_jones)
                oracle_apply_jones(S, n_tiles, gains + (int64_t)f * n_tiles * 8, V);
            else if (gains)
                oracle_apply_gains(S, n_tiles, gains + (int64_t)f * n_tiles * 4, V);
            else
                for (int64_t e = 0; e < B * 8; e++) V[e] = (double)S[e];
            if (phased) oracle_apply_phase(V, uvw, B);
        }
        if (support >= 2)
            W = oracle_grid_kb(V, n_tiles, flags, K, pol, autos, uvw, du, support, ng, G);
        else if (V)
            W = oracle_grid_v(V, n_tiles, flags, K, pol, autos, iu, iv, keep, n_pix, G);
        else
            W = oracle_grid(S, n_tiles, flags, K, pol, autos, iu, iv, keep, n_pix, G);
        free(V);
        if (grids) memcpy(grids + q * 2 * ng * ng, G, sizeof(double) * 2 * ng * ng);
        if (oracle_ifft2(G, ng)) bad = 1;
        double mx = oracle_image(G, ng, W > 0.0 ? W : 1.0, im);
        if (imgs && support >= 2)
            oracle_kb_crop_correct(im, n_pix, support, imgs + q * n_pix * n_pix);
        else if (imgs)
            memcpy(imgs + q * n_pix * n_pix, im, sizeof(double) * n_pix * n_pix);
        if (W_out) W_out[q] = W;
        if (maxim_out) maxim_out[q] = mx;
        free(S); free(uvw); free(iu); free(iv); free(keep); free(G); free(im);
    }
    free(fout);
    return bad ? -1 : 0;
}

/*
 * Incoherent dedispersion of an image cube (the FRB search the images feed, Sec. 2, 7): img is double
 * [T][F][P] (integration, channel, pixel), d[f] >= 0 the delay of channel f in integrations; for every
 * t < T - max(d), out[t][p] = (1/F) sum_f img[t + d_f][f][p].  Zero delays give the band-averaged image.
 * Returns the number of output integrations, or -1 on bad arguments.
 */
int oracle_dedisperse(const double* img, int T, int F, int64_t P, const int32_t* d, double* out)
{
    if (T < 1 || F < 1 || P < 1) return -1;
    int dmax = 0;
    for (int f = 0; f < F; f++) {
        if (d[f] < 0) return -1;
        if (d[f] > dmax) dmax = d[f];
    }
    int To = T - dmax;
    if (To < 1) return -1;
    for (int t = 0; t < To; t++) {
        for (int64_t p = 0; p < P; p++) {
            double acc = 0.0;
            for (int f = 0; f < F; f++) acc += img[((int64_t)(t + d[f]) * F + f) * P + p];
            out[(int64_t)t * P + p] = acc / (double)F;
        }
    }
    return To;
}

