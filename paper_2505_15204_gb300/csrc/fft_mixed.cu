// Imaging (gridding + Eq. 4's inverse 2D transform; Sec. 5.2.4) for image sides the side-specialised
// kernels do not cover: any even side N = 2^a 3^b 5^c up to 8192 (1200, 2400, 4096, 8192, ...).
//
// Two launches per wave of images, the column results kept in L2 between them when the wave fits:
//   column pass  one CTA per `cw` consecutive u columns of the half plane: the columns' cells are gathered
//                (or read from a stored grid), multiplied by (-1)^(u+v) (the shift by N/2), transformed
//                along v by an N-point mixed-radix FFT in shared memory and written to H[y][u];
//   row pass     one CTA per `rb` image rows: the complex-to-real transform along u, formed from an
//                N/2-point complex FFT of the paired half spectrum, scaled by 1/W (and, with a convolution
//                kernel, cropped to the central half and grid-corrected).
// The FFT is a Stockham autosort iteration over the factors of the length (radices 16, 8, 4, 2, 3, 5) between two
// shared-memory buffers per transform: a thread reads a butterfly's inputs, transforms them in registers
// and writes the outputs to the other buffer in the next stage's order, so only one butterfly is live in
// registers at a time and blocks of many threads stay resident.
#include <algorithm>

#include "blink_internal.cuh"
#include "fft_ct.cuh"

namespace blink {

namespace {

constexpr int kMaxThreads = 1024;

__host__ __device__ __forceinline__ int pd(int i) { return i + (i >> 5); }     // one pad slot per 32 points

// v[p] *= w^p for 0 < p < R, with w^1, w^2, w^4, w^8 read from the table (tw[p e], each p e < n) and the
// other powers formed as products of at most three of them, so every factor carries the rounding of a few
// multiplications; only a handful of powers is live at a time.
template <int R>
__device__ __forceinline__ void twiddle(float2* v, const float2* __restrict__ tw, int e) {
    const float2 w1 = __ldg(tw + e);
    v[1] = cmul(v[1], w1);
    if (R <= 2) return;
    const float2 w2 = __ldg(tw + 2 * e);
    v[2] = cmul(v[2], w2);
    if (R <= 3) return;
    const float2 w3 = cmul(w1, w2);
    v[3] = cmul(v[3], w3);
    if (R <= 4) return;
    const float2 w4 = __ldg(tw + 4 * e);
    v[4] = cmul(v[4], w4);
    if (R <= 5) return;
    v[5] = cmul(v[5], cmul(w4, w1));
    v[6] = cmul(v[6], cmul(w4, w2));
    v[7] = cmul(v[7], cmul(w4, w3));
    if (R <= 8) return;
    const float2 w8 = __ldg(tw + 8 * e), w12 = cmul(w8, w4);
    v[8] = cmul(v[8], w8);
    v[9] = cmul(v[9], cmul(w8, w1));
    v[10] = cmul(v[10], cmul(w8, w2));
    v[11] = cmul(v[11], cmul(w8, w3));
    v[12] = cmul(v[12], w12);
    v[13] = cmul(v[13], cmul(w12, w1));
    v[14] = cmul(v[14], cmul(w12, w2));
    v[15] = cmul(v[15], cmul(w12, w3));
}

// One Stockham stage of radix R of an n-point transform after stages whose radices multiply to L, from
// buffer `in` to buffer `out`.  Point addresses: before the stage, Y(j, k1) (j < n/L, k1 < L) sits at
// j L + k1 and holds the L-point transform of the points j + (n/L) t; butterfly b = j' L + k1 (j' < n/(LR))
// reads Y(j' + m p, k1) for p < R (at b + p n/R, m = n/(LR)), multiplies input p by w_n^(p k1 m), transforms
// over p and writes output q to Y'(j', k1 + L q) at j' L R + k1 + L q.  tw[k * tws] = exp(+2 pi i k / n).
// A thread takes butterflies t, t + nt, ...: (j', k1) advance by (nt / L, nt % L) with a carry, so the
// stage divides once per thread, not once per butterfly.
template <int R>
__device__ __forceinline__ void stage(const float2* in, float2* out, int n, int L, const float2* __restrict__ tw,
                                      int tws, int t, int nt) {
    const int nb = n / R, m = nb / L;
    const int dj = nt / L, dk = nt - dj * L;
    int j = t / L, k1 = t - j * L;
    for (int b = t; b < nb; b += nt) {
        float2 v[R];
#pragma unroll
        for (int p = 0; p < R; p++) v[p] = in[pd(b + p * nb)];
        if (L > 1) twiddle<R>(v, tw, k1 * m * tws);
        idft<R>(v);
        const int d = j * L * R + k1;
#pragma unroll
        for (int q = 0; q < R; q++) out[pd(d + q * L)] = v[q];
        j += dj;
        k1 += dk;
        if (k1 >= L) {
            k1 -= L;
            j++;
        }
    }
    __syncthreads();
}

// The whole n-point transform of a[pd(0 .. n-1)] by the threads t < nt of each transform, alternating
// between the buffers a and b; radices packed 5 bits per stage, first stage lowest.  Every thread of the
// block runs the same stages.  Returns the buffer that holds the result.
__device__ __forceinline__ float2* fft_any(float2* a, float2* b, int n, uint64_t rad, int n_rad,
                                           const float2* __restrict__ tw, int tws, int t, int nt) {
    int L = 1;
    for (int k = 0; k < n_rad; k++) {
        const int R = (int)((rad >> (5 * k)) & 31u);
        switch (R) {
            case 16: stage<16>(a, b, n, L, tw, tws, t, nt); break;
            case 8: stage<8>(a, b, n, L, tw, tws, t, nt); break;
            case 4: stage<4>(a, b, n, L, tw, tws, t, nt); break;
            case 2: stage<2>(a, b, n, L, tw, tws, t, nt); break;
            case 3: stage<3>(a, b, n, L, tw, tws, t, nt); break;
            default: stage<5>(a, b, n, L, tw, tws, t, nt); break;
        }
        float2* x = a;
        a = b;
        b = x;
        L *= R;
    }
    return a;
}

// exp(+2 pi i k / n) for k < n: FP64 sincospi, rounded to FP32
__global__ void k_unit_roots(float2* out, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double sn, cs;
    sincospi(2.0 * (double)k / (double)n, &sn, &cs);
    out[k] = make_float2((float)cs, (float)sn);
}

struct MixedCol {
    int N, half, cw_log, nt, ld;           // grid side, N/2, log2(columns per CTA), threads per column, column stride
    uint64_t rad;
    int n_rad;
    const float2* tw;                      // exp(+2 pi i k / N), k < N
    // input: a stored half-plane grid [img][N][N/2 + 1] ...
    const float2* grid;
    // ... or the gather lists: item i's sums at vis + i * vstride, channel (first + i) % F, in baseline order
    // or (gathered) in the channel's entry order, planar (e_stride real parts, then e_stride imaginary parts).
    // Output o (o_first + blockIdx.y) sums the fa items (o / Fo) F + (o % Fo) fa + m, m < fa, each scaled by
    // 1 / (max(wk[channel], 1) fa) when wk is given (an average of normalised images), else by 1.
    const float2* vis;
    int64_t vstride;
    int gathered, e_stride;
    int first, F, o_first, fa, Fo;
    const float* wk;
    const int* ent_off;
    const uint2* ent;
    const float* wt;                       // per-entry kernel weights, or NULL (nearest cell)
    // output: rows [y0, y0 + ny) of the column transforms (all rows, or the central half with a kernel)
    void* H;
    int ldh, y0, ny;
};

// FIX = 1200: the side-1200 form, fixed plan (fft_ct.cuh): 80 threads per column, cw columns per CTA, columns
// unpadded in slots of kFixLd, the unit roots of 1200 copied to shared memory after the buffers.
constexpr int kFixLd = 1280;                       // column slots: >= kCol1200Slots, even
constexpr int kFixRowLd = 680;                     // row slots: >= kRow600Slots, even
constexpr int kFixCols = 4;                        // columns per CTA of the side-1200 column pass
constexpr int kFixRows = 8;                        // rows per CTA of the side-1200 row pass

// The gather of a column CTA's columns from its output's members (fa consecutive channels, or the image's own
// channel): a warp owns a column and adds the members' entries in member order, the members' column ranges,
// first chunks of entries and their sums loaded G at a time.  SHIFT: cells multiplied by (-1)^(u+v) (the image
// shift), else stored as they are.  GATH: sums in gather order, loaded beside their entries (one round trip
// fewer per G members).
template <int G, bool SHIFT, bool GATH, typename Idx>
__device__ __forceinline__ void gather_members(const MixedCol& P, int u0, int ncol, int it0, float2* s, Idx idx) {
    const int tid = threadIdx.x, lane = tid & 31;
    for (int c = tid >> 5; c < ncol; c += blockDim.x >> 5) {
        const int u = u0 + c;
        if (u >= P.half) continue;             // no cell reaches the Nyquist column
        for (int m0 = 0; m0 < P.fa; m0 += G) {
            int beg[G], end[G];
            float sc[G];
            const float2* V[G];
            const float* Vr[G];                // gathered: the member's real parts, indexed by the entry
#pragma unroll
            for (int g = 0; g < G; g++) {
                beg[g] = end[g] = 0;
                sc[g] = 1.0f;
                V[g] = P.vis;
                Vr[g] = nullptr;
                if (m0 + g < P.fa) {
                    const int it = it0 + m0 + g, f = (P.first + it) % P.F;
                    const int* off = P.ent_off + (int64_t)f * (P.half + 1);
                    beg[g] = off[u];
                    end[g] = off[u + 1];
                    V[g] = P.vis + (int64_t)it * P.vstride;
                    if constexpr (GATH) Vr[g] = reinterpret_cast<const float*>(V[g]) - off[0];
                    if (P.wk) sc[g] = 1.0f / (fmaxf(P.wk[f], 1.0f) * (float)P.fa);
                }
            }
            uint2 e[G];
            float2 xv[G];
#pragma unroll
            for (int g = 0; g < G; g++) {
                const int i = beg[g] + lane;
                if (i < end[g]) {
                    e[g] = P.ent[i];
                    if constexpr (GATH) xv[g] = make_float2(Vr[g][i], Vr[g][P.e_stride + i]);
                }
            }
            if constexpr (!GATH) {
#pragma unroll
                for (int g = 0; g < G; g++)
                    if (beg[g] + lane < end[g]) xv[g] = V[g][e[g].y];
            }
#pragma unroll
            for (int g = 0; g < G; g++) {
                if (m0 + g >= P.fa) break;
                const float2* Vg = V[g];
                const float* Vrg = Vr[g];
                const float scg = sc[g];
                auto val = [&](int i, uint32_t b) {
                    const float2 x = GATH ? make_float2(Vrg[i], Vrg[P.e_stride + i]) : Vg[b];
                    return make_float2(x.x * scg, x.y * scg);
                };
                // the member's first chunk as gather_entry forms it, from the values loaded above
                uint32_t key = 0xFFFFFFFFu;
                float2 x = make_float2(0.f, 0.f);
                const int i = beg[g] + lane;
                if (i < end[g]) {
                    key = ent_cell(e[g].x);
                    x = make_float2(xv[g].x * scg, xv[g].y * scg);
                    if (e[g].x >> 31) x.y = -x.y;
                    if (P.wt) {
                        const float w = P.wt[i];
                        x = make_float2(x.x * w, x.y * w);
                    }
                }
                warp_gather_column(P.ent, P.wt, beg[g], end[g], lane, s, val, idx, SHIFT, key, x);
            }
        }
    }
}

// The grids of averaged outputs over many channels, summed in global memory (zeroed by the caller) with one
// warp per column of the half plane, so that every warp of the GPU gathers (inside the column pass one warp per
// column does, while the rest of its CTA waits).  Per cell the members are added in the same order as there;
// cells are stored unshifted, for the column pass's grid input; the Nyquist column stays zero.
constexpr int kAvgGridWarps = 8;
__global__ void __launch_bounds__(32 * kAvgGridWarps) k_avg_grid(const MixedCol P, float2* grid) {
    const int img = blockIdx.y, u0 = blockIdx.x * kAvgGridWarps;
    const int ncol = min(kAvgGridWarps, P.half + 1 - u0);
    const int o = P.o_first + img;
    const int it0 = (o / P.Fo) * P.F + (o % P.Fo) * P.fa;
    float2* G = grid + (int64_t)img * P.N * (P.half + 1);
    auto idx = [&](int u, int v) { return (int64_t)v * (P.half + 1) + u; };
    if (P.gathered)
        gather_members<8, false, true>(P, u0, ncol, it0, G, idx);
    else
        gather_members<8, false, false>(P, u0, ncol, it0, G, idx);
}

template <typename T, int FIX>
__global__ void __launch_bounds__(FIX ? kFixCols * kCol1200Threads : kMaxThreads / 2, 2) k_mixed_col(const MixedCol P) {
    extern __shared__ float2 s[];          // [cw][ld] transform inputs, then [cw][ld] the second buffers
    const int img = blockIdx.y, tid = threadIdx.x, nthr = blockDim.x;
    static_assert(!FIX || kFixCols == 4, "the side-1200 form takes four columns per CTA");
    const int cw_log = FIX ? 2 : P.cw_log;
    const int cw = 1 << cw_log, u0 = blockIdx.x * cw;
    const int ncol = min(cw, P.half + 1 - u0);
    const int ld = FIX ? kFixLd : P.ld;
    auto pv = [&](int v) { return FIX ? v : pd(v); };      // a point's slot in a column
    float2* roots = s + 2 * cw * ld;
    if constexpr (FIX != 0)
        for (int e = tid; e < FIX; e += nthr) roots[e] = __ldg(P.tw + e);
    if (P.grid) {
        const float2* G = P.grid + (int64_t)img * P.N * (P.half + 1);
        for (int e = tid; e < P.N * cw; e += nthr) {
            const int v = e >> cw_log, c = e & (cw - 1), u = u0 + c;
            float2 x = make_float2(0.f, 0.f);
            if (c < ncol) {
                x = G[(int64_t)v * (P.half + 1) + u];
                if ((u + v) & 1) x = make_float2(-x.x, -x.y);
            }
            s[c * ld + pv(v)] = x;
        }
    } else {
        for (int e = tid; e < cw * ld; e += nthr) s[e] = make_float2(0.f, 0.f);
        __syncthreads();
        const int o = P.o_first + img;
        const int it0 = (o / P.Fo) * P.F + (o % P.Fo) * P.fa;
        auto idx = [&](int u, int v) { return (u - u0) * ld + pv(v); };
        // A warp owns a column and adds its members' entries in member order (reproducible sums); with an
        // average the members' column ranges, first chunks of entries and their sums are loaded kMembers at a
        // time, so an average over many channels costs a few load round trips per kMembers members.
        constexpr int GM = FIX ? 8 : 4;
        if (P.fa == 1)
            P.gathered ? gather_members<1, true, true>(P, u0, ncol, it0, s, idx)
                       : gather_members<1, true, false>(P, u0, ncol, it0, s, idx);
        else
            P.gathered ? gather_members<GM, true, true>(P, u0, ncol, it0, s, idx)
                       : gather_members<GM, true, false>(P, u0, ncol, it0, s, idx);
    }
    __syncthreads();
    int off;                                          // the result buffer's offset, the same for every column
    if constexpr (FIX == 1200) {
        const int c = tid / kCol1200Threads, t = tid - c * kCol1200Threads;
        fft1200_cols(s + c * ld, s + (cw + c) * ld, roots, t, [] { __syncthreads(); });
        off = cw * ld;
    } else {
        const int c = tid / P.nt, t = tid - c * P.nt;
        const float2* res = fft_any(s + c * ld, s + (cw + c) * ld, P.N, P.rad, P.n_rad, P.tw, 1, t, P.nt);
        off = (int)(res - (s + c * ld));
    }
    T* H = static_cast<T*>(P.H) + (int64_t)img * P.ny * P.ldh + u0;
    for (int e = tid; e < P.ny * cw; e += nthr) {
        const int r = e >> cw_log, cc = e & (cw - 1);
        if (cc < ncol) st_c(H + (int64_t)r * P.ldh + cc, s[off + cc * ld + pv(P.y0 + r)]);
    }
}

struct MixedRow {
    int N, M, nt, rb, ld;                  // grid side, N/2, threads per row, rows per CTA, row stride
    uint64_t rad;
    int n_rad;
    const float2* tw;                      // exp(+2 pi i k / N), k < N
    const void* H;
    int ldh, ny, has_nyq;                  // H rows per image; has_nyq: column u = N/2 holds data
    const float* wts;
    int w_mod;
    WaveMap wm;
    int out_first;
    int x0, nout;                          // output columns [x0, x0 + nout) of each row; image side nout
    const float* corr;                     // grid correction per output pixel index, or NULL
    float* img;
};

// With M = N/2 and the half spectrum Z[0..M] of a row, x[n] = sum_k Z[k] exp(+2 pi i k n / N) for the real
// sequence x is x[2m] = Re y[m], x[2m+1] = Im y[m] with y the M-point inverse transform of
// Y[k] = (Z[k] + conj Z[M-k]) + i (Z[k] - conj Z[M-k]) exp(+2 pi i k / N)  (any M, odd included).
template <typename T, int FIX>
__global__ void __launch_bounds__(FIX ? kFixRows * kRow600Threads : kMaxThreads / 2, 2) k_mixed_row(const MixedRow P) {
    extern __shared__ float2 s[];          // [rb][ld] transform inputs, then [rb][ld] the second buffers
    const int img = blockIdx.y, tid = threadIdx.x;
    const int nt = FIX ? kRow600Threads : P.nt, rb = FIX ? kFixRows : P.rb, ld = FIX ? kFixRowLd : P.ld;
    const int r = tid / nt, t = tid - r * nt, y = blockIdx.x * rb + r;
    const int M = FIX ? FIX / 2 : P.M;
    auto pv = [&](int k) { return FIX ? k : pd(k); };
    float2* roots = s + 2 * rb * ld;                 // FIX: exp(+2 pi i x / M), x < M
    if constexpr (FIX != 0)
        for (int e = tid; e < M; e += blockDim.x) roots[e] = __ldg(P.tw + 2 * e);
    float2* dst = s + r * ld;
    const T* row = static_cast<const T*>(P.H) + ((int64_t)img * P.ny + y) * P.ldh;
    if constexpr (FIX != 0) {
        // every load of the thread's share of the row first, then the pre-twiddles
        constexpr int MF = FIX / 2, KN = (MF / 2 + kRow600Threads) / kRow600Threads;
        float2 zk[KN], zm[KN], wk[KN], wm[KN];
#pragma unroll
        for (int i = 0; i < KN; i++) {
            const int k = t + i * kRow600Threads;
            if (k <= MF / 2) {
                zk[i] = ld_c(row + k);
                zm[i] = k == 0 ? (P.has_nyq ? ld_c(row + MF) : make_float2(0.f, 0.f)) : ld_c(row + (MF - k));
                wk[i] = __ldg(P.tw + k);
                wm[i] = __ldg(P.tw + (MF - k));
            }
        }
#pragma unroll
        for (int i = 0; i < KN; i++) {
            const int k = t + i * kRow600Threads;
            if (k <= MF / 2) {
                dst[k] = cadd(cadd(zk[i], conjf2(zm[i])), cmul_i(cmul(csub(zk[i], conjf2(zm[i])), wk[i])));
                if (k > 0 && k < MF - k)
                    dst[MF - k] = cadd(cadd(zm[i], conjf2(zk[i])), cmul_i(cmul(csub(zm[i], conjf2(zk[i])), wm[i])));
            }
        }
    } else {
    for (int k = t; k <= M / 2; k += nt) {
        const float2 zk = ld_c(row + k);
        const float2 zm = (k == 0) ? (P.has_nyq ? ld_c(row + M) : make_float2(0.f, 0.f)) : ld_c(row + (M - k));
        dst[pv(k)] = cadd(cadd(zk, conjf2(zm)), cmul_i(cmul(csub(zk, conjf2(zm)), __ldg(P.tw + k))));
        if (k > 0 && k < M - k)
            dst[pv(M - k)] = cadd(cadd(zm, conjf2(zk)), cmul_i(cmul(csub(zm, conjf2(zk)), __ldg(P.tw + (M - k)))));
    }
    }
    __syncthreads();
    const float2* res;
    if constexpr (FIX == 1200) {
        fft600_rows(dst, s + (rb + r) * ld, roots, t, [] { __syncthreads(); });
        res = s + (rb + r) * ld;
    } else {
        res = fft_any(dst, s + (rb + r) * ld, M, P.rad, P.n_rad, P.tw, 2, t, nt);
    }
    const int id = P.wm.id(img);
    const float w = P.wts ? P.wts[id % P.w_mod] : 1.f;
    float scale = 1.0f / (w > 0.f ? w : 1.f);
    if (P.corr) scale *= P.corr[y];
    float* out = P.img + ((int64_t)(id - P.out_first) * P.ny + y) * P.nout;
    if (!P.corr && (P.nout & 3) == 0 && (reinterpret_cast<uintptr_t>(P.img) & 15) == 0) {
        // whole rows (x0 = 0) on a 16-byte aligned output: four pixels, two results y[m], per 16-byte store
        float4* o4 = reinterpret_cast<float4*>(out);
        for (int q = t; q < P.nout / 4; q += nt) {
            const float2 a = res[pv(2 * q)], b = res[pv(2 * q + 1)];
            o4[q] = make_float4(a.x * scale, a.y * scale, b.x * scale, b.y * scale);
        }
        return;
    }
    for (int x = t; x < P.nout; x += nt) {
        const int X = P.x0 + x;
        const float2 z = res[pv(X >> 1)];
        const float a = (X & 1) ? z.y : z.x;
        out[x] = P.corr ? a * scale * P.corr[x] : a * scale;
    }
}

// radices of n in stage order (16s, then one 8, 4 or 2, then 3s and 5s), packed 5 bits each; false if n has
// another prime factor
bool factor(int n, uint64_t* rad, int* n_rad) {
    int k = 0;
    uint64_t r = 0;
    auto push = [&](int x) {
        r |= (uint64_t)x << (5 * k);
        k++;
    };
    while (n % 16 == 0 && k < 12) { push(16); n /= 16; }
    for (int x : {8, 4, 2})
        if (n % x == 0 && k < 12) { push(x); n /= x; }
    while (n % 3 == 0 && k < 12) { push(3); n /= 3; }
    while (n % 5 == 0 && k < 12) { push(5); n /= 5; }
    *rad = r;
    *n_rad = k;
    return n == 1;
}

int stride_for(int n) { return (pd(n - 1) + 1 + 15) / 16 * 16 + 1; }     // odd: columns spread over banks

struct Shape {
    uint64_t rad_c = 0, rad_r = 0;
    int nrad_c = 0, nrad_r = 0, nt_c = 0, nt_r = 0, cw_log = 0, rb = 1, ld_c = 0, ld_r = 0;   // threads per transform, ...
    size_t smem_c = 0, smem_r = 0;
};

bool shape_for(int N, Shape* sh) {
    if (N < 4 || (N & 1) || N > 8192) return false;
    if (!factor(N, &sh->rad_c, &sh->nrad_c) || !factor(N / 2, &sh->rad_r, &sh->nrad_r)) return false;
    sh->ld_c = stride_for(N);
    sh->ld_r = stride_for(N / 2);
    const size_t col = 2 * (size_t)sh->ld_c * sizeof(float2), row = 2 * (size_t)sh->ld_r * sizeof(float2);
    // The passes are bound by instruction issue, not by occupancy: measured sweeps over threads per
    // transform and transforms per CTA (sides 1200 and 8192) favoured few threads per transform (about one
    // per 16 points for columns, one per 16 of the half-length row transform's, at least 64) and CTAs of
    // about 128 threads.
    auto pow2_floor = [](int x) {
        int p = 1;
        while (2 * p <= x) p *= 2;
        return p;
    };
    sh->nt_c = std::max(64, std::min(kMaxThreads / 2, pow2_floor(N / 16)));
    int cw_log = 0;
    while (cw_log < 3 && (sh->nt_c << (cw_log + 1)) <= 128 && (col << (cw_log + 1)) <= (size_t)100 * 1024) cw_log++;
    sh->cw_log = cw_log;
    sh->smem_c = col << cw_log;
    sh->nt_r = std::max(64, std::min(kMaxThreads / 2, pow2_floor(N / 32)));     // side 8192: 256 beat 512
    int rb = 1;
    while (2 * rb <= 8 && 2 * rb * sh->nt_r <= 128 && (N / 2) % (2 * rb) == 0 && 2 * rb * row <= (size_t)100 * 1024)
        rb *= 2;
    sh->rb = rb;
    sh->smem_r = row * rb;
    return sh->smem_c <= (size_t)227 * 1024 && sh->smem_r <= (size_t)227 * 1024;
}

}  // namespace

bool mixed_side_ok(int N) {
    Shape sh;
    return shape_for(N, &sh);
}

blink_status launch_avg_grid(const MixedIn& in, int n_out, float2* d_grid, cudaStream_t st) {
    if (n_out <= 0) return BLINK_OK;
    if (n_out > 65535) return set_error(BLINK_ERR_UNSUPPORTED, "wave of more than 65535 images");
    MixedCol C{};
    C.N = in.N;
    C.half = in.N / 2;
    C.tw = in.tw;
    C.vis = in.vis;
    C.vstride = in.vstride;
    C.gathered = in.gathered;
    C.e_stride = in.e_stride;
    C.first = in.first;
    C.F = in.F;
    C.o_first = in.o_first;
    C.fa = in.fa;
    C.Fo = in.F / in.fa;
    C.wk = in.wk;
    C.ent_off = in.ent_off;
    C.ent = in.ent;
    C.wt = in.wt;
    const dim3 g((in.N / 2 + 1 + kAvgGridWarps - 1) / kAvgGridWarps, n_out);
    k_avg_grid<<<g, 32 * kAvgGridWarps, 0, st>>>(C, d_grid);
    BLINK_CUDA(cudaGetLastError());
    return BLINK_OK;
}

blink_status make_unit_roots(float2* d_out, int N, cudaStream_t st) {
    k_unit_roots<<<(N + 255) / 256, 256, 0, st>>>(d_out, N);
    BLINK_CUDA(cudaGetLastError());
    return BLINK_OK;
}

size_t mixed_h_row(int N) { return ((size_t)N / 2 + 1 + 3) / 4 * 4; }

blink_status launch_mixed(const MixedIn& in, int pass, int prec, int n_images, void* d_H, const float* d_w, int w_mod,
                          WaveMap wm, int out_first, float* d_img, cudaStream_t st) {
    Shape sh;
    const int N = in.N;
    if (!shape_for(N, &sh)) return set_error(BLINK_ERR_UNSUPPORTED, "image side has a prime factor other than 2, 3, 5");
    if (n_images <= 0) return BLINK_OK;
    if (n_images > 65535) return set_error(BLINK_ERR_UNSUPPORTED, "wave of more than 65535 images");
    const bool crop = in.corr != nullptr;
    const int ny = crop ? N / 2 : N, y0 = crop ? N / 4 : 0;
    const bool bf16 = prec == BLINK_PREC_BF16;
    if (pass == 0) {
        MixedCol C{};
        C.N = N;
        C.half = N / 2;
        C.cw_log = sh.cw_log;
        C.nt = sh.nt_c;
        C.ld = sh.ld_c;
        C.rad = sh.rad_c;
        C.n_rad = sh.nrad_c;
        C.tw = in.tw;
        C.grid = in.grid;
        C.vis = in.vis;
        C.vstride = in.vstride;
        C.gathered = in.gathered;
        C.e_stride = in.e_stride;
        C.first = in.first;
        C.F = in.F;
        C.o_first = in.o_first;
        C.fa = in.fa;
        C.Fo = in.F / in.fa;
        C.wk = in.wk;
        C.ent_off = in.ent_off;
        C.ent = in.ent;
        C.wt = in.wt;
        C.H = d_H;
        C.ldh = (int)mixed_h_row(N);
        C.y0 = y0;
        C.ny = ny;
        if (N == 1200) {
            // the fixed plan: four columns of 80 threads per CTA, the unit roots beside the buffers
            const dim3 g((N / 2 + 1 + kFixCols - 1) / kFixCols, n_images);
            const size_t smem = (size_t)(2 * kFixCols * kFixLd + 1200) * sizeof(float2);
            if (bf16) {
                BLINK_TRY(kernel_smem((const void*)k_mixed_col<__nv_bfloat162, 1200>, smem));
                k_mixed_col<__nv_bfloat162, 1200><<<g, kFixCols * kCol1200Threads, smem, st>>>(C);
            } else {
                BLINK_TRY(kernel_smem((const void*)k_mixed_col<float2, 1200>, smem));
                k_mixed_col<float2, 1200><<<g, kFixCols * kCol1200Threads, smem, st>>>(C);
            }
            BLINK_CUDA(cudaGetLastError());
            return BLINK_OK;
        }
        const int cw = 1 << sh.cw_log;
        const dim3 g((N / 2 + 1 + cw - 1) / cw, n_images);
        if (bf16) {
            BLINK_TRY(kernel_smem((const void*)k_mixed_col<__nv_bfloat162, 0>, sh.smem_c));
            k_mixed_col<__nv_bfloat162, 0><<<g, sh.nt_c * cw, sh.smem_c, st>>>(C);
        } else {
            BLINK_TRY(kernel_smem((const void*)k_mixed_col<float2, 0>, sh.smem_c));
            k_mixed_col<float2, 0><<<g, sh.nt_c * cw, sh.smem_c, st>>>(C);
        }
    } else {
        MixedRow R{};
        R.N = N;
        R.M = N / 2;
        R.nt = sh.nt_r;
        R.rb = sh.rb;
        R.ld = sh.ld_r;
        R.rad = sh.rad_r;
        R.n_rad = sh.nrad_r;
        R.tw = in.tw;
        R.H = d_H;
        R.ldh = (int)mixed_h_row(N);
        R.ny = ny;
        R.has_nyq = in.grid != nullptr;
        R.wts = d_w;
        R.w_mod = w_mod;
        R.wm = wm;
        R.out_first = out_first;
        R.x0 = y0;
        R.nout = ny;
        R.corr = in.corr;
        R.img = d_img;
        if (N == 1200 && ny % kFixRows == 0) {
            // the fixed plan: eight rows of 40 threads per CTA, the unit roots of 600 beside the buffers
            const dim3 g(ny / kFixRows, n_images);
            const size_t smem = (size_t)(2 * kFixRows * kFixRowLd + 600) * sizeof(float2);
            if (bf16) {
                BLINK_TRY(kernel_smem((const void*)k_mixed_row<__nv_bfloat162, 1200>, smem));
                k_mixed_row<__nv_bfloat162, 1200><<<g, kFixRows * kRow600Threads, smem, st>>>(R);
            } else {
                BLINK_TRY(kernel_smem((const void*)k_mixed_row<float2, 1200>, smem));
                k_mixed_row<float2, 1200><<<g, kFixRows * kRow600Threads, smem, st>>>(R);
            }
            BLINK_CUDA(cudaGetLastError());
            return BLINK_OK;
        }
        if (ny % sh.rb) return set_error(BLINK_ERR_UNSUPPORTED, "row blocking of the mixed-radix row pass");
        const dim3 g(ny / sh.rb, n_images);
        if (bf16) {
            BLINK_TRY(kernel_smem((const void*)k_mixed_row<__nv_bfloat162, 0>, sh.smem_r));
            k_mixed_row<__nv_bfloat162, 0><<<g, sh.nt_r * sh.rb, sh.smem_r, st>>>(R);
        } else {
            BLINK_TRY(kernel_smem((const void*)k_mixed_row<float2, 0>, sh.smem_r));
            k_mixed_row<float2, 0><<<g, sh.nt_r * sh.rb, sh.smem_r, st>>>(R);
        }
    }
    BLINK_CUDA(cudaGetLastError());
    return BLINK_OK;
}

}  // namespace blink
