// C ABI entry points, argument validation, plans and workspace.
#include <algorithm>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "blink_internal.cuh"
#include "kb_lists.h"

namespace blink {

int col_block_width(int N);

static thread_local std::string g_err;

blink_status set_error(blink_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

blink_status cuda_error(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? BLINK_ERR_OOM : BLINK_ERR_CUDA;
}

// Argument checks shared by the entry points (also used by blink_image_noalloc).
blink_status check_imaging(const blink_imaging* im) {
    if (!im) return set_error(BLINK_ERR_INVALID_ARG, "imaging descriptor is NULL");
    const int n = im->n_pix;
    if (n < 64 || n > 8192 || !mixed_side_ok(n))
        return set_error(BLINK_ERR_UNSUPPORTED, "imaging.n_pix must be even, in [64, 8192], with no prime factor above 5");
    if (im->pol != BLINK_POL_I && im->pol != BLINK_POL_XX)
        return set_error(BLINK_ERR_INVALID_ARG, "imaging.pol must be BLINK_POL_I or BLINK_POL_XX");
    if (im->precision != BLINK_PREC_FP32 && im->precision != BLINK_PREC_BF16)
        return set_error(BLINK_ERR_INVALID_ARG, "imaging.precision must be BLINK_PREC_FP32 or BLINK_PREC_BF16");
    if (!std::isfinite(im->cell_lambda)) return set_error(BLINK_ERR_INVALID_ARG, "imaging.cell_lambda is not finite");
    if (im->support < 0 || im->support > 16)
        return set_error(BLINK_ERR_INVALID_ARG, "imaging.support must be 0 or 1 (nearest cell) or a kernel width in [2, 16]");
    if (im->support >= 2 && n > 4096)
        return set_error(BLINK_ERR_UNSUPPORTED, "with a convolution kernel imaging.n_pix is at most 4096 (grid side 2 n_pix)");
    if (!std::isfinite(im->phase_l) || !std::isfinite(im->phase_m) ||
        !(im->phase_l * im->phase_l + im->phase_m * im->phase_m < 1.0))
        return set_error(BLINK_ERR_INVALID_ARG, "imaging.phase_l, phase_m must be direction cosines with l^2 + m^2 < 1");
    return BLINK_OK;
}

// The entry points that grid to the nearest cell only (stage calls and the plain per-image form).
blink_status nearest_only(const blink_imaging* im, const char* what) {
    if (im && im->support >= 2)
        return set_error(BLINK_ERR_UNSUPPORTED, std::string(what) + ": gridding with a convolution kernel runs in the "
                                                "batched pipeline forms only");
    return BLINK_OK;
}

namespace {

constexpr double kSpeedOfLight = 299792458.0;

struct Hasher {
    uint64_t h = 1469598103934665603ull;
    void bytes(const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; i++) {
            h ^= c[i];
            h *= 1099511628211ull;
        }
    }
    template <typename T> void val(T v) { bytes(&v, sizeof(v)); }
};

blink_status check_array(const blink_array* a) {
    if (!a) return set_error(BLINK_ERR_INVALID_ARG, "array descriptor is NULL");
    if (a->n_tiles < 1 || a->n_tiles > 512) return set_error(BLINK_ERR_INVALID_ARG, "n_tiles must be in [1, 512]");
    if (!a->enu_m) return set_error(BLINK_ERR_INVALID_ARG, "array.enu_m is NULL");
    for (int i = 0; i < 3 * a->n_tiles; i++)
        if (!std::isfinite(a->enu_m[i])) return set_error(BLINK_ERR_INVALID_ARG, "array.enu_m has a non-finite value");
    return BLINK_OK;
}


blink_status check_obs(const blink_obs* o, bool need_freq) {
    if (!o) return set_error(BLINK_ERR_INVALID_ARG, "obs descriptor is NULL");
    if (o->n_fine < 1) return set_error(BLINK_ERR_INVALID_ARG, "obs.n_fine must be >= 1");
    if (o->fine_stride != 0 && o->fine_stride < o->n_fine)
        return set_error(BLINK_ERR_INVALID_ARG, "obs.fine_stride must be 0 or >= n_fine");
    if (o->chan_avg < 1 || o->n_fine % o->chan_avg)
        return set_error(BLINK_ERR_INVALID_ARG, "obs.chan_avg must be >= 1 and divide n_fine");
    if (o->samples_per_int < 1) return set_error(BLINK_ERR_INVALID_ARG, "obs.samples_per_int must be >= 1");
    if (o->n_samples < 0 || o->n_samples % o->samples_per_int)
        return set_error(BLINK_ERR_INVALID_ARG, "obs.n_samples must be a non-negative multiple of samples_per_int");
    if ((int64_t)(o->n_samples / o->samples_per_int) * (o->n_fine / o->chan_avg) > INT32_MAX)
        return set_error(BLINK_ERR_UNSUPPORTED, "more than 2^31 - 1 images (integrations x output channels) in one call");
    if ((int64_t)o->samples_per_int * o->chan_avg > 131072)
        return set_error(BLINK_ERR_UNSUPPORTED, "samples_per_int * chan_avg above 131072 (sums could leave the exact "
                                                "FP32 integer range)");
    if (need_freq) {
        if (!o->fine_freq_hz) return set_error(BLINK_ERR_INVALID_ARG, "obs.fine_freq_hz is NULL");
        for (int i = 0; i < o->n_fine; i++)
            if (!(o->fine_freq_hz[i] > 0.0) || !std::isfinite(o->fine_freq_hz[i]))
                return set_error(BLINK_ERR_INVALID_ARG, "obs.fine_freq_hz must be positive and finite");
    }
    return BLINK_OK;
}

bool off_zenith(const blink_imaging* im) { return im && (im->phase_l != 0.0 || im->phase_m != 0.0); }

// The pointing's basis (Sec. 5.2.3): e_l, e_m = East and North carried to s0 = (l0, m0, n0) by the rotation
// about Up x s0 that takes Up to s0 (Rodrigues' formula); e[0..2] = e_l, e[3..5] = e_m, e[6..8] = s0.
void pointing_basis(double l0, double m0, double* e) {
    const double r2 = l0 * l0 + m0 * m0, n0 = std::sqrt(1.0 - r2);
    e[6] = l0;
    e[7] = m0;
    e[8] = n0;
    if (r2 == 0.0) {
        const double id[6] = {1, 0, 0, 0, 1, 0};
        for (int k = 0; k < 6; k++) e[k] = id[k];
        return;
    }
    const double r = std::sqrt(r2), kx = -m0 / r, ky = l0 / r, c1 = 1.0 - n0;
    e[0] = n0 + kx * kx * c1;
    e[1] = kx * ky * c1;
    e[2] = -ky * r;
    e[3] = kx * ky * c1;
    e[4] = n0 + ky * ky * c1;
    e[5] = kx * r;
}

// blink_grid grids the caller's visibilities as they are: no phase centre.
blink_status zenith_only(const blink_imaging* im, const char* what) {
    if (off_zenith(im))
        return set_error(BLINK_ERR_UNSUPPORTED, std::string(what) + ": an off-zenith phase centre runs in the "
                                                "pipeline forms only");
    return BLINK_OK;
}

blink_status make_current(blink_context* ctx) {
    if (!ctx) return set_error(BLINK_ERR_INVALID_ARG, "context is NULL");
    int cur = -1;
    BLINK_CUDA(cudaGetDevice(&cur));
    if (cur != ctx->device) BLINK_CUDA(cudaSetDevice(ctx->device));
    return BLINK_OK;
}

template <typename T>
blink_status dmalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(plan)");
    return BLINK_OK;
}

void free_plan(Plan* p) {
    if (!p) return;
    cudaFree(p->d_bl);
    cudaFree(p->d_flags);
    cudaFree(p->d_enu);
    cudaFree(p->d_freq);
    cudaFree(p->d_cells);
    cudaFree(p->d_ent_off);
    cudaFree(p->d_ent);
    cudaFree(p->d_W);
    cudaFree(p->d_Wk);
    cudaFree(p->d_tw);
    cudaFree(p->d_wt);
    cudaFree(p->d_sep_off);
    cudaFree(p->d_sep);
    cudaFree(p->d_sep_w);
    cudaFree(p->d_corr);
    cudaFree(p->d_phase);
    cudaFree(p->d_gsrc);
    cudaFree(p->d_gpos);
    cudaFree(p->d_gphase);
    delete p;
}

// Output-channel centre = mean of its fine-channel centres, summed in order (host FP64, no contraction).
std::vector<double> output_freqs(const blink_obs* o) {
    const int F = o->n_fine / o->chan_avg;
    std::vector<double> out(F);
    for (int f = 0; f < F; f++) {
        double s = 0.0;
        for (int k = 0; k < o->chan_avg; k++) s += o->fine_freq_hz[f * o->chan_avg + k];
        out[f] = s / (double)o->chan_avg;
    }
    return out;
}

// Default uv cell: u_max / (N/2 - 1), u_max = longest unflagged projected baseline * nu_max / c, for a grid of
// side N; with a kernel of W cells the support must stay inside the grid too: u_max / (N/2 - 1 - W/2).
// Off zenith the baselines are projected on the pointing's (e_l, e_m) (`basis`, NULL at zenith).
double default_cell(const blink_array* a, double nu_max, int n_pix, int support, const double* basis) {
    double dmax = 0.0;
    for (int i = 0; i < a->n_tiles; i++)
        for (int j = 0; j < i; j++) {
            if (a->flags && (a->flags[i] || a->flags[j])) continue;
            double be = a->enu_m[i * 3 + 0] - a->enu_m[j * 3 + 0];
            double bn = a->enu_m[i * 3 + 1] - a->enu_m[j * 3 + 1];
            if (basis) {
                const double bu = a->enu_m[i * 3 + 2] - a->enu_m[j * 3 + 2], bx = be, by = bn;
                be = bx * basis[0] + by * basis[1] + bu * basis[2];
                bn = bx * basis[3] + by * basis[4] + bu * basis[5];
            }
            const double d = std::sqrt(be * be + bn * bn);
            if (d > dmax) dmax = d;
        }
    const double umax = dmax * (nu_max / kSpeedOfLight);
    if (!(umax > 0.0)) return 1.0;
    if (support >= 2) return umax / ((double)(n_pix / 2 - 1) - 0.5 * (double)support);
    return umax / (double)(n_pix / 2 - 1);
}

// Cell-sorted gather list of the u >= 0 half plane for every output channel: one entry per visibility (and
// per mirror) contribution that lands in the half plane, ordered by (u, v, baseline), with the offsets of
// every column u so that a column, or a block of consecutive columns, is one contiguous range.  A channel's
// contributions are collected as (key = u * N + v, (b << 1) | conj) and appended by `add_channel`.
struct GatherBuilder {
    int N, half;
    int64_t nkeys;
    std::vector<int> count, ent_off;
    std::vector<uint2> ent;
    std::vector<uint32_t> ekey, eval, sorted, skey;
    std::vector<std::vector<uint16_t>> gsrc;   // per channel: the baseline of each entry (nearest-cell lists only)
    std::vector<uint32_t> gpos;                // [F][B]: the entries of each baseline (positions below 0xFFFF)
    int64_t B = 0;
    bool src16 = false, pos16 = false;
    int max_per_channel = 0;
    GatherBuilder(int n, int F) : N(n), half(n / 2), nkeys((int64_t)(n / 2) * n), ent_off((size_t)F * (n / 2 + 1)) {}
    uint32_t key(int u, int v) const { return (uint32_t)((int64_t)u * N + v); }
    void clear() {
        ekey.clear();
        eval.clear();
    }
    // stable sort by key: the entries of a cell stay in the order they were added (a counting sort while
    // the keys are few next to the entries, a comparison sort on large grids)
    blink_status add_channel(int f) {
        if (count.empty() && nkeys <= (int64_t)16 * (int64_t)ekey.size() + 4096) count.assign(nkeys + 1, 0);
        sorted.assign(ekey.size(), 0);
        skey.assign(ekey.size(), 0);
        const int64_t base = (int64_t)ent.size();
        if (nkeys <= (int64_t)16 * (int64_t)ekey.size() + 4096) {
            std::fill(count.begin(), count.end(), 0);
            for (uint32_t k : ekey) count[k + 1]++;
            for (int64_t k = 0; k < nkeys; k++) count[k + 1] += count[k];
            std::vector<int> cur(count.begin(), count.end() - 1);
            for (size_t e = 0; e < ekey.size(); e++) {
                const int at = cur[ekey[e]]++;
                sorted[at] = eval[e];
                skey[at] = ekey[e];
            }
            for (int u = 0; u <= half; u++)
                ent_off[(size_t)f * (half + 1) + u] = (int)(base + count[std::min<int64_t>((int64_t)u * N, nkeys)]);
        } else {
            std::vector<uint32_t> ord(ekey.size());
            for (size_t e = 0; e < ord.size(); e++) ord[e] = (uint32_t)e;
            std::stable_sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t b) { return ekey[a] < ekey[b]; });
            for (size_t e = 0; e < ord.size(); e++) {
                sorted[e] = eval[ord[e]];
                skey[e] = ekey[ord[e]];
            }
            for (int u = 0; u <= half; u++)
                ent_off[(size_t)f * (half + 1) + u] =
                    (int)(base + (std::lower_bound(skey.begin(), skey.end(), (uint32_t)std::min<int64_t>((int64_t)u * N, nkeys)) -
                                  skey.begin()));
        }
        for (size_t e = 0; e < sorted.size(); e++) {
            const uint32_t u = skey[e] / N, v = skey[e] % N;
            ent.push_back(make_uint2(u | (v << 13) | ((sorted[e] & 1u) << 31), sorted[e] >> 1));
        }
        max_per_channel = std::max(max_per_channel, (int)sorted.size());
        if (src16) {
            std::vector<uint16_t>& g = gsrc[f];
            g.resize(sorted.size());
            for (size_t e = 0; e < sorted.size(); e++) g[e] = (uint16_t)(sorted[e] >> 1);
            if (sorted.size() < 0xFFFFu) {
                uint32_t* gp = gpos.data() + (size_t)f * B;
                for (size_t e = 0; e < sorted.size(); e++) {
                    uint32_t& w = gp[sorted[e] >> 1];
                    w = (w & 0xFFFFu) == 0xFFFFu ? ((w & 0xFFFF0000u) | (uint32_t)e) : ((w & 0xFFFFu) | ((uint32_t)e << 16));
                }
            } else {
                pos16 = false;
            }
        }
        if ((int64_t)ent.size() > INT32_MAX / 2) return set_error(BLINK_ERR_UNSUPPORTED, "gather list too large");
        return BLINK_OK;
    }
    blink_status upload(Plan* p) {
        p->n_contrib = (int64_t)ent.size();
        p->n_cells = p->n_contrib;
        BLINK_TRY(dmalloc(&p->d_ent_off, ent_off.size()));
        BLINK_TRY(dmalloc(&p->d_ent, ent.size()));
        BLINK_CUDA(cudaMemcpy(p->d_ent_off, ent_off.data(), ent_off.size() * sizeof(int), cudaMemcpyHostToDevice));
        if (!ent.empty())
            BLINK_CUDA(cudaMemcpy(p->d_ent, ent.data(), ent.size() * sizeof(uint2), cudaMemcpyHostToDevice));
        if (src16) {
            p->e_stride = std::max(8, (max_per_channel + 7) / 8 * 8);
            std::vector<uint16_t> all((size_t)gsrc.size() * p->e_stride, 0);
            for (size_t f = 0; f < gsrc.size(); f++)
                std::copy(gsrc[f].begin(), gsrc[f].end(), all.begin() + f * p->e_stride);
            BLINK_TRY(dmalloc(&p->d_gsrc, all.size()));
            BLINK_CUDA(cudaMemcpy(p->d_gsrc, all.data(), all.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
            if (pos16) {
                BLINK_TRY(dmalloc(&p->d_gpos, gpos.size()));
                BLINK_CUDA(cudaMemcpy(p->d_gpos, gpos.data(), gpos.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
            }
        }
        return BLINK_OK;
    }
};

// Nearest-cell gather list: every kept visibility in its cell, its mirror in the mirrored cell.
blink_status build_gather(Plan* p, const std::vector<uint32_t>& cells, const std::vector<short2>& bl,
                          const blink_array* a) {
    const int N = p->N;
    const int64_t B = p->B;
    GatherBuilder g(N, p->F);
    g.ent.reserve((size_t)p->F * (B + B / 16));
    g.src16 = B <= 0x10000;
    if (g.src16) {
        g.gsrc.resize(p->F);
        g.B = B;
        g.pos16 = true;
        g.gpos.assign((size_t)p->F * B, 0xFFFFFFFFu);
    }
    p->W.assign(p->F, 0.f);
    int64_t dropped = 0;
    for (int f = 0; f < p->F; f++) {
        g.clear();
        int64_t w = 0;
        auto add = [&](int u, int v, int64_t b, uint32_t conj) {
            g.ekey.push_back(g.key(u, v));
            g.eval.push_back((uint32_t)(b << 1) | conj);
        };
        for (int64_t b = 0; b < B; b++) {
            const uint32_t c = cells[(size_t)f * B + b];
            const int i = bl[b].x, j = bl[b].y;
            if (i == j) {
                if (c == CELL_NONE || !p->autos) continue;
                add(0, 0, b, 0);
                w += 1;
                continue;
            }
            if (c == CELL_NONE) {
                if (!(a->flags && (a->flags[i] || a->flags[j]))) dropped++;
                continue;
            }
            const int iu = (int16_t)(c & 0xFFFF), iv = (int16_t)(c >> 16);
            const int vpos = ((iv % N) + N) % N, vneg = ((-iv % N) + N) % N;
            if (iu > 0) {
                add(iu, vpos, b, 0);
            } else if (iu < 0) {
                add(-iu, vneg, b, 1);
            } else {
                add(0, vpos, b, 0);
                add(0, vneg, b, 1);
            }
            w += 2;
        }
        p->W[f] = (float)w;
        BLINK_TRY(g.add_channel(f));
    }
    p->n_dropped = dropped;
    return g.upload(p);
}

// ---- gridding with a convolution kernel (the kernel C(t) and its weights: kb_lists.h) ------------------
constexpr double kPi = 3.14159265358979323846;
static_assert(kSepMaxW == kSepRowW, "the kernel's row weights per record and the plan's agree");

// Its Fourier transform at nu cycles per cell (1 at nu = 0): with a = pi W nu and r = sqrt(|beta^2 - a^2|),
// (sinh r / r) / (sinh beta / beta) below a = beta and (sin r / r) / (sinh beta / beta) above.
double kb_transform(double nu, int W, double beta) {
    const double a = kPi * W * nu, d = beta * beta - a * a;
    const double r = std::sqrt(std::fabs(d));
    const double s = r == 0.0 ? 1.0 : (d > 0.0 ? std::sinh(r) / r : std::sin(r) / r);
    return s * beta / std::sinh(beta);
}

// Kernel gather list: a cross visibility at g = (u, v) / du is kept iff its support lies inside the grid
// (|gu|, |gv| <= N/2 - W/2); each support cell c (|c - g| < W/2 on both axes) gets weight C(cu - gu) C(cv - gv):
// the visibility's contribution at c lands in the half plane when cu > 0, its mirror's (conjugate, at -c)
// when cu < 0, both when cu = 0.  Autocorrelations sit at g = 0 without mirror; their cells with cu >= 0
// stand for the whole (real, symmetric) spread.  uvw: host [F][B][3] from the geometry kernel.
// Channels are independent: a first pass counts each channel's entries, a second sorts every channel into
// its own range of the list; both run on host threads, channel by channel, with the same result as in turn.
blink_status build_gather_kb(Plan* p, const std::vector<double>& uvw, const std::vector<short2>& bl,
                             const blink_array* a) {
    const int N = p->N, W = p->support, half = N / 2, F = p->F;
    const int64_t B = p->B, nkeys = (int64_t)half * N;
    const double beta = kb_beta(W), h = 0.5 * W, lim = 0.5 * N - h;
    // the cells within W/2 of x and, when `ws` is given, their weights
    auto support_cells = [&](double x, int* cs, double* ws) { return kb_support_cells(x, W, beta, cs, ws); };
    auto key = [&](int u, int v) { return (uint32_t)((int64_t)u * N + ((v % N) + N) % N); };
    // every half-plane contribution of channel f in baseline order: emit(key, (b << 1) | conj, weight)
    auto channel = [&](int f, bool weights, auto&& emit, int64_t& wsum, int64_t& dropped) {
        int cu[20], cv[20];
        double wu[20], wv[20];
        double* pu = weights ? wu : nullptr;
        double* pv = weights ? wv : nullptr;
        wsum = 0;
        dropped = 0;
        for (int64_t b = 0; b < B; b++) {
            const int i = bl[b].x, j = bl[b].y;
            if (a->flags && (a->flags[i] || a->flags[j])) continue;
            if (i == j) {
                if (!p->autos) continue;
                const int n = support_cells(0.0, cu, pu);
                for (int q = 0; q < n; q++)
                    for (int r = 0; r < n; r++)
                        if (cu[r] >= 0) emit(key(cu[r], cu[q]), (uint32_t)(b << 1), weights ? (float)(wu[r] * wu[q]) : 0.f);
                wsum += 1;
                continue;
            }
            const double gu = uvw[((size_t)f * B + b) * 3 + 0] / p->du, gv = uvw[((size_t)f * B + b) * 3 + 1] / p->du;
            if (!(std::fabs(gu) <= lim && std::fabs(gv) <= lim)) {
                dropped++;
                continue;
            }
            const int nu = support_cells(gu, cu, pu), nv = support_cells(gv, cv, pv);
            for (int q = 0; q < nv; q++)
                for (int r = 0; r < nu; r++) {
                    const float wgt = weights ? (float)(wu[r] * wv[q]) : 0.f;
                    if (cu[r] >= 0) emit(key(cu[r], cv[q]), (uint32_t)(b << 1), wgt);
                    if (cu[r] <= 0) emit(key(-cu[r], -cv[q]), (uint32_t)(b << 1) | 1u, wgt);
                }
            wsum += 2;
        }
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int n_thr = (int)std::min<unsigned>(std::min<unsigned>(hw, 16u), (unsigned)F);
    auto parallel = [&](auto&& body) {
        std::vector<std::thread> pool;
        for (int t = 0; t < n_thr; t++)
            pool.emplace_back([&, t] {
                for (int f = t; f < F; f += n_thr) body(f);
            });
        for (std::thread& th : pool) th.join();
    };
    std::vector<int64_t> n_ent(F), wsum(F), drop(F);
    parallel([&](int f) {
        int64_t c = 0;
        channel(f, false, [&](uint32_t, uint32_t, float) { c++; }, wsum[f], drop[f]);
        n_ent[f] = c;
    });
    std::vector<int64_t> base(F + 1, 0);
    for (int f = 0; f < F; f++) base[f + 1] = base[f] + n_ent[f];
    if (base[F] > INT32_MAX / 2) return set_error(BLINK_ERR_UNSUPPORTED, "gather list too large");
    std::vector<uint2> ent((size_t)base[F]);
    std::vector<float> wt((size_t)base[F]);
    std::vector<int> ent_off((size_t)F * (half + 1));
    parallel([&](int f) {
        std::vector<uint32_t> ekey, eval;
        std::vector<float> ewt;
        ekey.reserve(n_ent[f]);
        eval.reserve(n_ent[f]);
        ewt.reserve(n_ent[f]);
        int64_t w_, d_;
        channel(f, true, [&](uint32_t k, uint32_t v, float x) {
            ekey.push_back(k);
            eval.push_back(v);
            ewt.push_back(x);
        }, w_, d_);
        // stable sort by key into the channel's range: a cell's entries stay in baseline order (a counting
        // sort while the keys are few next to the entries, a comparison sort on large grids)
        std::vector<uint32_t> ord(ekey.size());
        if (nkeys <= (int64_t)16 * (int64_t)ekey.size() + 4096) {
            std::vector<int> count(nkeys + 1, 0);
            for (uint32_t k : ekey) count[k + 1]++;
            for (int64_t k = 0; k < nkeys; k++) count[k + 1] += count[k];
            for (size_t q = 0; q < ekey.size(); q++) ord[count[ekey[q]]++] = (uint32_t)q;
        } else {
            for (size_t q = 0; q < ord.size(); q++) ord[q] = (uint32_t)q;
            std::stable_sort(ord.begin(), ord.end(), [&](uint32_t x, uint32_t y) { return ekey[x] < ekey[y]; });
        }
        int64_t e = 0;
        for (int u = 0; u <= half; u++) {
            const uint32_t lim = (uint32_t)std::min<int64_t>((int64_t)u * N, nkeys);
            while (e < (int64_t)ord.size() && ekey[ord[e]] < lim) e++;
            ent_off[(size_t)f * (half + 1) + u] = (int)(base[f] + e);
        }
        for (size_t q = 0; q < ord.size(); q++) {
            const uint32_t k = ekey[ord[q]], u = k / N, v = k % N;
            ent[base[f] + q] = make_uint2(u | (v << 13) | ((eval[ord[q]] & 1u) << 31), eval[ord[q]] >> 1);
            wt[base[f] + q] = ewt[ord[q]];
        }
    });
    // the separable form: per channel, records in baseline order (a visibility, then its mirror), and per
    // column the entries of the records whose support meets it, sorted by (v0, record)
    if (W <= kSepMaxW && fast_side(N) && B <= 0x7FFFFFFF) {
        struct Sep {
            std::vector<uint4> ent;            // sorted, channel-local record numbers in .w
            std::vector<float> wrow;           // [records][kSepMaxW]
            std::vector<int> off;              // [half + 1], channel-local
        };
        std::vector<Sep> sep(F);
        parallel([&](int f) {
            std::vector<SepEntry> ent;
            kb_sep_channel(N, W, B, p->autos, p->du, uvw.data() + (size_t)f * B * 3,
                           [&](int64_t b) { return a->flags && (a->flags[bl[b].x] || a->flags[bl[b].y]); },
                           [&](int64_t b) { return bl[b].x == bl[b].y; }, ent, sep[f].wrow, sep[f].off);
            sep[f].ent.resize(ent.size());
            for (size_t q = 0; q < ent.size(); q++) {
                uint32_t wbits;
                std::memcpy(&wbits, &ent[q].wu, 4);
                sep[f].ent[q] = make_uint4(ent[q].bc, (uint32_t)ent[q].v0, wbits, ent[q].rec);
            }
        });
        std::vector<int64_t> e0(F + 1, 0), r0(F + 1, 0);
        for (int f = 0; f < F; f++) {
            e0[f + 1] = e0[f] + (int64_t)sep[f].ent.size();
            r0[f + 1] = r0[f] + (int64_t)sep[f].wrow.size() / kSepMaxW;
        }
        if (e0[F] > INT32_MAX / 2 || r0[F] * kSepMaxW > INT32_MAX) return set_error(BLINK_ERR_UNSUPPORTED, "gather list too large");
        std::vector<int> soff((size_t)F * (half + 1) + 1);
        std::vector<uint4> sent((size_t)e0[F]);
        std::vector<float> swt((size_t)r0[F] * kSepMaxW);
        for (int f = 0; f < F; f++) {
            for (int u = 0; u <= half; u++) soff[(size_t)f * (half + 1) + u] = (int)(e0[f] + sep[f].off[u]);
            for (size_t q = 0; q < sep[f].ent.size(); q++) {
                uint4 x = sep[f].ent[q];
                x.w = (uint32_t)((r0[f] + x.w) * kSepMaxW);
                sent[(size_t)e0[f] + q] = x;
            }
            std::copy(sep[f].wrow.begin(), sep[f].wrow.end(), swt.begin() + r0[f] * kSepMaxW);
        }
        soff[(size_t)F * (half + 1)] = (int)e0[F];
        BLINK_TRY(dmalloc(&p->d_sep_off, soff.size()));
        BLINK_CUDA(cudaMemcpy(p->d_sep_off, soff.data(), soff.size() * sizeof(int), cudaMemcpyHostToDevice));
        if (!sent.empty()) {
            BLINK_TRY(dmalloc(&p->d_sep, sent.size()));
            BLINK_TRY(dmalloc(&p->d_sep_w, swt.size()));
            BLINK_CUDA(cudaMemcpy(p->d_sep, sent.data(), sent.size() * sizeof(uint4), cudaMemcpyHostToDevice));
            BLINK_CUDA(cudaMemcpy(p->d_sep_w, swt.data(), swt.size() * sizeof(float), cudaMemcpyHostToDevice));
        }
    }
    p->W.assign(F, 0.f);
    int64_t dropped = 0;
    for (int f = 0; f < F; f++) {
        p->W[f] = (float)wsum[f];
        dropped += drop[f];
    }
    p->n_dropped = dropped;
    p->n_contrib = base[F];
    p->n_cells = p->n_contrib;
    BLINK_TRY(dmalloc(&p->d_ent_off, ent_off.size()));
    BLINK_TRY(dmalloc(&p->d_ent, ent.size()));
    BLINK_TRY(dmalloc(&p->d_wt, wt.size()));
    BLINK_CUDA(cudaMemcpy(p->d_ent_off, ent_off.data(), ent_off.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (!ent.empty()) {
        BLINK_CUDA(cudaMemcpy(p->d_ent, ent.data(), ent.size() * sizeof(uint2), cudaMemcpyHostToDevice));
        BLINK_CUDA(cudaMemcpy(p->d_wt, wt.data(), wt.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    return BLINK_OK;
}

// Grid correction of an image of side Ni from a grid of side 2 Ni: 1 / c((x - Ni/2) / (2 Ni)) per pixel index.
std::vector<float> kb_correction(int Ni, int W) {
    const double beta = kb_beta(W);
    std::vector<float> c(Ni);
    for (int x = 0; x < Ni; x++) c[x] = (float)(1.0 / kb_transform((double)(x - Ni / 2) / (2.0 * Ni), W, beta));
    return c;
}

}  // namespace

blink_status workspace(blink_context* ctx, int slot, size_t bytes, void** out) {
    Workspace& w = ctx->ws[slot];
    if (w.bytes < bytes) {
        if (w.ptr) {
            BLINK_CUDA(cudaDeviceSynchronize());
            cudaFree(w.ptr);
            w.ptr = nullptr;
            w.bytes = 0;
        }
        cudaError_t e = cudaMalloc(&w.ptr, bytes);
        if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(workspace)");
        w.bytes = bytes;
    }
    *out = w.ptr;
    return BLINK_OK;
}

// The call's calibration (F output channels) copied to device workspace: full Jones matrices when given,
// else diagonal gains, else an empty reference.
blink_status upload_gains(blink_context* ctx, const blink_array* a, int F, cudaStream_t st, GainRef* out) {
    *out = GainRef{};
    const float* src = a->jones ? a->jones : a->gains;
    if (!src || F < 1) return BLINK_OK;
    const size_t n = (size_t)F * a->n_tiles * (a->jones ? 8 : 4);
    for (size_t i = 0; i < n; i++)
        if (!std::isfinite(src[i]))
            return set_error(BLINK_ERR_INVALID_ARG, "array.gains or array.jones has a non-finite value");
    void* d = nullptr;
    BLINK_TRY(workspace(ctx, 6, n * sizeof(float), &d));
    BLINK_CUDA(cudaMemcpyAsync(d, src, n * sizeof(float), cudaMemcpyHostToDevice, st));
    out->d = static_cast<const float2*>(d);
    out->full = a->jones != nullptr;
    return BLINK_OK;
}

// The twiddle set of side N (see tws_total), made on the device on first use and kept in the context.
blink_status kernel_smem(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::vector<std::pair<const void*, size_t>> done;
    std::lock_guard<std::mutex> lock(mu);
    for (auto& d : done)
        if (d.first == fn) {
            if (d.second >= bytes) return BLINK_OK;
            BLINK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
            d.second = bytes;
            return BLINK_OK;
        }
    if (bytes > 48 * 1024) BLINK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    done.emplace_back(fn, bytes);
    return BLINK_OK;
}

blink_status twiddles(blink_context* ctx, int N, float2** out) {
    if (!fast_side(N)) {
        for (auto& t : ctx->tw_any)
            if (t.first == N) {
                *out = t.second;
                return BLINK_OK;
            }
        float2* d = nullptr;
        BLINK_CUDA(cudaMalloc(&d, sizeof(float2) * N));
        blink_status s = make_unit_roots(d, N, 0);
        cudaError_t e = cudaDeviceSynchronize();
        if (s != BLINK_OK || e != cudaSuccess) {
            cudaFree(d);
            return s != BLINK_OK ? s : cuda_error(e, "twiddle kernel");
        }
        ctx->tw_any.emplace_back(N, d);
        *out = d;
        return BLINK_OK;
    }
    int lg = 0;
    while ((1 << lg) < N) lg++;
    if (lg >= 16 || (1 << lg) != N) return set_error(BLINK_ERR_UNSUPPORTED, "twiddle table side");
    if (!ctx->tw[lg]) {
        float2* d = nullptr;
        BLINK_CUDA(cudaMalloc(&d, sizeof(float2) * tws_total(N)));
        blink_status s = make_twiddles(d, N, 0);
        cudaError_t e = cudaDeviceSynchronize();
        if (s != BLINK_OK || e != cudaSuccess) {
            cudaFree(d);
            return s != BLINK_OK ? s : cuda_error(e, "twiddle kernel");
        }
        ctx->tw[lg] = d;
    }
    *out = ctx->tw[lg];
    return BLINK_OK;
}

static cudaEvent_t take_event(blink_context* ctx) {
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

StageTimer::StageTimer(blink_context* c, int s, cudaStream_t stream) : ctx(c), stage(s), st(stream) {
    if (!ctx->profiling) return;
    cudaEvent_t a = take_event(ctx);
    b = take_event(ctx);
    if (!a || !b) {
        b = nullptr;
        return;
    }
    cudaEventRecord(a, st);
    ctx->recs.push_back({stage, a, b});
}

StageTimer::~StageTimer() {
    if (b) cudaEventRecord(b, st);
}

// Plans are keyed by every input they depend on.  Imaging-free plans (im == NULL) serve correlation.
blink_status get_plan(blink_context* ctx, const blink_array* a, const blink_obs* o, const blink_imaging* im,
                      bool need_gather, cudaStream_t st, Plan** out) {
    Hasher h;
    h.val(a->n_tiles);
    h.val(a->flags != nullptr);
    if (a->flags) h.bytes(a->flags, a->n_tiles);
    h.val(im != nullptr);
    if (im) {
        h.bytes(a->enu_m, sizeof(double) * 3 * a->n_tiles);
        h.val(o->n_fine);
        h.val(o->chan_avg);
        h.val(o->samples_per_int);
        h.bytes(o->fine_freq_hz, sizeof(double) * o->n_fine);
        h.val(im->n_pix);
        h.val(im->cell_lambda);
        h.val(im->pol);
        h.val(im->include_autos != 0);
        h.val(im->support >= 2 ? im->support : 0);
        h.val(im->phase_l);
        h.val(im->phase_m);
        h.val(need_gather);
    } else {
        h.val(o->n_fine / o->chan_avg);
        h.val(o->chan_avg);
    }
    for (size_t k = 0; k < ctx->plans.size(); k++) {
        Plan* p = ctx->plans[k];
        if (p->key == h.h) {
            ctx->plans.erase(ctx->plans.begin() + k);
            ctx->plans.push_back(p);
            *out = p;
            return BLINK_OK;
        }
    }
    if (ctx->plans.size() >= 8) {
        BLINK_CUDA(cudaDeviceSynchronize());
        free_plan(ctx->plans.front());
        ctx->plans.erase(ctx->plans.begin());
    }
    Plan* p = new Plan();
    p->key = h.h;
    p->n_tiles = a->n_tiles;
    p->n_fine = o->n_fine;
    p->chan_avg = o->chan_avg;
    p->F = o->n_fine / o->chan_avg;
    p->B = blink_n_baselines(a->n_tiles);
    std::vector<short2> bl(p->B);
    for (int i = 0, b = 0; i < a->n_tiles; i++)
        for (int j = 0; j <= i; j++, b++) bl[b] = make_short2((short)i, (short)j);
    std::vector<uint8_t> flags(a->n_tiles, 0);
    if (a->flags)
        for (int i = 0; i < a->n_tiles; i++) flags[i] = a->flags[i] ? 1 : 0;
    blink_status s = BLINK_OK;
    auto fail = [&](blink_status e) {
        free_plan(p);
        return e;
    };
    if ((s = dmalloc(&p->d_bl, p->B)) != BLINK_OK) return fail(s);
    if ((s = dmalloc(&p->d_flags, a->n_tiles)) != BLINK_OK) return fail(s);
    cudaError_t e = cudaMemcpy(p->d_bl, bl.data(), bl.size() * sizeof(short2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_flags, flags.data(), flags.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(cuda_error(e, "cudaMemcpy(plan)"));
    if (im) {
        p->support = im->support >= 2 ? im->support : 0;
        p->Ni = im->n_pix;
        p->N = p->support ? 2 * im->n_pix : im->n_pix;     // with a kernel the grid is oversampled by 2
        p->pol = im->pol;
        p->autos = im->include_autos ? 1 : 0;
        p->cw = col_block_width(p->N);
        p->n_cb = (p->N / 2) / p->cw;
        p->out_freq = output_freqs(o);
        double numax = p->out_freq[0];
        for (double f : p->out_freq) numax = std::max(numax, f);
        p->phased = off_zenith(im);
        if (p->phased) pointing_basis(im->phase_l, im->phase_m, p->basis);
        p->du = im->cell_lambda > 0.0 ? im->cell_lambda
                                      : default_cell(a, numax, p->N, p->support, p->phased ? p->basis : nullptr);
        if ((s = dmalloc(&p->d_enu, 3 * a->n_tiles)) != BLINK_OK) return fail(s);
        if ((s = dmalloc(&p->d_freq, p->F)) != BLINK_OK) return fail(s);
        if ((s = dmalloc(&p->d_cells, (size_t)p->F * p->B)) != BLINK_OK) return fail(s);
        if ((s = dmalloc(&p->d_W, p->F)) != BLINK_OK) return fail(s);
        if ((s = dmalloc(&p->d_Wk, p->F)) != BLINK_OK) return fail(s);
        const bool fast = fast_side(p->N);
        if ((s = dmalloc(&p->d_tw, fast ? tws_total(p->N) : p->N)) != BLINK_OK) return fail(s);
        e = cudaMemcpy(p->d_enu, a->enu_m, sizeof(double) * 3 * a->n_tiles, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p->d_freq, p->out_freq.data(), sizeof(double) * p->F, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(cuda_error(e, "cudaMemcpy(plan)"));
        if ((s = fast ? make_twiddles(p->d_tw, p->N, st) : make_unit_roots(p->d_tw, p->N, st)) != BLINK_OK)
            return fail(s);
        if (fast && (s = fft_constants(p->N)) != BLINK_OK) return fail(s);
        // with a kernel the gather list is built from the exact (u, v), kept on the device only meanwhile
        const bool kb = p->support && need_gather;
        if (kb && (s = dmalloc(&p->d_uvw, (size_t)p->F * p->B * 3)) != BLINK_OK) return fail(s);
        if (p->phased && need_gather && (s = dmalloc(&p->d_phase, (size_t)p->F * p->B)) != BLINK_OK) return fail(s);
        launch_cells(*p, st);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(cuda_error(e, "geometry kernel"));
        if (kb) {
            std::vector<double> uvw((size_t)p->F * p->B * 3);
            e = cudaMemcpy(uvw.data(), p->d_uvw, uvw.size() * sizeof(double), cudaMemcpyDeviceToHost);
            cudaFree(p->d_uvw);
            p->d_uvw = nullptr;
            if (e != cudaSuccess) return fail(cuda_error(e, "cudaMemcpy(uvw)"));
            if ((s = build_gather_kb(p, uvw, bl, a)) != BLINK_OK) return fail(s);
            const std::vector<float> corr = kb_correction(p->Ni, p->support);
            if ((s = dmalloc(&p->d_corr, corr.size())) != BLINK_OK) return fail(s);
            e = cudaMemcpy(p->d_corr, corr.data(), corr.size() * sizeof(float), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return fail(cuda_error(e, "cudaMemcpy(correction)"));
        }
        if (need_gather) {
            if (!kb) {
                std::vector<uint32_t> cells((size_t)p->F * p->B);
                e = cudaMemcpy(cells.data(), p->d_cells, cells.size() * 4, cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) return fail(cuda_error(e, "cudaMemcpy(cells)"));
                if ((s = build_gather(p, cells, bl, a)) != BLINK_OK) return fail(s);
                if (p->d_phase && p->d_gsrc) {
                    if ((s = dmalloc(&p->d_gphase, (size_t)p->F * p->e_stride)) != BLINK_OK) return fail(s);
                    if ((s = launch_gather_phase(*p, st)) != BLINK_OK) return fail(s);
                }
            }
            // the imaging path grids raw correlation sums: scale by 1 / (W * 2K) (Stokes I) or 1 / (W * K)
            const double div = (p->pol == BLINK_POL_I ? 2.0 : 1.0) * o->samples_per_int * o->chan_avg;
            std::vector<float> wk(p->F);
            for (int f = 0; f < p->F; f++) wk[f] = (float)(p->W[f] * div);
            e = cudaMemcpy(p->d_W, p->W.data(), sizeof(float) * p->F, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(p->d_Wk, wk.data(), sizeof(float) * p->F, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return fail(cuda_error(e, "cudaMemcpy(W)"));
        }
    }
    ctx->plans.push_back(p);
    *out = p;
    return BLINK_OK;
}

namespace {

__global__ void k_fill_weights(float* out, const float* W, int F, int first, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = W[(first + i) % F];
}

int64_t sample_stride_bytes(const blink_obs* o, int n_tiles) {
    const int stride = o->fine_stride ? o->fine_stride : o->n_fine;
    return (int64_t)stride * n_tiles * 2;
}

// Batched path for the integrations [tau0, tau1) (images [tau0 F, tau1 F)), written to d_img starting at
// image tau0 F: one correlator launch over as many integrations as the visibility workspace holds, then
// one persistent launch that grids and transforms all of their images (fft_persistent.cu).
constexpr size_t kVisCapBytes = (size_t)4 << 30;
constexpr int kAvgGridMembers = 16;              // channels per averaged output from which its grid is built first

// Batched path on a side outside the side-specialised kernels, and every averaged call: one correlator
// launch per chunk of integrations, then per wave of output images (their column results about the size of
// L2: 96 MB measured a little faster than 48 MB at side 1200, with half the launches) the mixed-radix column
// pass, gathering each output's cells from the sums of its fa channels, and the row pass (fft_mixed.cu).
// fa = 1: one image per (integration, channel), divided by W in the row pass; fa > 1: the mean of fa
// consecutive channels' normalised images, each channel's sums divided by its own W in the gather.
// Outputs [tau0 F/fa, tau1 F/fa) are written from d_img on.
blink_status run_mixed(blink_context* ctx, const Plan& p, const blink_obs* o, int prec, int arith,
                       const uint8_t* d_volt, int64_t sstride, int tau0, int tau1, float* d_img, cudaStream_t st,
                       GainRef gains, int fa = 1) {
    const int F = p.F, T = tau1 - tau0, Fo = F / fa;
    if (T <= 0) return BLINK_OK;
    const int kind = p.pol == BLINK_POL_I ? CORR_OUT_STOKES_I : CORR_OUT_XX;
    // nearest cell with FP8: the correlator writes the sums in the gather's entry order
    const bool gathered = arith == BLINK_CORR_FP8 && !p.d_wt && p.d_gsrc && p.e_stride > 0 &&
                          corr_fp8_gathers(p, o->samples_per_int, kind, gains);
    const int64_t vstride = gathered ? p.e_stride : p.B;          // float2 per item
    const int t_chunk = (int)std::max<int64_t>(1, std::min<int64_t>(T, (int64_t)(kVisCapBytes / ((size_t)vstride * 8 * F))));
    const bool crop = p.support != 0;
    const size_t el = prec == BLINK_PREC_BF16 ? 4 : 8;
    const size_t per_img = (size_t)(crop ? p.N / 2 : p.N) * mixed_h_row(p.N) * el;
    const int wave = (int)std::max<size_t>(1, std::min<size_t>(65535, ((size_t)96 << 20) / per_img));
    void* vis = nullptr;
    void* H = nullptr;
    BLINK_TRY(workspace(ctx, 0, (size_t)t_chunk * F * vstride * sizeof(float2), &vis));
    BLINK_TRY(workspace(ctx, 1, (size_t)std::min(wave, t_chunk * Fo) * per_img, &H));
    // averages over many channels: their grids first, summed by every warp of the GPU (k_avg_grid), then the
    // column pass from those grids
    const bool grid_first = fa >= kAvgGridMembers;
    const size_t grid_bytes = (size_t)p.N * (p.N / 2 + 1) * sizeof(float2);
    void* G = nullptr;
    if (grid_first) BLINK_TRY(workspace(ctx, 8, (size_t)std::min(wave, t_chunk * Fo) * grid_bytes, &G));
    ImgOut io;
    io.phase = p.d_phase;
    io.gather = gathered;
    MixedIn in;
    in.N = p.N;
    in.tw = p.d_tw;
    in.vis = static_cast<const float2*>(vis);
    in.vstride = vstride;
    in.gathered = gathered;
    in.e_stride = p.e_stride;
    in.F = F;
    in.fa = fa;
    in.wk = fa > 1 ? p.d_Wk : nullptr;
    in.ent_off = p.d_ent_off;
    in.ent = p.d_ent;
    in.wt = p.d_wt;
    in.corr = crop ? p.d_corr : nullptr;
    const float* row_w = fa > 1 ? nullptr : p.d_Wk;
    const int out_first = tau0 * Fo;
    for (int ta = tau0; ta < tau1; ta += t_chunk) {
        const int tb = std::min(tau1, ta + t_chunk);
        const int first = ta * F, n_items = (tb - ta) * F, n_out = (tb - ta) * Fo;
        {
            StageTimer t(ctx, BLINK_STAGE_CORRELATE, st);
            if (arith == BLINK_CORR_FP8)
                BLINK_TRY(launch_corr_fp8(kind, d_volt, sstride, p, o->samples_per_int, first, n_items, vis, p.B,
                                          ctx->d_status, ctx->n_sm, st, gains, io));
            else
                BLINK_TRY(launch_corr_fp32(kind, d_volt, sstride, p, o->samples_per_int, first, n_items, vis, p.B,
                                           ctx->d_status, st, gains, io));
        }
        in.first = first;
        for (int w0 = 0; w0 < n_out; w0 += wave) {
            const int nw = std::min(wave, n_out - w0);
            in.o_first = w0;
            const WaveMap wm{1, 0, ta * Fo + w0, nw};
            {
                StageTimer t(ctx, BLINK_STAGE_GRID_FFT, st);
                if (grid_first) {
                    BLINK_CUDA(cudaMemsetAsync(G, 0, (size_t)nw * grid_bytes, st));
                    BLINK_TRY(launch_avg_grid(in, nw, static_cast<float2*>(G), st));
                    MixedIn ig = in;
                    ig.grid = static_cast<const float2*>(G);
                    BLINK_TRY(launch_mixed(ig, 0, prec, nw, H, nullptr, 1, wm, out_first, nullptr, st));
                } else {
                    BLINK_TRY(launch_mixed(in, 0, prec, nw, H, nullptr, 1, wm, out_first, nullptr, st));
                }
            }
            StageTimer t(ctx, BLINK_STAGE_ROW_FFT, st);
            BLINK_TRY(launch_mixed(in, 1, prec, nw, H, row_w, F, wm, out_first, d_img, st));
        }
    }
    return BLINK_OK;
}

blink_status run_batched(blink_context* ctx, const Plan& p, const blink_obs* o, int prec, int arith,
                         const uint8_t* d_volt, int64_t sstride, int tau0, int tau1, float* d_img, cudaStream_t st,
                         bool may_tune = true, GainRef gains = {}) {
    if (!fast_side(p.N)) return run_mixed(ctx, p, o, prec, arith, d_volt, sstride, tau0, tau1, d_img, st, gains);
    const int N = p.N, F = p.F;
    const size_t el = prec == BLINK_PREC_BF16 ? 4 : 8;
    const int T = tau1 - tau0;
    if (T <= 0) return BLINK_OK;
    const int kind = p.pol == BLINK_POL_I ? CORR_OUT_STOKES_I : CORR_OUT_XX;
    // the side-512 kernel reads the sums in gather order, which the FP8 correlator writes directly
    const bool gathered = fft_takes_gathered(p) && arith == BLINK_CORR_FP8 &&
                          corr_fp8_gathers(p, o->samples_per_int, kind, gains);
    const int64_t vstride = gathered ? p.e_stride : p.B;          // float2 per item
    // fused: one launch correlates (tensor cores) and images every item, the sums never leaving L2
    const bool fused = gathered && ctx->fused && !gains.d && !p.d_phase &&
                       fft_fused_ok(p, o->samples_per_int, kind, d_volt, sstride);
    const int t_chunk = fused ? T : (int)std::max<int64_t>(1, std::min<int64_t>(T, (int64_t)(kVisCapBytes /
                                                                                              ((size_t)vstride * 8 * F))));
    ImgOut io;
    io.phase = p.d_phase;
    io.gather = gathered;
    void* vis = nullptr;
    void* H = nullptr;
    void* cnt = nullptr;
    BLINK_TRY(workspace(ctx, 0, fused ? fused_ring_floats(p) * sizeof(float) : (size_t)t_chunk * F * vstride * sizeof(float2),
                        &vis));
    BLINK_TRY(workspace(ctx, 1, (size_t)fft_ring_images_max() * N * (N / 2) * el, &H));
    BLINK_TRY(workspace(ctx, 4, sizeof(int) * (2 + 3 * (size_t)t_chunk * F), &cnt));
    FusedIn fz;
    fz.d_volt = d_volt;
    fz.sample_stride = sstride;
    fz.ns = o->samples_per_int;
    fz.kind = kind;
    fz.d_vring = static_cast<float*>(vis);
    const FusedIn* fzp = fused ? &fz : nullptr;
    const int stage = fused ? BLINK_STAGE_FUSED : BLINK_STAGE_GRID_FFT;
    const int out_first = tau0 * F;
    for (int ta = tau0; ta < tau1; ta += t_chunk) {
        const int tb = std::min(tau1, ta + t_chunk);
        const int first = ta * F, n_items = (tb - ta) * F;
        if (!fused) {
            StageTimer t(ctx, BLINK_STAGE_CORRELATE, st);
            if (arith == BLINK_CORR_FP8)
                BLINK_TRY(launch_corr_fp8(kind, d_volt, sstride, p, o->samples_per_int, first, n_items, vis, p.B,
                                          ctx->d_status, ctx->n_sm, st, gains, io));
            else
                BLINK_TRY(launch_corr_fp32(kind, d_volt, sstride, p, o->samples_per_int, first, n_items, vis, p.B,
                                           ctx->d_status, st, gains, io));
        }
        if (!p.tuned && !may_tune) {
            // output over the host link: timings would measure the link, so run the default shape untuned
            StageTimer t(ctx, stage, st);
            BLINK_TRY(launch_fft_persistent(p, fft_tune_candidates(p)[0], prec, static_cast<float2*>(vis), vstride, first,
                                            ta, tb - ta, H, static_cast<int*>(cnt), d_img, out_first, ctx->d_status,
                                            ctx->n_sm, st, ctx->fft_wait, gathered, fzp));
        } else if (!p.tuned) {
            // autotune the FFT launch shape on this first batch: time each candidate (every run writes the
            // same images), keep the fastest for every later call of the plan
            struct Events {
                cudaEvent_t e[2] = {nullptr, nullptr};
                ~Events() {
                    for (cudaEvent_t x : e)
                        if (x) cudaEventDestroy(x);
                }
            } ev;
            BLINK_CUDA(cudaEventCreate(&ev.e[0]));
            BLINK_CUDA(cudaEventCreate(&ev.e[1]));
            cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
            float best = 0.f;
            for (const FftTune& c : fft_tune_candidates(p)) {
                BLINK_CUDA(cudaEventRecord(e0, st));
                BLINK_TRY(launch_fft_persistent(p, c, prec, static_cast<float2*>(vis), vstride, first, ta, tb - ta, H,
                                                static_cast<int*>(cnt), d_img, out_first, ctx->d_status, ctx->n_sm,
                                                st, ctx->fft_wait, gathered, fzp));
                BLINK_CUDA(cudaEventRecord(e1, st));
                BLINK_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                BLINK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (!p.tuned || ms < best) {
                    best = ms;
                    p.tune = c;
                    p.tuned = true;
                }
            }
            p.tune_ms = best;
        } else {
            StageTimer t(ctx, stage, st);
            BLINK_TRY(launch_fft_persistent(p, p.tune, prec, static_cast<float2*>(vis), vstride, first, ta, tb - ta, H,
                                            static_cast<int*>(cnt), d_img, out_first, ctx->d_status, ctx->n_sm, st,
                                            ctx->fft_wait, gathered, fzp));
        }
    }
    return BLINK_OK;
}

// Device address of a host buffer of `bytes` bytes that the current device can write: page-locked
// (cudaHostAlloc or cudaHostRegister) memory mapped for the device, judged by its first and last byte, or
// pageable memory on a device that reaches it through the host's page tables (hardware-coherent host
// links); NULL otherwise.
float* device_view(float* h, size_t bytes) {
    if (!h || !bytes) return nullptr;
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeUnregistered) {
        int dev = 0, pageable = 0, host_tables = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return pageable && host_tables ? h : nullptr;
    }
    const char* last = reinterpret_cast<const char*>(h) + bytes - 1;
    if (cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
        return nullptr;
    if (static_cast<char*>(b.devicePointer) - static_cast<char*>(a.devicePointer) != (ptrdiff_t)(bytes - 1))
        return nullptr;
    return static_cast<float*>(a.devicePointer);
}

}  // namespace

}  // namespace blink

using namespace blink;

extern "C" {

const char* blink_last_error(void) { return g_err.c_str(); }

const char* blink_status_name(blink_status s) {
    switch (s) {
        case BLINK_OK: return "BLINK_OK";
        case BLINK_ERR_INVALID_ARG: return "BLINK_ERR_INVALID_ARG";
        case BLINK_ERR_UNSUPPORTED: return "BLINK_ERR_UNSUPPORTED";
        case BLINK_ERR_OOM: return "BLINK_ERR_OOM";
        case BLINK_ERR_CUDA: return "BLINK_ERR_CUDA";
        case BLINK_ERR_TIMEOUT: return "BLINK_ERR_TIMEOUT";
        case BLINK_ERR_DEVICE: return "BLINK_ERR_DEVICE";
    }
    return "BLINK_UNKNOWN";
}

int64_t blink_n_baselines(int32_t n_tiles) { return n_tiles < 0 ? 0 : (int64_t)n_tiles * (n_tiles + 1) / 2; }

blink_status blink_create(int32_t device, blink_context** out) {
    if (!out) return set_error(BLINK_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    BLINK_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return set_error(BLINK_ERR_INVALID_ARG, "no such CUDA device");
    BLINK_CUDA(cudaSetDevice(device));
    cudaDeviceProp prop;
    BLINK_CUDA(cudaGetDeviceProperties(&prop, device));
    if (prop.major < 10)
        return set_error(BLINK_ERR_UNSUPPORTED, "this library is built for sm_103a (Blackwell) devices");
    blink_context* ctx = new blink_context();
    ctx->device = device;
    ctx->n_sm = prop.multiProcessorCount;
    cudaError_t e = cudaMalloc(&ctx->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
    if (e != cudaSuccess) {
        delete ctx;
        return cuda_error(e, "cudaMalloc(status)");
    }
    *out = ctx;
    return BLINK_OK;
}

void blink_destroy(blink_context* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (Plan* p : ctx->plans) free_plan(p);
    for (auto& w : ctx->ws) cudaFree(w.ptr);
    for (float2* t : ctx->tw) cudaFree(t);
    for (auto& t : ctx->tw_any) cudaFree(t.second);
    for (auto& r : ctx->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
    cudaFree(ctx->d_status);
    delete ctx;
}

blink_status blink_sync(blink_context* ctx, void* stream) {
    BLINK_TRY(make_current(ctx));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BLINK_CUDA(cudaStreamSynchronize(st));
    int status = 0;
    BLINK_CUDA(cudaMemcpy(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) {
        BLINK_CUDA(cudaMemset(ctx->d_status, 0, sizeof(int)));
        if (status & DEV_ERR_TIMEOUT) return set_error(BLINK_ERR_TIMEOUT, "a bounded device-side wait ran out");
        return set_error(BLINK_ERR_DEVICE, "a device-side index guard failed");
    }
    return BLINK_OK;
}

blink_status blink_set_wait_budget(blink_context* ctx, int64_t budget_cycles, int32_t unreachable) {
    if (!ctx) return set_error(BLINK_ERR_INVALID_ARG, "context is NULL");
    ctx->fft_wait.budget = budget_cycles > 0 ? (long long)budget_cycles : FftWait{}.budget;
    ctx->fft_wait.extra = unreachable ? 1 : 0;
    return BLINK_OK;
}

blink_status blink_set_fused(blink_context* ctx, int32_t enable) {
    if (!ctx) return set_error(BLINK_ERR_INVALID_ARG, "context is NULL");
    ctx->fused = enable != 0;
    return BLINK_OK;
}

blink_status blink_tuned_shape(blink_context* ctx, int32_t* out) {
    if (!ctx || !out) return set_error(BLINK_ERR_INVALID_ARG, "context or out is NULL");
    out[0] = out[1] = out[2] = 0;
    if (!ctx->plans.empty() && ctx->plans.back()->tuned) {
        const FftTune& t = ctx->plans.back()->tune;
        out[0] = t.ring;
        out[1] = t.lag;
        out[2] = t.ctas_per_sm;
    }
    return BLINK_OK;
}

blink_status blink_set_profiling(blink_context* ctx, int32_t enable) {
    if (!ctx) return set_error(BLINK_ERR_INVALID_ARG, "context is NULL");
    ctx->profiling = enable != 0;
    return BLINK_OK;
}

blink_status blink_read_profile(blink_context* ctx, void* stream, double* ms, int64_t* launches, int32_t reset) {
    BLINK_TRY(make_current(ctx));
    if (!ms || !launches) return set_error(BLINK_ERR_INVALID_ARG, "ms or launches is NULL");
    BLINK_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    for (int s = 0; s < BLINK_N_STAGES; s++) {
        ms[s] = 0.0;
        launches[s] = 0;
    }
    for (auto& r : ctx->recs) {
        float t = 0.f;
        BLINK_CUDA(cudaEventSynchronize(r.b));
        BLINK_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        if (r.stage >= 0 && r.stage < BLINK_N_STAGES) {
            ms[r.stage] += t;
            launches[r.stage] += 1;
        }
    }
    if (reset) {
        for (auto& r : ctx->recs) {
            ctx->pool.push_back(r.a);
            ctx->pool.push_back(r.b);
        }
        ctx->recs.clear();
    }
    return BLINK_OK;
}

blink_status blink_cells(blink_context* ctx, const blink_array* array, const blink_obs* obs,
                         const blink_imaging* imaging, int32_t* d_cells, double* d_uvw, double* h_du, void* stream) {
    BLINK_TRY(check_array(array));
    BLINK_TRY(check_obs(obs, true));
    BLINK_TRY(check_imaging(imaging));
    BLINK_TRY(nearest_only(imaging, "blink_cells"));
    if (!d_cells) return set_error(BLINK_ERR_INVALID_ARG, "d_cells is NULL");
    BLINK_TRY(make_current(ctx));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Plan* p = nullptr;
    BLINK_TRY(get_plan(ctx, array, obs, imaging, false, st, &p));
    Plan q = *p;                   // same geometry inputs, caller's output buffers
    q.d_cells = reinterpret_cast<uint32_t*>(d_cells);
    q.d_uvw = d_uvw;
    q.d_phase = nullptr;
    launch_cells(q, st);
    BLINK_CUDA(cudaGetLastError());
    if (h_du) *h_du = p->du;
    return BLINK_OK;
}

blink_status blink_correlate(blink_context* ctx, const blink_array* array, const blink_obs* obs, int32_t arith,
                             const uint8_t* d_volt, float* d_vis, void* stream) {
    BLINK_TRY(check_array(array));
    BLINK_TRY(check_obs(obs, false));
    if (arith != BLINK_CORR_FP32 && arith != BLINK_CORR_FP8)
        return set_error(BLINK_ERR_INVALID_ARG, "arith must be BLINK_CORR_FP32 or BLINK_CORR_FP8");
    if (!d_volt || !d_vis) return set_error(BLINK_ERR_INVALID_ARG, "d_volt or d_vis is NULL");
    if (((uintptr_t)d_volt & 1) || ((uintptr_t)d_vis & 15))
        return set_error(BLINK_ERR_INVALID_ARG, "d_volt must be 2-byte and d_vis 16-byte aligned");
    BLINK_TRY(make_current(ctx));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Plan* p = nullptr;
    BLINK_TRY(get_plan(ctx, array, obs, nullptr, false, st, &p));
    const int T = obs->n_samples / obs->samples_per_int;
    const int n_items = T * p->F;
    if (n_items == 0) return BLINK_OK;
    const int64_t ss = sample_stride_bytes(obs, array->n_tiles);
    GainRef g;
    BLINK_TRY(upload_gains(ctx, array, p->F, st, &g));
    if (arith == BLINK_CORR_FP8)
        return launch_corr_fp8(CORR_OUT_VIS4, d_volt, ss, *p, obs->samples_per_int, 0, n_items, d_vis, p->B * 8,
                               ctx->d_status, ctx->n_sm, st, g);
    return launch_corr_fp32(CORR_OUT_VIS4, d_volt, ss, *p, obs->samples_per_int, 0, n_items, d_vis, p->B * 8,
                            ctx->d_status, st, g);
}

blink_status blink_grid(blink_context* ctx, const blink_array* array, const blink_obs* obs,
                        const blink_imaging* imaging, const float* d_vis, int32_t first_image, int32_t n_images,
                        float* d_grid, float* d_weight, void* stream) {
    BLINK_TRY(check_array(array));
    BLINK_TRY(check_obs(obs, true));
    BLINK_TRY(check_imaging(imaging));
    BLINK_TRY(nearest_only(imaging, "blink_grid"));
    BLINK_TRY(zenith_only(imaging, "blink_grid"));
    if (!d_vis || !d_grid) return set_error(BLINK_ERR_INVALID_ARG, "d_vis or d_grid is NULL");
    if (first_image < 0 || n_images < 0) return set_error(BLINK_ERR_INVALID_ARG, "negative image range");
    if (((uintptr_t)d_vis & 7) || ((uintptr_t)d_grid & 7))
        return set_error(BLINK_ERR_INVALID_ARG, "d_vis and d_grid must be 8-byte aligned");
    const int64_t total = (int64_t)(obs->n_samples / obs->samples_per_int) * (obs->n_fine / obs->chan_avg);
    if ((int64_t)first_image + n_images > total)
        return set_error(BLINK_ERR_INVALID_ARG, "image range beyond the observation's T * F images");
    BLINK_TRY(make_current(ctx));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Plan* p = nullptr;
    BLINK_TRY(get_plan(ctx, array, obs, imaging, true, st, &p));
    if (n_images == 0) return BLINK_OK;
    BLINK_TRY(launch_grid_gather(*p, d_vis, first_image, n_images, d_grid, ctx->d_status, st));
    if (d_weight) {
        k_fill_weights<<<(n_images + 255) / 256, 256, 0, st>>>(d_weight, p->d_W, p->F, first_image, n_images);
        BLINK_CUDA(cudaGetLastError());
    }
    return BLINK_OK;
}

blink_status blink_image(blink_context* ctx, const blink_imaging* imaging, const float* d_grid, int32_t n_images,
                         const float* d_weight, float* d_img, void* stream) {
    BLINK_TRY(check_imaging(imaging));
    BLINK_TRY(nearest_only(imaging, "blink_image"));
    if (!d_grid || !d_weight || !d_img) return set_error(BLINK_ERR_INVALID_ARG, "d_grid, d_weight or d_img is NULL");
    if (n_images < 0) return set_error(BLINK_ERR_INVALID_ARG, "n_images < 0");
    if (((uintptr_t)d_grid & 7) || ((uintptr_t)d_img & 7))
        return set_error(BLINK_ERR_INVALID_ARG, "d_grid and d_img must be 8-byte aligned");
    BLINK_TRY(make_current(ctx));
    if (n_images == 0) return BLINK_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int N = imaging->n_pix, prec = imaging->precision;
    if (!fast_side(N)) {
        MixedIn in;
        in.N = N;
        BLINK_TRY(twiddles(ctx, N, const_cast<float2**>(&in.tw)));
        const size_t per_img = (size_t)N * mixed_h_row(N) * (prec == BLINK_PREC_BF16 ? 4 : 8);
        const int wave = (int)std::max<size_t>(1, std::min<size_t>({(size_t)n_images, (size_t)65535, ((size_t)48 << 20) / per_img}));
        void* H = nullptr;
        BLINK_TRY(workspace(ctx, 1, (size_t)wave * per_img, &H));
        for (int w0 = 0; w0 < n_images; w0 += wave) {
            const int nw = std::min(wave, n_images - w0);
            in.grid = reinterpret_cast<const float2*>(d_grid) + (int64_t)w0 * N * (N / 2 + 1);
            BLINK_TRY(launch_mixed(in, 0, prec, nw, H, nullptr, 1, WaveMap{1, 0, w0, nw}, 0, nullptr, st));
            BLINK_TRY(launch_mixed(in, 1, prec, nw, H, d_weight, n_images, WaveMap{1, 0, w0, nw}, 0, d_img, st));
        }
        return BLINK_OK;
    }
    const int cw = col_block_width(N);
    const int ldh = N / 2 + cw;                 // room for the Nyquist column u = N/2
    float2* tw = nullptr;
    BLINK_TRY(twiddles(ctx, N, &tw));
    const size_t el = prec == BLINK_PREC_BF16 ? 4 : 8;
    const size_t per_img = (size_t)N * ldh * el;
    const int wave = (int)std::min<size_t>((size_t)n_images, std::max<size_t>(1, ((size_t)64 << 20) / per_img));
    void* H = nullptr;
    BLINK_TRY(workspace(ctx, 1, (size_t)wave * per_img, &H));
    for (int w0 = 0; w0 < n_images; w0 += wave) {
        const int nw = std::min(wave, n_images - w0);
        BLINK_TRY(launch_colpass_grid(N, prec, tw,
                                      reinterpret_cast<const float2*>(d_grid) + (int64_t)w0 * N * (N / 2 + 1), nw, H,
                                      ldh, st));
        BLINK_TRY(launch_rowpass(N, prec, tw, H, ldh, 1, d_weight, n_images, WaveMap{1, 0, w0, nw}, nw, 0, d_img, st));
    }
    return BLINK_OK;
}

blink_status blink_pipeline(blink_context* ctx, const blink_array* array, const blink_obs* obs,
                            const blink_imaging* imaging, int32_t arith, int32_t mode, const uint8_t* d_volt,
                            float* d_img, float* d_weight, void* stream) {
    BLINK_TRY(check_array(array));
    BLINK_TRY(check_obs(obs, true));
    BLINK_TRY(check_imaging(imaging));
    if (arith != BLINK_CORR_FP32 && arith != BLINK_CORR_FP8)
        return set_error(BLINK_ERR_INVALID_ARG, "arith must be BLINK_CORR_FP32 or BLINK_CORR_FP8");
    if (mode != BLINK_MODE_BATCHED && mode != BLINK_MODE_PLAIN)
        return set_error(BLINK_ERR_INVALID_ARG, "mode must be BLINK_MODE_BATCHED or BLINK_MODE_PLAIN");
    if (mode == BLINK_MODE_PLAIN) BLINK_TRY(nearest_only(imaging, "blink_pipeline (plain form)"));
    if (!d_volt || !d_img) return set_error(BLINK_ERR_INVALID_ARG, "d_volt or d_img is NULL");
    if (((uintptr_t)d_volt & 1) || ((uintptr_t)d_img & 7))
        return set_error(BLINK_ERR_INVALID_ARG, "d_volt must be 2-byte and d_img 8-byte aligned");
    BLINK_TRY(make_current(ctx));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Plan* p = nullptr;
    BLINK_TRY(get_plan(ctx, array, obs, imaging, true, st, &p));
    const int T = obs->n_samples / obs->samples_per_int;
    const int n_img = T * p->F;
    if (n_img == 0) return BLINK_OK;
    const int64_t ss = sample_stride_bytes(obs, array->n_tiles);
    const int N = p->N;
    GainRef g;
    BLINK_TRY(upload_gains(ctx, array, p->F, st, &g));
    if (mode == BLINK_MODE_BATCHED) {
        BLINK_TRY(run_batched(ctx, *p, obs, imaging->precision, arith, d_volt, ss, 0, T, d_img, st, true, g));
    } else if (!fast_side(N)) {
        // the plain form on a mixed-radix side: per image, atomic gridding into a stored grid, then the
        // column and row passes of that grid
        const size_t el = imaging->precision == BLINK_PREC_BF16 ? 4 : 8;
        void *vis = nullptr, *H = nullptr, *grid = nullptr;
        BLINK_TRY(workspace(ctx, 0, (size_t)p->B * sizeof(float2), &vis));
        BLINK_TRY(workspace(ctx, 1, (size_t)N * mixed_h_row(N) * el, &H));
        BLINK_TRY(workspace(ctx, 2, (size_t)N * (N / 2 + 1) * sizeof(float2), &grid));
        const int kind = p->pol == BLINK_POL_I ? CORR_OUT_STOKES_I : CORR_OUT_XX;
        ImgOut io;
        io.phase = p->d_phase;
        MixedIn in;
        in.N = N;
        in.tw = p->d_tw;
        in.grid = static_cast<const float2*>(grid);
        for (int id = 0; id < n_img; id++) {
            if (arith == BLINK_CORR_FP8)
                BLINK_TRY(launch_corr_fp8(kind, d_volt, ss, *p, obs->samples_per_int, id, 1, vis, p->B, ctx->d_status,
                                          ctx->n_sm, st, g, io));
            else
                BLINK_TRY(launch_corr_fp32(kind, d_volt, ss, *p, obs->samples_per_int, id, 1, vis, p->B,
                                           ctx->d_status, st, g, io));
            BLINK_CUDA(cudaMemsetAsync(grid, 0, (size_t)N * (N / 2 + 1) * sizeof(float2), st));
            BLINK_TRY(launch_grid_atomic(*p, static_cast<float2*>(vis), id, static_cast<float2*>(grid), st));
            const WaveMap wm{p->F, id % p->F, id / p->F, 1};
            BLINK_TRY(launch_mixed(in, 0, imaging->precision, 1, H, nullptr, 1, wm, 0, nullptr, st));
            BLINK_TRY(launch_mixed(in, 1, imaging->precision, 1, H, p->d_Wk, p->F, wm, 0, d_img, st));
        }
    } else {
        const int cw = p->cw, ldh = N / 2 + cw;
        const size_t el = imaging->precision == BLINK_PREC_BF16 ? 4 : 8;
        void *vis = nullptr, *H = nullptr, *grid = nullptr;
        BLINK_TRY(workspace(ctx, 0, (size_t)p->B * sizeof(float2), &vis));
        BLINK_TRY(workspace(ctx, 1, (size_t)N * ldh * el, &H));
        BLINK_TRY(workspace(ctx, 2, (size_t)N * (N / 2 + 1) * sizeof(float2), &grid));
        const int kind = p->pol == BLINK_POL_I ? CORR_OUT_STOKES_I : CORR_OUT_XX;
        ImgOut io;
        io.phase = p->d_phase;
        for (int id = 0; id < n_img; id++) {
            if (arith == BLINK_CORR_FP8)
                BLINK_TRY(launch_corr_fp8(kind, d_volt, ss, *p, obs->samples_per_int, id, 1, vis, p->B, ctx->d_status,
                                          ctx->n_sm, st, g, io));
            else
                BLINK_TRY(launch_corr_fp32(kind, d_volt, ss, *p, obs->samples_per_int, id, 1, vis, p->B,
                                           ctx->d_status, st, g, io));
            BLINK_CUDA(cudaMemsetAsync(grid, 0, (size_t)N * (N / 2 + 1) * sizeof(float2), st));
            BLINK_TRY(launch_grid_atomic(*p, static_cast<float2*>(vis), id, static_cast<float2*>(grid), st));
            BLINK_TRY(launch_colpass_grid(N, imaging->precision, p->d_tw, static_cast<float2*>(grid), 1, H, ldh, st));
            BLINK_TRY(launch_rowpass(N, imaging->precision, p->d_tw, H, ldh, 0, p->d_Wk, p->F,
                                     WaveMap{p->F, id % p->F, id / p->F, 1}, 1, 0, d_img, st));
        }
    }
    if (d_weight) {
        k_fill_weights<<<(n_img + 255) / 256, 256, 0, st>>>(d_weight, p->d_W, p->F, 0, n_img);
        BLINK_CUDA(cudaGetLastError());
    }
    return BLINK_OK;
}

blink_status blink_pipeline_tracking(blink_context* ctx, const blink_array* array, const blink_obs* obs,
                                     const blink_imaging* imaging, const double* h_lm, int32_t arith,
                                     const uint8_t* d_volt, float* d_img, void* stream) {
    BLINK_TRY(check_array(array));
    BLINK_TRY(check_obs(obs, true));
    BLINK_TRY(check_imaging(imaging));
    if (arith != BLINK_CORR_FP32 && arith != BLINK_CORR_FP8)
        return set_error(BLINK_ERR_INVALID_ARG, "arith must be BLINK_CORR_FP32 or BLINK_CORR_FP8");
    if (!h_lm || !d_volt || !d_img) return set_error(BLINK_ERR_INVALID_ARG, "h_lm, d_volt or d_img is NULL");
    if (((uintptr_t)d_volt & 1) || ((uintptr_t)d_img & 7))
        return set_error(BLINK_ERR_INVALID_ARG, "d_volt must be 2-byte and d_img 8-byte aligned");
    const int T = obs->n_samples / obs->samples_per_int;
    for (int t = 0; t < T; t++) {
        const double l = h_lm[2 * t], m = h_lm[2 * t + 1];
        if (!std::isfinite(l) || !std::isfinite(m) || !(l * l + m * m < 1.0))
            return set_error(BLINK_ERR_INVALID_ARG, "h_lm: every pointing must be direction cosines with l^2 + m^2 < 1");
    }
    BLINK_TRY(make_current(ctx));
    if (T == 0) return BLINK_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t ss = sample_stride_bytes(obs, array->n_tiles);
    blink_imaging im = *imaging;
    GainRef g;
    bool have_g = false;
    for (int ta = 0; ta < T;) {
        int tb = ta + 1;
        while (tb < T && h_lm[2 * tb] == h_lm[2 * ta] && h_lm[2 * tb + 1] == h_lm[2 * ta + 1]) tb++;
        im.phase_l = h_lm[2 * ta];
        im.phase_m = h_lm[2 * ta + 1];
        Plan* p = nullptr;
        BLINK_TRY(get_plan(ctx, array, obs, &im, true, st, &p));
        if (im.cell_lambda <= 0.0) im.cell_lambda = p->du;      // one pixel scale for the whole call
        if (!have_g) {
            BLINK_TRY(upload_gains(ctx, array, p->F, st, &g));
            have_g = true;
        }
        // run_batched writes image tau0 * F at its output pointer
        BLINK_TRY(run_batched(ctx, *p, obs, im.precision, arith, d_volt, ss, ta, tb,
                              d_img + (int64_t)ta * p->F * p->Ni * p->Ni, st, true, g));
        ta = tb;
    }
    return BLINK_OK;
}

blink_status blink_pipeline_averaged(blink_context* ctx, const blink_array* array, const blink_obs* obs,
                                     const blink_imaging* imaging, int32_t arith, int32_t t_avg, int32_t f_avg,
                                     const uint8_t* d_volt, float* d_img, void* stream) {
    BLINK_TRY(check_array(array));
    BLINK_TRY(check_obs(obs, true));
    BLINK_TRY(check_imaging(imaging));
    if (arith != BLINK_CORR_FP32 && arith != BLINK_CORR_FP8)
        return set_error(BLINK_ERR_INVALID_ARG, "arith must be BLINK_CORR_FP32 or BLINK_CORR_FP8");
    const int T = obs->n_samples / obs->samples_per_int, F = obs->n_fine / obs->chan_avg;
    if (t_avg < 1 || f_avg < 1 || (T > 0 && T % t_avg) || F % f_avg)
        return set_error(BLINK_ERR_INVALID_ARG, "t_avg and f_avg must be >= 1 and divide the integrations and the "
                                                "output channels of the call");
    if ((int64_t)obs->samples_per_int * t_avg > INT32_MAX)
        return set_error(BLINK_ERR_INVALID_ARG, "t_avg * samples_per_int overflows");
    if (!d_volt || !d_img) return set_error(BLINK_ERR_INVALID_ARG, "d_volt or d_img is NULL");
    if (((uintptr_t)d_volt & 1) || ((uintptr_t)d_img & 7))
        return set_error(BLINK_ERR_INVALID_ARG, "d_volt must be 2-byte and d_img 8-byte aligned");
    BLINK_TRY(make_current(ctx));
    if (T == 0) return BLINK_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the mean over t_avg integrations is the image of their summed correlations (one pointing, so the
    // cells do not change within the call): correlate over integrations t_avg times longer
    blink_obs ob = *obs;
    ob.samples_per_int = obs->samples_per_int * t_avg;
    Plan* p = nullptr;
    BLINK_TRY(get_plan(ctx, array, &ob, imaging, true, st, &p));
    GainRef g;
    BLINK_TRY(upload_gains(ctx, array, p->F, st, &g));
    return run_mixed(ctx, *p, &ob, imaging->precision, arith, d_volt, sample_stride_bytes(obs, array->n_tiles), 0,
                     T / t_avg, d_img, st, g, f_avg);
}

blink_status blink_pipeline_sets(blink_context* ctx, const blink_array* array, const blink_obs* obs,
                                 const blink_set* sets, int32_t n_sets, int32_t arith, const uint8_t* d_volt,
                                 float* d_img, size_t img_capacity, void* stream) {
    BLINK_TRY(check_array(array));
    BLINK_TRY(check_obs(obs, true));
    if (arith != BLINK_CORR_FP32 && arith != BLINK_CORR_FP8)
        return set_error(BLINK_ERR_INVALID_ARG, "arith must be BLINK_CORR_FP32 or BLINK_CORR_FP8");
    if (!sets || n_sets < 1) return set_error(BLINK_ERR_INVALID_ARG, "no sets");
    if (!d_volt || !d_img) return set_error(BLINK_ERR_INVALID_ARG, "d_volt or d_img is NULL");
    if (((uintptr_t)d_volt & 1) || ((uintptr_t)d_img & 7))
        return set_error(BLINK_ERR_INVALID_ARG, "d_volt must be 2-byte and d_img 8-byte aligned");
    const int T = obs->n_samples / obs->samples_per_int;
    const int stride = obs->fine_stride ? obs->fine_stride : obs->n_fine;
    // validate every set and the packed output size before launching anything
    size_t need = 0;
    for (int s = 0; s < n_sets; s++) {
        const blink_set& st = sets[s];
        if (st.fine0 < 0 || st.n_fine < 1 || st.fine0 + st.n_fine > obs->n_fine || st.n_fine % obs->chan_avg)
            return set_error(BLINK_ERR_INVALID_ARG, "set channel range outside the buffer or not a multiple of chan_avg");
        BLINK_TRY(check_imaging(&st.imaging));
        need += (size_t)T * (st.n_fine / obs->chan_avg) * st.imaging.n_pix * st.imaging.n_pix;
    }
    if (need > img_capacity) return set_error(BLINK_ERR_INVALID_ARG, "img_capacity smaller than the sets' images");
    if (array->gains || array->jones)
        for (int s = 0; s < n_sets; s++)
            if (sets[s].fine0 % obs->chan_avg)
                return set_error(BLINK_ERR_INVALID_ARG, "with gains, every set must start on an output channel");
    BLINK_TRY(make_current(ctx));
    cudaStream_t strm = static_cast<cudaStream_t>(stream);
    GainRef g_all;
    BLINK_TRY(upload_gains(ctx, array, obs->n_fine / obs->chan_avg, strm, &g_all));
    size_t at = 0;
    for (int s = 0; s < n_sets; s++) {
        const blink_set& st = sets[s];
        blink_array a = *array;
        a.flags = st.flags;
        blink_obs o = *obs;
        o.n_fine = st.n_fine;
        o.fine_stride = stride;
        o.fine_freq_hz = obs->fine_freq_hz + st.fine0;
        Plan* p = nullptr;
        BLINK_TRY(get_plan(ctx, &a, &o, &st.imaging, true, strm, &p));
        const int64_t ss = sample_stride_bytes(&o, a.n_tiles);
        GainRef g = g_all;
        g.f0 = st.fine0 / obs->chan_avg;
        if (T > 0)
            BLINK_TRY(run_batched(ctx, *p, &o, st.imaging.precision, arith, d_volt + (int64_t)st.fine0 * a.n_tiles * 2,
                                  ss, 0, T, d_img + at, strm, true, g));
        at += (size_t)T * p->F * p->Ni * p->Ni;
    }
    return BLINK_OK;
}

blink_status blink_dedisperse(blink_context* ctx, const float* d_img, int32_t n_int, int32_t n_chan, int32_t n_pix,
                              const int32_t* h_delays, float* d_out, void* stream) {
    if (!d_img || !d_out || !h_delays) return set_error(BLINK_ERR_INVALID_ARG, "d_img, d_out or h_delays is NULL");
    if (n_int < 1 || n_chan < 1) return set_error(BLINK_ERR_INVALID_ARG, "n_int and n_chan must be >= 1");
    if (n_pix < 64 || n_pix > 8192 || (n_pix & 1))
        return set_error(BLINK_ERR_INVALID_ARG, "n_pix must be even, in [64, 8192]");
    if (((uintptr_t)d_img & 15) || ((uintptr_t)d_out & 15))
        return set_error(BLINK_ERR_INVALID_ARG, "d_img and d_out must be 16-byte aligned");
    int dmax = 0;
    for (int f = 0; f < n_chan; f++) {
        if (h_delays[f] < 0) return set_error(BLINK_ERR_INVALID_ARG, "delays must be >= 0");
        dmax = std::max(dmax, (int)h_delays[f]);
    }
    if (dmax >= n_int) return set_error(BLINK_ERR_INVALID_ARG, "max(delays) must be < n_int");
    BLINK_TRY(make_current(ctx));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* d = nullptr;
    BLINK_TRY(workspace(ctx, 7, sizeof(int32_t) * (size_t)n_chan, &d));
    BLINK_CUDA(cudaMemcpyAsync(d, h_delays, sizeof(int32_t) * (size_t)n_chan, cudaMemcpyHostToDevice, st));
    return launch_dedisperse(d_img, n_int - dmax, n_chan, n_pix, static_cast<const int*>(d), d_out, st);
}

blink_status blink_dedisperse_stream(blink_context* ctx, float* d_carry, int64_t t0, const float* d_img, int32_t n_int,
                                     int32_t n_chan, int32_t n_pix, const int32_t* h_delays, float* d_out,
                                     int32_t* h_n_out, void* stream) {
    if (!d_img || !d_out || !h_delays || !h_n_out)
        return set_error(BLINK_ERR_INVALID_ARG, "d_img, d_out, h_delays or h_n_out is NULL");
    *h_n_out = 0;
    if (n_int < 1 || n_chan < 1) return set_error(BLINK_ERR_INVALID_ARG, "n_int and n_chan must be >= 1");
    if (t0 < 0) return set_error(BLINK_ERR_INVALID_ARG, "t0 must be >= 0");
    if (n_pix < 64 || n_pix > 8192 || (n_pix & 1))
        return set_error(BLINK_ERR_INVALID_ARG, "n_pix must be even, in [64, 8192]");
    int dmax = 0;
    for (int f = 0; f < n_chan; f++) {
        if (h_delays[f] < 0) return set_error(BLINK_ERR_INVALID_ARG, "delays must be >= 0");
        dmax = std::max(dmax, (int)h_delays[f]);
    }
    if (dmax > 0 && !d_carry) return set_error(BLINK_ERR_INVALID_ARG, "d_carry is NULL while max(delays) > 0");
    if (((uintptr_t)d_img & 15) || ((uintptr_t)d_out & 15) || ((uintptr_t)d_carry & 15))
        return set_error(BLINK_ERR_INVALID_ARG, "d_img, d_out and d_carry must be 16-byte aligned");
    BLINK_TRY(make_current(ctx));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* d = nullptr;
    BLINK_TRY(workspace(ctx, 7, sizeof(int32_t) * (size_t)n_chan, &d));
    BLINK_CUDA(cudaMemcpyAsync(d, h_delays, sizeof(int32_t) * (size_t)n_chan, cudaMemcpyHostToDevice, st));
    int n_out = 0;
    BLINK_TRY(launch_dedisperse_stream(d_img, t0, n_int, n_chan, n_pix, static_cast<const int*>(d), dmax, d_carry, d_out,
                                       &n_out, st));
    *h_n_out = n_out;
    return BLINK_OK;
}

blink_status blink_pipeline_host(blink_context* ctx, const blink_array* array, const blink_obs* obs,
                                 const blink_imaging* imaging, int32_t arith, const uint8_t* h_volt, float* h_img,
                                 int32_t images_per_pass, void* stream) {
    BLINK_TRY(check_array(array));
    BLINK_TRY(check_obs(obs, true));
    BLINK_TRY(check_imaging(imaging));
    if (arith != BLINK_CORR_FP32 && arith != BLINK_CORR_FP8)
        return set_error(BLINK_ERR_INVALID_ARG, "arith must be BLINK_CORR_FP32 or BLINK_CORR_FP8");
    if (!h_volt || !h_img) return set_error(BLINK_ERR_INVALID_ARG, "h_volt or h_img is NULL");
    if (images_per_pass < 0) return set_error(BLINK_ERR_INVALID_ARG, "images_per_pass < 0");
    BLINK_TRY(make_current(ctx));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Plan* p = nullptr;
    BLINK_TRY(get_plan(ctx, array, obs, imaging, true, st, &p));
    const int T = obs->n_samples / obs->samples_per_int;
    const int n_img = T * p->F;
    if (n_img == 0) return BLINK_OK;
    const int64_t ss = sample_stride_bytes(obs, array->n_tiles);
    const size_t vbytes = (size_t)obs->n_samples * ss;
    GainRef g;
    BLINK_TRY(upload_gains(ctx, array, p->F, st, &g));
    // output the device can write: the imaging kernel writes the images straight into h_img, so the transfer
    // over the host link overlaps the computation instead of following it
    float* direct = images_per_pass == 0 ? device_view(h_img, (size_t)n_img * p->Ni * p->Ni * sizeof(float)) : nullptr;
    if (direct) {
        void* dv = nullptr;
        BLINK_TRY(workspace(ctx, 2, vbytes, &dv));
        BLINK_CUDA(cudaMemcpyAsync(dv, h_volt, vbytes, cudaMemcpyHostToDevice, st));
        return run_batched(ctx, *p, obs, imaging->precision, arith, static_cast<uint8_t*>(dv), ss, 0, T, direct, st,
                           false, g);
    }
    // passes of whole integrations (F images each), at least one integration per pass
    const int t_per = images_per_pass > 0 ? std::max(1, std::min(T, images_per_pass / p->F)) : T;
    const int N = p->Ni;                                // image side
    void* dv = nullptr;
    void* di = nullptr;
    BLINK_TRY(workspace(ctx, 2, vbytes, &dv));
    BLINK_TRY(workspace(ctx, 3, (size_t)t_per * p->F * N * N * sizeof(float), &di));
    BLINK_CUDA(cudaMemcpyAsync(dv, h_volt, vbytes, cudaMemcpyHostToDevice, st));
    for (int t0 = 0; t0 < T; t0 += t_per) {
        const int t1 = std::min(T, t0 + t_per);
        const size_t n = (size_t)(t1 - t0) * p->F;
        BLINK_TRY(run_batched(ctx, *p, obs, imaging->precision, arith, static_cast<uint8_t*>(dv), ss, t0, t1,
                              static_cast<float*>(di), st, true, g));
        BLINK_CUDA(cudaMemcpyAsync(h_img + (int64_t)t0 * p->F * N * N, di, n * N * N * sizeof(float),
                                   cudaMemcpyDeviceToHost, st));
    }
    return BLINK_OK;
}

}  // extern "C"
