// Baseline geometry in FP64 (Sec. 5.2.3-5.2.4): (u, v, w) per baseline and output channel, and the
// nearest uv cell.  Each operation is an explicitly rounded FP64 intrinsic, in a fixed order, so the
// result is the correctly rounded value of that sequence (no fused multiply-add).  Off zenith, (u, v, w)
// are the baseline's components on the pointing's basis (e_l, e_m, s0) times nu / c, and the phase
// exp(+2 pi i w) that centres the visibilities on the pointing is tabled per baseline and channel.
#include "blink_internal.cuh"

namespace blink {

namespace {

constexpr double kSpeedOfLight = 299792458.0;   // m/s

struct Basis {
    double e[9];    // e_l, e_m, s0 in (E, N, Up)
};

// (d . e[k..k+2]) as ((d0 e0 + d1 e1) + d2 e2), each step rounded once
__device__ __forceinline__ double dot3(double dx, double dy, double dz, const double* e) {
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, e[0]), __dmul_rn(dy, e[1])), __dmul_rn(dz, e[2]));
}

__global__ void k_cells(const double* __restrict__ enu, const short2* __restrict__ bl,
                        const uint8_t* __restrict__ flags, const double* __restrict__ freq, int64_t B, int F,
                        double du, int half, int phased, Basis bs, uint32_t* __restrict__ cells,
                        double* __restrict__ uvw, float2* __restrict__ phase) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * F) return;
    const int f = (int)(idx / B);
    const int64_t b = idx - (int64_t)f * B;
    const short2 ij = bl[b];
    const int i = ij.x, j = ij.y;
    const double inv_lambda = __ddiv_rn(freq[f], kSpeedOfLight);
    const double dx = __dsub_rn(enu[i * 3 + 0], enu[j * 3 + 0]);
    const double dy = __dsub_rn(enu[i * 3 + 1], enu[j * 3 + 1]);
    const double dz = __dsub_rn(enu[i * 3 + 2], enu[j * 3 + 2]);
    double u, v, w;
    if (phased) {
        u = __dmul_rn(dot3(dx, dy, dz, bs.e + 0), inv_lambda);
        v = __dmul_rn(dot3(dx, dy, dz, bs.e + 3), inv_lambda);
        w = __dmul_rn(dot3(dx, dy, dz, bs.e + 6), inv_lambda);
    } else {
        u = __dmul_rn(dx, inv_lambda);
        v = __dmul_rn(dy, inv_lambda);
        w = __dmul_rn(dz, inv_lambda);
    }
    if (phase) {
        // exp(+2 pi i w) from w's fractional part (exact), sin and cos of pi * (2 fr) in FP64
        const double fr = __dsub_rn(w, rint(w));
        double sn, cs;
        sincospi(2.0 * fr, &sn, &cs);
        phase[idx] = make_float2((float)cs, (float)sn);
    }
    if (uvw) {
        uvw[idx * 3 + 0] = u;
        uvw[idx * 3 + 1] = v;
        uvw[idx * 3 + 2] = w;
    }
    const double x = floor(__dadd_rn(__ddiv_rn(u, du), 0.5));
    const double y = floor(__dadd_rn(__ddiv_rn(v, du), 0.5));
    const bool keep = fabs(x) < (double)half && fabs(y) < (double)half && !flags[i] && !flags[j];
    uint32_t c = CELL_NONE;
    if (keep) c = ((uint32_t)((int)x) & 0xFFFFu) | ((uint32_t)((int)y) << 16);
    cells[idx] = c;
}

// gphase[f][p] = phase[f][gsrc[f][p]]: the phase-centre factors in the gather order of the plan's list
__global__ void k_gather_phase(const float2* __restrict__ phase, const uint16_t* __restrict__ gsrc, int64_t B,
                               int e_stride, int F, float2* __restrict__ gphase) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)F * e_stride) return;
    const int64_t f = idx / e_stride;
    gphase[idx] = phase[f * B + gsrc[idx]];
}

}  // namespace

void launch_cells(const Plan& p, cudaStream_t st) {
    const int64_t n = p.B * p.F;
    const int thr = 256;
    const int64_t blocks = (n + thr - 1) / thr;
    Basis bs;
    for (int k = 0; k < 9; k++) bs.e[k] = p.basis[k];
    k_cells<<<(unsigned)blocks, thr, 0, st>>>(p.d_enu, p.d_bl, p.d_flags, p.d_freq, p.B, p.F, p.du, p.N / 2,
                                              p.phased ? 1 : 0, bs, p.d_cells, p.d_uvw, p.d_phase);
}

blink_status launch_gather_phase(const Plan& p, cudaStream_t st) {
    if (!p.d_phase || !p.d_gsrc || !p.d_gphase) return BLINK_OK;
    const int64_t n = (int64_t)p.F * p.e_stride;
    k_gather_phase<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p.d_phase, p.d_gsrc, p.B, p.e_stride, p.F, p.d_gphase);
    BLINK_CUDA(cudaGetLastError());
    return BLINK_OK;
}

}  // namespace blink
