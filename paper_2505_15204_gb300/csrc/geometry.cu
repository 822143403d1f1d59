// Baseline geometry in FP64 (Sec. 5.2.3-5.2.4): (u, v, w) per baseline and output channel, and the
// nearest uv cell.  Each operation is an explicitly rounded FP64 intrinsic, in a fixed order, so the
// result is the correctly rounded value of that sequence (no fused multiply-add).
#include "blink_internal.cuh"

namespace blink {

namespace {

constexpr double kSpeedOfLight = 299792458.0;   // m/s

__global__ void k_cells(const double* __restrict__ enu, const short2* __restrict__ bl,
                        const uint8_t* __restrict__ flags, const double* __restrict__ freq, int64_t B, int F,
                        double du, int half, uint32_t* __restrict__ cells, double* __restrict__ uvw) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * F) return;
    const int f = (int)(idx / B);
    const int64_t b = idx - (int64_t)f * B;
    const short2 ij = bl[b];
    const int i = ij.x, j = ij.y;
    const double inv_lambda = __ddiv_rn(freq[f], kSpeedOfLight);
    const double u = __dmul_rn(__dsub_rn(enu[i * 3 + 0], enu[j * 3 + 0]), inv_lambda);
    const double v = __dmul_rn(__dsub_rn(enu[i * 3 + 1], enu[j * 3 + 1]), inv_lambda);
    const double w = __dmul_rn(__dsub_rn(enu[i * 3 + 2], enu[j * 3 + 2]), inv_lambda);
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

}  // namespace

void launch_cells(const Plan& p, cudaStream_t st) {
    const int64_t n = p.B * p.F;
    const int thr = 256;
    const int64_t blocks = (n + thr - 1) / thr;
    k_cells<<<(unsigned)blocks, thr, 0, st>>>(p.d_enu, p.d_bl, p.d_flags, p.d_freq, p.B, p.F, p.du, p.N / 2,
                                              p.d_cells, p.d_uvw);
}

}  // namespace blink
