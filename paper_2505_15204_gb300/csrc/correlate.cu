// Correlation on CUDA cores (Eq. 2; Sec. 5.2.2), the plain FP32 form.
//
// One CTA per (integration x output channel, block of baselines).  The CTA stages K-chunks of the
// item's voltages in shared memory, unpacked to float4 (X re, X im, Y re, Y im) per tile, and each
// thread accumulates the four polarisation products of BPT baselines.  All values are integers below
// 2^24, so the FP32 sums are exact and independent of the summation order.
#include "blink_internal.cuh"

namespace blink {

namespace {

constexpr int kThreads = 256;
constexpr int kBpt = 2;                               // baselines per thread
constexpr int kStageFloat4 = 3072;                    // 48 KiB of staged samples

__device__ __forceinline__ float nib_lo(unsigned b) { return (float)((int)(b << 28) >> 28); }
__device__ __forceinline__ float nib_hi(unsigned b) { return (float)((int)(b << 24) >> 28); }

// Gains (when given) multiply the products in the epilogue: V^pq = g_i^p S^pq conj(g_j^q).
__device__ __forceinline__ float2 gain_prod(float2 gi, float sr, float si, float2 gjc) {
    const float tr = gi.x * sr - gi.y * si, ti = gi.x * si + gi.y * sr;
    return make_float2(tr * gjc.x - ti * gjc.y, tr * gjc.y + ti * gjc.x);
}

// FULL: gains are 2x2 Jones matrices, V^pq = sum_rs J_i[p][r] S^rs conj(J_j[q][s]); all four products formed.
template <int OUT, bool FULL>
__global__ void __launch_bounds__(kThreads)
k_corr_fp32(const uint8_t* __restrict__ volt, int64_t sample_stride, int n_tiles, int ns, int c, int F,
            int first_item, const short2* __restrict__ bl, int64_t B, const uint8_t* __restrict__ flags,
            void* __restrict__ out, int64_t out_item_stride, int kc, const float2* __restrict__ gains, int gain_f0,
            ImgOut io) {
    extern __shared__ float4 xs[];                    // [kc][n_tiles]
    const int item = first_item + blockIdx.y;
    const int tau = item / F, f = item - (item / F) * F;
    const int K = ns * c;
    const int tid = threadIdx.x;

    int bi[kBpt], bj[kBpt];
    bool act[kBpt];
    float acc[kBpt][8];
#pragma unroll
    for (int m = 0; m < kBpt; m++) {
        const int64_t b = (int64_t)blockIdx.x * kThreads * kBpt + m * kThreads + tid;
        act[m] = b < B;
        bi[m] = 0;
        bj[m] = 0;
        if (act[m]) {
            const short2 ij = bl[b];
            bi[m] = ij.x;
            bj[m] = ij.y;
            act[m] = !flags[ij.x] && !flags[ij.y];
        }
#pragma unroll
        for (int q = 0; q < 8; q++) acc[m][q] = 0.f;
    }

    for (int k0 = 0; k0 < K; k0 += kc) {
        const int kn = min(kc, K - k0);
        for (int e = tid; e < kn * n_tiles; e += kThreads) {
            const int kk = e / n_tiles, a = e - (e / n_tiles) * n_tiles;
            const int k = k0 + kk;
            const int s = tau * ns + k / c, ch = f * c + k % c;
            const unsigned two = *reinterpret_cast<const uint16_t*>(volt + s * sample_stride +
                                                                    ((int64_t)ch * n_tiles + a) * 2);
            xs[kk * n_tiles + a] = make_float4(nib_lo(two & 0xFF), nib_hi(two & 0xFF), nib_lo(two >> 8),
                                               nib_hi(two >> 8));
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < kBpt; m++) {
            if (!act[m]) continue;
            const float4* pi = xs + bi[m];
            const float4* pj = xs + bj[m];
            for (int kk = 0; kk < kn; kk++) {
                const float4 a = pi[kk * n_tiles], b = pj[kk * n_tiles];
                // (ar + i ai) conj(br + i bi) = (ar br + ai bi) + i (ai br - ar bi)
                acc[m][0] += a.x * b.x + a.y * b.y;           // XX
                acc[m][1] += a.y * b.x - a.x * b.y;
                acc[m][6] += a.z * b.z + a.w * b.w;           // YY
                acc[m][7] += a.w * b.z - a.z * b.w;
                if (OUT == CORR_OUT_VIS4 || FULL) {
                    acc[m][2] += a.x * b.z + a.y * b.w;       // XY
                    acc[m][3] += a.y * b.z - a.x * b.w;
                    acc[m][4] += a.z * b.x + a.w * b.y;       // YX
                    acc[m][5] += a.w * b.x - a.z * b.y;
                }
            }
        }
        __syncthreads();
    }

    const float fk = (float)K;
    const float2* g = gains ? gains + (int64_t)(gain_f0 + f) * n_tiles * (FULL ? 4 : 2) : nullptr;
#pragma unroll
    for (int m = 0; m < kBpt; m++) {
        const int64_t b = (int64_t)blockIdx.x * kThreads * kBpt + m * kThreads + tid;
        if (b >= B) continue;
        if (FULL) {
            // V = J_i S J_j^H over the four products (slots 2 (p, q) and 2 (p, q) + 1: re, im)
            const float2* Ji = g + bi[m] * 4;
            const float2* Jj = g + bj[m] * 4;
            float v[8];
#pragma unroll
            for (int pq = 0; pq < 4; pq++) {
                const int p = pq >> 1, q = pq & 1;
                float vr = 0.f, vi = 0.f;
#pragma unroll
                for (int rs = 0; rs < 4; rs++) {
                    const int r = rs >> 1, s2 = rs & 1;
                    const float2 t = gain_prod(Ji[2 * p + r], acc[m][2 * rs], acc[m][2 * rs + 1],
                                               make_float2(Jj[2 * q + s2].x, -Jj[2 * q + s2].y));
                    vr += t.x;
                    vi += t.y;
                }
                v[2 * pq] = vr;
                v[2 * pq + 1] = vi;
            }
#pragma unroll
            for (int q = 0; q < 8; q++) acc[m][q] = v[q];
        } else if (g) {
            // calibrated products (p, q) = (X, X), (X, Y), (Y, X), (Y, Y) in acc slots 0-1, 2-3, 4-5, 6-7
#pragma unroll
            for (int pq = 0; pq < 4; pq++) {
                const int p = pq >> 1, q = pq & 1;
                if (OUT != CORR_OUT_VIS4 && p != q) continue;
                const float2 gi = g[bi[m] * 2 + p], gj = g[bj[m] * 2 + q];
                const float2 v = gain_prod(gi, acc[m][2 * pq], acc[m][2 * pq + 1], make_float2(gj.x, -gj.y));
                acc[m][2 * pq] = v.x;
                acc[m][2 * pq + 1] = v.y;
            }
        }
        if (OUT == CORR_OUT_VIS4) {
            float4* o = reinterpret_cast<float4*>(static_cast<float*>(out) + (int64_t)blockIdx.y * out_item_stride +
                                                  b * 8);
            float r[8];
#pragma unroll
            for (int q = 0; q < 8; q++) r[q] = __fdiv_rn(acc[m][q], fk);
            o[0] = make_float4(r[0], r[1], r[2], r[3]);
            o[1] = make_float4(r[4], r[5], r[6], r[7]);
        } else {
            // imaging kinds: the exact integer sums (the 1/K or 1/2K is applied together with 1/W), times the
            // phase-centre factor when given
            float re = OUT == CORR_OUT_STOKES_I ? acc[m][0] + acc[m][6] : acc[m][0];
            float im = OUT == CORR_OUT_STOKES_I ? acc[m][1] + acc[m][7] : acc[m][1];
            if (io.phase) {
                const float2 ph = io.phase[(int64_t)f * B + b];
                const float r = re * ph.x - im * ph.y, i = re * ph.y + im * ph.x;
                re = r;
                im = i;
            }
            static_cast<float2*>(out)[(int64_t)blockIdx.y * out_item_stride + b] = make_float2(re, im);
        }
    }
}

}  // namespace

template <int OUT, bool FULL>
void corr_fp32(dim3 grid, size_t smem, cudaStream_t st, const uint8_t* d_volt, int64_t sample_stride, const Plan& p,
               int ns, int first, void* o, int64_t out_item_stride, int kc, GainRef gains, ImgOut io) {
    k_corr_fp32<OUT, FULL><<<grid, kThreads, smem, st>>>(d_volt, sample_stride, p.n_tiles, ns, p.chan_avg, p.F, first,
                                                         p.d_bl, p.B, p.d_flags, o, out_item_stride, kc, gains.d, gains.f0,
                                                         OUT == CORR_OUT_VIS4 ? ImgOut{} : io);
}

blink_status launch_corr_fp32(int out_kind, const uint8_t* d_volt, int64_t sample_stride, const Plan& p, int ns,
                              int first_item, int n_items, void* out, int64_t out_item_stride, int*,
                              cudaStream_t st, GainRef gains, ImgOut io) {
    if (io.gather) return set_error(BLINK_ERR_UNSUPPORTED, "the CUDA-core correlator writes baseline order only");
    const int kc = std::max(1, std::min(ns * p.chan_avg, kStageFloat4 / p.n_tiles));
    const size_t smem = (size_t)kc * p.n_tiles * sizeof(float4);
    const unsigned gx = (unsigned)((p.B + kThreads * kBpt - 1) / (kThreads * kBpt));
    for (int i0 = 0; i0 < n_items; i0 += 65535) {
        const int n = std::min(65535, n_items - i0);
        dim3 grid(gx, n);
        char* o = static_cast<char*>(out) + (int64_t)i0 * out_item_stride *
                                                (out_kind == CORR_OUT_VIS4 ? sizeof(float) : sizeof(float2));
        const bool full = gains.d && gains.full;
        switch (out_kind) {
            case CORR_OUT_VIS4:
                if (full) corr_fp32<CORR_OUT_VIS4, true>(grid, smem, st, d_volt, sample_stride, p, ns, first_item + i0, o,
                                                         out_item_stride, kc, gains, io);
                else corr_fp32<CORR_OUT_VIS4, false>(grid, smem, st, d_volt, sample_stride, p, ns, first_item + i0, o,
                                                     out_item_stride, kc, gains, io);
                break;
            case CORR_OUT_STOKES_I:
                if (full) corr_fp32<CORR_OUT_STOKES_I, true>(grid, smem, st, d_volt, sample_stride, p, ns, first_item + i0,
                                                             o, out_item_stride, kc, gains, io);
                else corr_fp32<CORR_OUT_STOKES_I, false>(grid, smem, st, d_volt, sample_stride, p, ns, first_item + i0,
                                                         o, out_item_stride, kc, gains, io);
                break;
            default:
                if (full) corr_fp32<CORR_OUT_XX, true>(grid, smem, st, d_volt, sample_stride, p, ns, first_item + i0, o,
                                                       out_item_stride, kc, gains, io);
                else corr_fp32<CORR_OUT_XX, false>(grid, smem, st, d_volt, sample_stride, p, ns, first_item + i0, o,
                                                   out_item_stride, kc, gains, io);
        }
    }
    BLINK_CUDA(cudaGetLastError());
    return BLINK_OK;
}

}  // namespace blink
