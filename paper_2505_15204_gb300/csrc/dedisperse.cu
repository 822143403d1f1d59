// Incoherent dedispersion of an image cube (the FRB search the images feed, Sec. 2 and 7):
// out[t][p] = (1/F) sum_f img[t + d_f][f][p] for every output integration t, over the images of
// blink_pipeline (image id = integration * F + channel).  Zero delays give the band-averaged image.
//
// Bandwidth-bound: every output pixel reads F input pixels once.  A thread owns four consecutive pixels
// (16-byte loads) of one output integration and walks the channels with eight loads in flight; the input
// is streamed (evict-first), the output written once.
#include "blink_internal.cuh"

namespace blink {

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 8;

__global__ void __launch_bounds__(kThreads) k_dedisperse(const float4* __restrict__ img, int F, int64_t P4,
                                                       const int* __restrict__ delay, float inv_f,
                                                       float4* __restrict__ out) {
    const int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int t = blockIdx.y;
    if (p >= P4) return;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int f = 0;
    for (; f + kUnroll <= F; f += kUnroll) {
        float4 v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; u++)
            v[u] = __ldcs(img + ((int64_t)(t + __ldg(delay + f + u)) * F + f + u) * P4 + p);
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            acc.x += v[u].x;
            acc.y += v[u].y;
            acc.z += v[u].z;
            acc.w += v[u].w;
        }
    }
    for (; f < F; f++) {
        const float4 v = __ldcs(img + ((int64_t)(t + __ldg(delay + f)) * F + f) * P4 + p);
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
    }
    __stcs(out + (int64_t)t * P4 + p, make_float4(acc.x * inv_f, acc.y * inv_f, acc.z * inv_f, acc.w * inv_f));
}

}  // namespace

blink_status launch_dedisperse(const float* d_img, int n_out, int F, int n_pix, const int* d_delay, float* d_out,
                               cudaStream_t st) {
    const int64_t P4 = (int64_t)n_pix * n_pix / 4;
    const dim3 grid((unsigned)((P4 + kThreads - 1) / kThreads), (unsigned)n_out);
    k_dedisperse<<<grid, kThreads, 0, st>>>(reinterpret_cast<const float4*>(d_img), F, P4, d_delay, 1.0f / (float)F,
                                            reinterpret_cast<float4*>(d_out));
    BLINK_CUDA(cudaGetLastError());
    return BLINK_OK;
}

}  // namespace blink
