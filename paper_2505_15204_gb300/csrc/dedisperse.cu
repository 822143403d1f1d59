// Incoherent dedispersion of an image cube (the FRB search the images feed, Sec. 2 and 7):
// out[t][p] = (1/F) sum_f img[t + d_f][f][p] for every output integration t, over the images of
// blink_pipeline (image id = integration * F + channel).  Zero delays give the band-averaged image.
//
// A dispersed burst sweeps the band over seconds (Table 1: tens of seconds at the lowest frequencies), longer
// than one call's cube, so a streaming form takes the cubes of consecutive integration ranges one call at a
// time and carries, for each output still waiting for later integrations, its partial channel sum: D = max(d)
// images of N^2 pixels, whatever the channel count.
//
// Bandwidth-bound: every output pixel reads F input pixels once.  A thread owns four consecutive pixels
// (16-byte loads) of one output integration and walks the channels with eight loads in flight; the input
// is streamed (evict-first), the output written once.
#include <algorithm>

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

// One call of the streaming form: the cube holds integrations [t0, t0 + n) of a longer stream, and blockIdx.y
// walks the outputs t = t_lo + blockIdx.y.  An output's sum starts from its carried partial sum when earlier
// cubes already contributed to it (t < t0), adds its channels that fall in this cube in channel order, and is
// either written out (emit: complete) or carried (slot t mod D) for the next cube.
__global__ void __launch_bounds__(kThreads) k_dedisperse_stream(const float4* __restrict__ img, int F, int64_t P4,
                                                              const int* __restrict__ delay, int64_t t0, int n,
                                                              int64_t t_lo, int D, float4* carry, int emit,
                                                              float inv_f, float4* __restrict__ out) {
    const int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int64_t t = t_lo + blockIdx.y;
    if (p >= P4) return;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t < t0) acc = carry[(t % D) * P4 + p];
    const int64_t base = t - t0;                      // cube integration of channel f: base + d_f
    int f = 0;
    for (; f + kUnroll <= F; f += kUnroll) {
        float4 v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const int64_t tt = base + __ldg(delay + f + u);
            v[u] = (tt >= 0 && tt < n) ? __ldcs(img + (tt * F + f + u) * P4 + p) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            acc.x += v[u].x;
            acc.y += v[u].y;
            acc.z += v[u].z;
            acc.w += v[u].w;
        }
    }
    for (; f < F; f++) {
        const int64_t tt = base + __ldg(delay + f);
        if (tt >= 0 && tt < n) {
            const float4 v = __ldcs(img + (tt * F + f) * P4 + p);
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
    }
    if (emit)
        __stcs(out + (t - t_lo) * P4 + p, make_float4(acc.x * inv_f, acc.y * inv_f, acc.z * inv_f, acc.w * inv_f));
    else
        carry[(t % D) * P4 + p] = acc;
}

}  // namespace

blink_status launch_dedisperse_stream(const float* d_img, int64_t t0, int n, int F, int n_pix, const int* d_delay,
                                      int D, float* d_carry, float* d_out, int* n_out, cudaStream_t st) {
    const int64_t P4 = (int64_t)n_pix * n_pix / 4;
    const unsigned gx = (unsigned)((P4 + kThreads - 1) / kThreads);
    // complete outputs: [max(0, t0 - D), t0 + n - D); outputs still waiting for later cubes: [max(0, t0 + n - D),
    // t0 + n).  The carried slots the second launch writes are those of outputs the first one has emitted or
    // of the outputs it carries on, so the launches run in this order.
    const int64_t a0 = std::max<int64_t>(0, t0 - D), a1 = t0 + n - D;
    *n_out = a1 > a0 ? (int)(a1 - a0) : 0;
    if (*n_out > 0) {
        k_dedisperse_stream<<<dim3(gx, (unsigned)*n_out), kThreads, 0, st>>>(
            reinterpret_cast<const float4*>(d_img), F, P4, d_delay, t0, n, a0, D, reinterpret_cast<float4*>(d_carry), 1,
            1.0f / (float)F, reinterpret_cast<float4*>(d_out));
        BLINK_CUDA(cudaGetLastError());
    }
    const int64_t b0 = std::max<int64_t>(0, t0 + n - D), b1 = t0 + n;
    if (D > 0 && b1 > b0) {
        k_dedisperse_stream<<<dim3(gx, (unsigned)(b1 - b0)), kThreads, 0, st>>>(
            reinterpret_cast<const float4*>(d_img), F, P4, d_delay, t0, n, b0, D, reinterpret_cast<float4*>(d_carry), 0,
            1.0f / (float)F, nullptr);
        BLINK_CUDA(cudaGetLastError());
    }
    return BLINK_OK;
}

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
