// Transforms of fixed length whose stages are planned at compile time (the mixed-radix passes' fast form for
// the paper's 1200^2 images, Sec. 6.2): every stage's radix, stride and butterfly count are constants, so a
// butterfly's addresses are a base plus immediates and its twiddles are single reads of a table of unit roots
// in shared memory.  The stages are Stockham autosort steps between two shared-memory buffers, like the
// generic passes, with larger register radices (16, 15, 8, 5) and so fewer stages.
#pragma once

#include "blink_internal.cuh"

namespace blink {

// i + i / 2^S: one pad slot per 2^S points (S < 0: none).  The first stage writes R = 2^S consecutive points
// per thread; with the pad its threads' writes fall in distinct banks.
template <int S> __host__ __device__ __forceinline__ int padk(int i) { return S >= 0 ? i + (i >> S) : i; }

// One Stockham stage of radix R of an N-point inverse transform after stages whose radices multiply to L, by
// NT threads (thread t takes the butterflies t, t + NT, ...).  Butterfly b = j L + k1 (j < N / (L R)) reads
// the points b + p N / R (p < R) of `in` (addressed through padk<SI>), multiplies point p by w^(p k1 m)
// (w = exp(+2 pi i / N), m = N / (L R); roots[x RS] = w^x), transforms over p and writes output q to
// j L R + k1 + q L of `out` (through padk<SO>).  After all stages the result is in natural order.
template <int N, int R, int L, int NT, int SI, int SO, int RS>
__host__ __device__ __forceinline__ void stage_ct(const float2* in, float2* out, const float2* roots, int t) {
    constexpr int nb = N / R, m = nb / L;
    static_assert(N % (R * L) == 0, "radix plan does not divide the length");
#pragma unroll
    for (int i = 0; i < (nb + NT - 1) / NT; i++) {
        const int b = t + i * NT;
        if (nb % NT != 0 && b >= nb) break;
        const int j = b / L, k1 = b - j * L;
        float2 v[R];
#pragma unroll
        for (int p = 0; p < R; p++) v[p] = in[padk<SI>(b + p * nb)];
        if (L > 1) {
            const int e = k1 * m * RS;
#pragma unroll
            for (int p = 1; p < R; p++) v[p] = cmul(v[p], roots[p * e]);
        }
        idft<R>(v);
        const int d = j * L * R + k1;
#pragma unroll
        for (int q = 0; q < R; q++) out[padk<SO>(d + q * L)] = v[q];
    }
}

// The 1200-point column transform (radices 16, 15, 5) by 80 threads: input a[0, 1200), natural order; the
// first stage's output is padded (1275 slots of b); the result is b[0, 1200) in natural order.
constexpr int kCol1200Threads = 80;
constexpr int kCol1200Slots = 1200 + 1200 / 16;
template <typename Sync>
__host__ __device__ __forceinline__ void fft1200_cols(float2* a, float2* b, const float2* roots, int t, Sync sync) {
    stage_ct<1200, 16, 1, kCol1200Threads, -1, 4, 1>(a, b, roots, t);
    sync();
    stage_ct<1200, 15, 16, kCol1200Threads, 4, -1, 1>(b, a, roots, t);
    sync();
    stage_ct<1200, 5, 240, kCol1200Threads, -1, -1, 1>(a, b, roots, t);
    sync();
}

// The 600-point transform of the 1200-point complex-to-real rows (radices 8, 15, 5) by 40 threads, with the
// unit roots of 600 (roots[x] = exp(+2 pi i x / 600)): input a[0, 600), result b[0, 600) in natural order
// (first-stage output padded, 675 slots).
constexpr int kRow600Threads = 40;
constexpr int kRow600Slots = 600 + 600 / 8;
template <typename Sync>
__host__ __device__ __forceinline__ void fft600_rows(float2* a, float2* b, const float2* roots, int t, Sync sync) {
    stage_ct<600, 8, 1, kRow600Threads, -1, 3, 1>(a, b, roots, t);
    sync();
    stage_ct<600, 15, 8, kRow600Threads, 3, -1, 1>(b, a, roots, t);
    sync();
    stage_ct<600, 5, 120, kRow600Threads, -1, -1, 1>(a, b, roots, t);
    sync();
}

}  // namespace blink
