// Gridding (Sec. 5.2.4) and the batched inverse 2D FFT (Eq. 4; Sec. 5.2.4) of the Hermitian half plane.
//
// Grid layout: half plane u in [0, N/2], row v (mod N), complex.  The 2D complex-to-real inverse
// transform runs in two passes:
//   column pass: for each u column, an N-point inverse FFT along v   -> H[y][u]
//   row pass:    for each image row y, an N-point complex-to-real inverse FFT along u, formed from an
//                N/2-point complex FFT plus a pre-twiddle, then scaled by 1/W.
// The shift that puts the phase centre at pixel (N/2, N/2) is applied as the factor (-1)^(u+v) on the
// grid (a shift by N/2 in both image axes), so the passes need no index remapping.
//
// Gridding never uses atomics in the batched form: a precomputed, cell-sorted gather list (one entry per
// visibility and mirror that lands in the half plane) lets one thread own each non-empty cell and sum
// its contributions in a fixed order, in shared memory, right before the column FFT of that tile.
#include <algorithm>

#include "blink_internal.cuh"

namespace blink {

namespace {

// ---------------------------------------------------------------------------------------------------
// gather gridding of the 4-polarisation visibility layout into the half-plane grid (blink_grid)
// ---------------------------------------------------------------------------------------------------
constexpr int kGridThreads = 256;

__global__ void __launch_bounds__(kGridThreads)
k_grid_gather(const float* __restrict__ vis4, int64_t B, int F, int first_image, int pol, int N, int cw,
              int n_cb, const int* __restrict__ cell_off, const uint32_t* __restrict__ cell_key,
              const int* __restrict__ cell_beg, const uint32_t* __restrict__ contrib, float2* __restrict__ grid,
              int* status) {
    extern __shared__ float2 sg[];                       // [N][cw]
    const int img = blockIdx.y, cb = blockIdx.x, tid = threadIdx.x;
    const int f = (first_image + img) % F;
    const int u0 = cb * cw, half = N / 2;
    for (int e = tid; e < N * cw; e += kGridThreads) sg[e] = make_float2(0.f, 0.f);
    __syncthreads();
    if (cb < n_cb) {
        const int beg = cell_off[f * (n_cb + 1) + cb], end = cell_off[f * (n_cb + 1) + cb + 1];
        const float* V = vis4 + (int64_t)img * B * 8;
        for (int c = beg + tid; c < end; c += kGridThreads) {
            const uint32_t key = cell_key[c];
            const int v = key >> 16, u = key & 0xFFFF;
            if (v >= N || u < u0 || u >= u0 + cw) {
                dev_fail(status, DEV_ERR_INDEX);
                continue;
            }
            float2 acc = make_float2(0.f, 0.f);
            for (int k = cell_beg[c]; k < cell_beg[c + 1]; k++) {
                const uint32_t w = contrib[k];
                const float* p = V + (int64_t)(w >> 1) * 8;
                float2 val = (pol == BLINK_POL_I) ? make_float2(0.5f * (p[0] + p[6]), 0.5f * (p[1] + p[7]))
                                                  : make_float2(p[0], p[1]);
                if (w & 1) val.y = -val.y;
                acc = cadd(acc, val);
            }
            sg[v * cw + (u - u0)] = acc;
        }
    }
    __syncthreads();
    const int ncols = min(cw, half + 1 - u0);
    for (int e = tid; e < N * ncols; e += kGridThreads) {
        const int v = e / ncols, cc = e - (e / ncols) * ncols;
        grid[((int64_t)img * N + v) * (half + 1) + u0 + cc] = sg[v * cw + cc];
    }
}

// ---------------------------------------------------------------------------------------------------
// atomic gridding of one image's Stokes-I (or XX) visibilities (the plain per-image form)
// ---------------------------------------------------------------------------------------------------
__global__ void k_grid_atomic(const float2* __restrict__ vis, int64_t B, const uint32_t* __restrict__ cells,
                              const short2* __restrict__ bl, int N, int autos, float2* __restrict__ grid) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const uint32_t c = cells[b];
    if (c == CELL_NONE) return;
    const short2 ij = bl[b];
    const float2 val = vis[b];
    const int ld = N / 2 + 1;
    float* g = reinterpret_cast<float*>(grid);
    if (ij.x == ij.y) {
        if (autos) {
            atomicAdd(g + 0, val.x);
            atomicAdd(g + 1, val.y);
        }
        return;
    }
    const int iu = (int16_t)(c & 0xFFFF), iv = (int16_t)(c >> 16);
    auto add = [&](int u, int v, float re, float im) {
        const int64_t o = ((int64_t)((v % N + N) % N) * ld + u) * 2;
        atomicAdd(g + o, re);
        atomicAdd(g + o + 1, im);
    };
    if (iu > 0) {
        add(iu, iv, val.x, val.y);
    } else if (iu < 0) {
        add(-iu, -iv, val.x, -val.y);
    } else {
        add(0, iv, val.x, val.y);
        add(0, -iv, val.x, -val.y);
    }
}

// ---------------------------------------------------------------------------------------------------
// column pass, fused with gather gridding (pipeline): one CTA per (image, block of CW u-columns)
// ---------------------------------------------------------------------------------------------------
template <int N, int CW, int NTHR, typename T>
__global__ void __launch_bounds__(NTHR)
k_colpass_gather(const float2* __restrict__ vis, int64_t vis_stride, int F, int first_image, int n_cb,
                 const int* __restrict__ cell_off, const uint32_t* __restrict__ cell_key,
                 const int* __restrict__ cell_beg, const uint32_t* __restrict__ contrib,
                 const float2* __restrict__ tw, T* __restrict__ H, int ldh, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s = reinterpret_cast<T*>(smem_raw);                 // [N][CW]
    const int img = blockIdx.y, cb = blockIdx.x, tid = threadIdx.x;
    const int f = (first_image + img) % F;
    const int u0 = cb * CW;
    for (int e = tid; e < N * CW; e += NTHR) st_c(s + e, make_float2(0.f, 0.f));
    __syncthreads();
    {
        const int beg = cell_off[f * (n_cb + 1) + cb], end = cell_off[f * (n_cb + 1) + cb + 1];
        const float2* V = vis + (int64_t)img * vis_stride;
        for (int c = beg + tid; c < end; c += NTHR) {
            const uint32_t key = cell_key[c];
            const int v = key >> 16, u = key & 0xFFFF;
            if (v >= N || u < u0 || u >= u0 + CW) {
                dev_fail(status, DEV_ERR_INDEX);
                continue;
            }
            float2 acc = make_float2(0.f, 0.f);
            const int k1 = cell_beg[c + 1];
            for (int k = cell_beg[c]; k < k1; k++) {
                const uint32_t w = __ldg(contrib + k);
                float2 val = __ldg(V + (w >> 1));
                if (w & 1) val.y = -val.y;
                acc = cadd(acc, val);
            }
            if ((u + v) & 1) acc = make_float2(-acc.x, -acc.y);   // (-1)^(u+v): image shift by N/2
            st_c(s + v * CW + (u - u0), acc);
        }
    }
    __syncthreads();
    fft_run<N, 1, CW, NTHR, CW, 1, 1, T>(s, tw, tid);
    T* out = H + (int64_t)img * N * ldh + u0;
    for (int e = tid; e < N * CW; e += NTHR) {
        const int y = e / CW, cc = e % CW;
        out[(int64_t)y * ldh + cc] = s[e];
    }
}

// column pass reading a stored half-plane grid (blink_image and the plain form)
template <int N, int CW, int NTHR, typename T>
__global__ void __launch_bounds__(NTHR)
k_colpass_grid(const float2* __restrict__ grid, const float2* __restrict__ tw, T* __restrict__ H, int ldh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s = reinterpret_cast<T*>(smem_raw);                 // [N][CW]
    const int img = blockIdx.y, cb = blockIdx.x, tid = threadIdx.x;
    const int u0 = cb * CW, half = N / 2;
    const float2* G = grid + (int64_t)img * N * (half + 1);
    for (int e = tid; e < N * CW; e += NTHR) {
        const int v = e / CW, cc = e % CW, u = u0 + cc;
        float2 val = make_float2(0.f, 0.f);
        if (u <= half) {
            val = G[(int64_t)v * (half + 1) + u];
            if ((u + v) & 1) val = make_float2(-val.x, -val.y);
        }
        st_c(s + e, val);
    }
    __syncthreads();
    fft_run<N, 1, CW, NTHR, CW, 1, 1, T>(s, tw, tid);
    T* out = H + (int64_t)img * N * ldh + u0;
    for (int e = tid; e < N * CW; e += NTHR) {
        const int y = e / CW, cc = e % CW;
        out[(int64_t)y * ldh + cc] = s[e];
    }
}

// ---------------------------------------------------------------------------------------------------
// row pass: complex-to-real along u for RB image rows per CTA, scaled by 1/W
//
// With M = N/2 and the half spectrum Z[0..M] of a row (Z[N-k] = conj Z[k]), the real sequence
// x[n] = sum_k Z[k] exp(+2 pi i k n / N) is obtained from y = IDFT_M(Y), x[2m] = Re y[m],
// x[2m+1] = Im y[m], where Y[k] = (Z[k] + conj Z[M-k]) + i (Z[k] - conj Z[M-k]) exp(+2 pi i k / N).
// ---------------------------------------------------------------------------------------------------
template <int N, int RB, int NTHR, typename T>
__global__ void __launch_bounds__(NTHR)
k_rowpass(const T* __restrict__ H, int ldh, int has_nyq, const float* __restrict__ wts, int w_offset, int w_mod,
          const float2* __restrict__ tw, float* __restrict__ img_out) {
    constexpr int M = N / 2;
    constexpr int LS = M + 1;
    __shared__ float2 s[RB * LS];
    const int img = blockIdx.y, y0 = blockIdx.x * RB, tid = threadIdx.x;
    const T* src = H + ((int64_t)img * N + y0) * ldh;
    for (int e = tid; e < RB * M; e += NTHR) {
        const int r = e / M, k = e % M;
        s[r * LS + k] = ld_c(src + (int64_t)r * ldh + k);
    }
    for (int r = tid; r < RB; r += NTHR) s[r * LS + M] = has_nyq ? ld_c(src + (int64_t)r * ldh + M) : make_float2(0.f, 0.f);
    __syncthreads();
    constexpr int PAIRS = M / 2 + 1;
    for (int e = tid; e < RB * PAIRS; e += NTHR) {
        const int r = e / PAIRS, k = e % PAIRS;
        float2* row = s + r * LS;
        const float2 zk = row[k], zm = row[M - k];
        const float2 yk = cadd(cadd(zk, conjf2(zm)), cmul_i(cmul(csub(zk, conjf2(zm)), __ldg(tw + k))));
        if (k > 0 && k < M - k) {
            const float2 ym = cadd(cadd(zm, conjf2(zk)), cmul_i(cmul(csub(zm, conjf2(zk)), __ldg(tw + (M - k)))));
            row[M - k] = ym;
        }
        row[k] = yk;
    }
    __syncthreads();
    fft_run<M, 1, RB, NTHR, 1, LS, 2, float2>(s, tw, tid);
    float w = wts[(w_offset + img) % w_mod];
    const float inv = 1.0f / (w > 0.f ? w : 1.f);
    float2* out = reinterpret_cast<float2*>(img_out + ((int64_t)img * N + y0) * N);
    for (int e = tid; e < RB * M; e += NTHR) {
        const int r = e / M, m = e % M;
        const float2 y = s[r * LS + m];
        out[(int64_t)r * M + m] = make_float2(y.x * inv, y.y * inv);
    }
}

template <typename K>
void set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

constexpr int col_threads(int N) { return N >= 512 ? 512 : 256; }
constexpr int col_cw(int N) { return N >= 2048 ? 8 : COL_CW; }
constexpr int row_rb(int N) { return N >= 2048 ? 4 : (N >= 1024 ? 8 : 16); }

template <int N, typename T>
blink_status colpass_gather_n(const Plan& p, const float2* vis, int64_t vis_stride, int first_image, int n_images,
                              void* H, int ldh, int* status, cudaStream_t st) {
    constexpr int CW = col_cw(N), NT = col_threads(N);
    auto kern = k_colpass_gather<N, CW, NT, T>;
    const size_t smem = (size_t)N * CW * sizeof(T);
    set_smem(kern, smem);
    for (int i0 = 0; i0 < n_images; i0 += 65535) {
        const int n = std::min(65535, n_images - i0);
        kern<<<dim3(p.n_cb, n), NT, smem, st>>>(vis + (int64_t)i0 * vis_stride, vis_stride, p.F, first_image + i0,
                                                p.n_cb, p.d_cell_off, p.d_cell_key, p.d_cell_beg, p.d_contrib,
                                                p.d_tw, static_cast<T*>(H) + (int64_t)i0 * N * ldh, ldh, status);
    }
    BLINK_CUDA(cudaGetLastError());
    return BLINK_OK;
}

template <int N, typename T>
blink_status colpass_grid_n(const float2* tw, const float2* grid, int n_images, void* H, int ldh, cudaStream_t st) {
    constexpr int CW = col_cw(N), NT = col_threads(N);
    auto kern = k_colpass_grid<N, CW, NT, T>;
    const size_t smem = (size_t)N * CW * sizeof(T);
    set_smem(kern, smem);
    const int nb = (N / 2 + 1 + CW - 1) / CW;
    for (int i0 = 0; i0 < n_images; i0 += 65535) {
        const int n = std::min(65535, n_images - i0);
        kern<<<dim3(nb, n), NT, smem, st>>>(grid + (int64_t)i0 * N * (N / 2 + 1), tw,
                                            static_cast<T*>(H) + (int64_t)i0 * N * ldh, ldh);
    }
    BLINK_CUDA(cudaGetLastError());
    return BLINK_OK;
}

template <int N, typename T>
blink_status rowpass_n(const float2* tw, const void* H, int ldh, int has_nyq, const float* w, int w_offset, int w_mod,
                       int n_images, float* img, cudaStream_t st) {
    constexpr int RB = row_rb(N);
    for (int i0 = 0; i0 < n_images; i0 += 65535) {
        const int n = std::min(65535, n_images - i0);
        k_rowpass<N, RB, 256, T><<<dim3(N / RB, n), 256, 0, st>>>(
            static_cast<const T*>(H) + (int64_t)i0 * N * ldh, ldh, has_nyq, w, w_offset + i0, w_mod, tw,
            img + (int64_t)i0 * N * N);
    }
    BLINK_CUDA(cudaGetLastError());
    return BLINK_OK;
}

#define BLINK_DISPATCH_N(N_, EXPR_T)                                          \
    switch (N_) {                                                             \
        case 64: { constexpr int NN = 64; EXPR_T; }                           \
        case 128: { constexpr int NN = 128; EXPR_T; }                         \
        case 256: { constexpr int NN = 256; EXPR_T; }                         \
        case 512: { constexpr int NN = 512; EXPR_T; }                         \
        case 1024: { constexpr int NN = 1024; EXPR_T; }                       \
        case 2048: { constexpr int NN = 2048; EXPR_T; }                       \
        default: return set_error(BLINK_ERR_UNSUPPORTED, "image side must be a power of two in [64, 2048]"); \
    }

}  // namespace

int col_block_width(int N) { return N >= 2048 ? 8 : COL_CW; }

blink_status launch_grid_gather(const Plan& p, const float* d_vis4, int first_image, int n_images, float* d_grid,
                                int* d_status, cudaStream_t st) {
    const size_t smem = (size_t)p.N * p.cw * sizeof(float2);
    set_smem(k_grid_gather, smem);
    const int nb = p.n_cb + 1;   // one more block for the Nyquist column u = N/2
    for (int i0 = 0; i0 < n_images; i0 += 65535) {
        const int n = std::min(65535, n_images - i0);
        k_grid_gather<<<dim3(nb, n), kGridThreads, smem, st>>>(
            d_vis4 + (int64_t)i0 * p.B * 8, p.B, p.F, first_image + i0, p.pol, p.N, p.cw, p.n_cb, p.d_cell_off,
            p.d_cell_key, p.d_cell_beg, p.d_contrib,
            reinterpret_cast<float2*>(d_grid) + (int64_t)i0 * p.N * (p.N / 2 + 1), d_status);
    }
    BLINK_CUDA(cudaGetLastError());
    return BLINK_OK;
}

blink_status launch_grid_atomic(const Plan& p, const float2* d_visI, int image, float2* d_grid_full,
                                cudaStream_t st) {
    const int f = image % p.F;
    const int thr = 256;
    k_grid_atomic<<<(unsigned)((p.B + thr - 1) / thr), thr, 0, st>>>(d_visI, p.B, p.d_cells + (int64_t)f * p.B,
                                                                     p.d_bl, p.N, p.autos, d_grid_full);
    BLINK_CUDA(cudaGetLastError());
    return BLINK_OK;
}

blink_status launch_colpass_gather(const Plan& p, int prec, const float2* d_visI, int64_t vis_stride,
                                   int first_image, int n_images, void* d_H, int ldh, int* d_status,
                                   cudaStream_t st) {
    if (prec == BLINK_PREC_BF16) {
        BLINK_DISPATCH_N(p.N, return (colpass_gather_n<NN, __nv_bfloat162>(p, d_visI, vis_stride, first_image,
                                                                            n_images, d_H, ldh, d_status, st)));
    }
    BLINK_DISPATCH_N(p.N, return (colpass_gather_n<NN, float2>(p, d_visI, vis_stride, first_image, n_images, d_H,
                                                                ldh, d_status, st)));
}

blink_status launch_colpass_grid(int N, int prec, const float2* d_tw, const float2* d_grid, int n_images,
                                 void* d_H, int ldh, cudaStream_t st) {
    if (prec == BLINK_PREC_BF16) {
        BLINK_DISPATCH_N(N, return (colpass_grid_n<NN, __nv_bfloat162>(d_tw, d_grid, n_images, d_H, ldh, st)));
    }
    BLINK_DISPATCH_N(N, return (colpass_grid_n<NN, float2>(d_tw, d_grid, n_images, d_H, ldh, st)));
}

blink_status launch_rowpass(int N, int prec, const float2* d_tw, const void* d_H, int ldh, int has_nyq,
                            const float* d_w, int w_offset, int w_mod, int n_images, float* d_img,
                            cudaStream_t st) {
    if (prec == BLINK_PREC_BF16) {
        BLINK_DISPATCH_N(N, return (rowpass_n<NN, __nv_bfloat162>(d_tw, d_H, ldh, has_nyq, d_w, w_offset, w_mod,
                                                                   n_images, d_img, st)));
    }
    BLINK_DISPATCH_N(N, return (rowpass_n<NN, float2>(d_tw, d_H, ldh, has_nyq, d_w, w_offset, w_mod, n_images,
                                                       d_img, st)));
}

}  // namespace blink
