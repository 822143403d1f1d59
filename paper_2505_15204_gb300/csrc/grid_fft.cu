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
// visibility and mirror that lands in the half plane) lets the thread holding the first entry of each
// cell sum that cell's contributions in a fixed order, in shared memory, right before the column FFT of
// that tile.  Each warp then transforms one column (or, in the row pass, one row) on its own, so the
// FFT passes synchronise with __syncwarp only.
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
              int n_cb, const int* __restrict__ ent_off, const uint2* __restrict__ ent, float2* __restrict__ grid,
              int* status) {
    extern __shared__ float2 sg[];                       // [N][cw]
    const int img = blockIdx.y, cb = blockIdx.x, tid = threadIdx.x;
    const int f = (first_image + img) % F;
    const int u0 = cb * cw, half = N / 2;
    for (int e = tid; e < N * cw; e += kGridThreads) sg[e] = make_float2(0.f, 0.f);
    __syncthreads();
    if (cb < n_cb) {
        const float* V = vis4 + (int64_t)img * B * 8;
        auto val = [&](uint32_t b) {
            const float* q = V + (int64_t)b * 8;
            return (pol == BLINK_POL_I) ? make_float2(0.5f * (q[0] + q[6]), 0.5f * (q[1] + q[7])) : make_float2(q[0], q[1]);
        };
        auto idx = [&](int u, int v) { return v * cw + (u - u0); };
        const int* off = ent_off + f * (half + 1);
        for (int u = u0 + (tid >> 5); u < min(u0 + cw, half); u += kGridThreads / 32)   // one warp per column
            warp_gather_column(ent, nullptr, off[u], off[u + 1], tid & 31, sg, val, idx, false);
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
// column pass reading a stored half-plane grid (blink_image and the plain form)
template <int N, int CW, int NTHR, typename T>
__global__ void __launch_bounds__(NTHR, (N <= 256 ? 4 : (N <= 512 ? 3 : 1)))
k_colpass_grid(const float2* __restrict__ grid, const float2* __restrict__ tw, T* __restrict__ H, int ldh) {
    static_assert(NTHR == 32 * CW, "one warp per column");
    constexpr int LD = col_ld<N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* stw = reinterpret_cast<float2*>(smem_raw);                 // column-transform twiddle table
    T* s = reinterpret_cast<T*>(smem_raw + (tw_size(N) + 1) / 2 * 2 * sizeof(float2));   // [CW][LD]
    const int img = blockIdx.y, cb = blockIdx.x, tid = threadIdx.x;
    const int u0 = cb * CW, half = N / 2;
    const float2* G = grid + (int64_t)img * N * (half + 1);
    for (int e = tid; e < tw_size(N); e += NTHR) stw[e] = tw[tws_col(N) + e];
    for (int e = tid; e < N * CW; e += NTHR) {
        const int v = e / CW, cc = e % CW, u = u0 + cc;
        float2 val = make_float2(0.f, 0.f);
        if (u <= half) {
            val = G[(int64_t)v * (half + 1) + u];
            if ((u + v) & 1) val = make_float2(-val.x, -val.y);
        }
        st_c(s + cc * LD + padx(v), val);
    }
    __syncthreads();
    NoOut none;
    fft_run<N, 1, 1, 32, 1, 0, true, false, true, T, NoOut, true>(s + (tid >> 5) * LD, stw, tid & 31, none);
    __syncthreads();
    T* out = H + (int64_t)img * N * ldh + u0;
    for (int e = tid; e < N * CW; e += NTHR) {
        const int y = e / CW, c = e % CW;
        out[(int64_t)y * ldh + c] = s[c * LD + padx(y)];
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
k_rowpass(const T* __restrict__ H, int ldh, int has_nyq, const float* __restrict__ wts, int w_mod, WaveMap wm,
          int out_first, const float2* __restrict__ tw, float* __restrict__ img_out) {
    static_assert(NTHR == 32 * RB, "one warp per row");
    constexpr int M = N / 2;
    constexpr int LS = M + M / 16 + 2;          // padded row (padx) with room for the Nyquist slot
    __shared__ float2 spre[M + 1];              // exp(+2 pi i k / N), k in [0, M]
    __shared__ float2 stw[tw_size(M)];          // row-transform twiddle table
    __shared__ float2 s[RB * LS];
    const int img = blockIdx.y, y0 = blockIdx.x * RB, tid = threadIdx.x;
    const int r = tid >> 5, lane = tid & 31;
    for (int e = tid; e <= M; e += NTHR) spre[e] = tw[tws_pre(N) + e];
    for (int e = tid; e < tw_size(M); e += NTHR) stw[e] = tw[tws_row(N) + e];
    __syncthreads();
    // this warp's row: load the half spectrum and form the M-point input of the complex-to-real transform
    const T* row = H + ((int64_t)img * N + y0 + r) * ldh;
    float2* dst = s + r * LS;
    for (int k = lane; k <= M / 2; k += 32) {
        const float2 zk = ld_c(row + k);
        const float2 zm = (k == 0) ? (has_nyq ? ld_c(row + M) : make_float2(0.f, 0.f)) : ld_c(row + (M - k));
        dst[padx(k)] = cadd(cadd(zk, conjf2(zm)), cmul_i(cmul(csub(zk, conjf2(zm)), spre[k])));
        if (k > 0 && k < M - k)
            dst[padx(M - k)] = cadd(cadd(zm, conjf2(zk)), cmul_i(cmul(csub(zm, conjf2(zk)), spre[M - k])));
    }
    __syncwarp();
    const int id = wm.id(img);
    float w = wts[id % w_mod];
    const float inv = 1.0f / (w > 0.f ? w : 1.f);
    float2* out = reinterpret_cast<float2*>(img_out + ((int64_t)(id - out_first) * N + y0 + r) * N);
    auto store = [&](int, int m, float2 y) { out[m] = make_float2(y.x * inv, y.y * inv); };
    fft_run<M, 1, 1, 32, 1, 0, false, true, true, float2, decltype(store), true>(dst, stw, lane, store);
}

template <typename K>
void set_smem(K kernel, size_t bytes) {
    kernel_smem(reinterpret_cast<const void*>(kernel), bytes);
}

constexpr int col_threads(int) { return 32 * COL_CW; }
constexpr int col_cw(int N) { return COL_CW; }
constexpr int row_rb(int N) { return N >= 2048 ? 2 : 8; }

template <int N, typename T>
blink_status colpass_grid_n(const float2* tw, const float2* grid, int n_images, void* H, int ldh, cudaStream_t st) {
    constexpr int CW = col_cw(N), NT = col_threads(N);
    auto kern = k_colpass_grid<N, CW, NT, T>;
    const size_t smem = (size_t)col_ld<N>() * CW * sizeof(T) + (tw_size(N) + 1) / 2 * 2 * sizeof(float2);
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
blink_status rowpass_n(const float2* tw, const void* H, int ldh, int has_nyq, const float* w, int w_mod, WaveMap wm,
                       int n_images, int out_first, float* img, cudaStream_t st) {
    constexpr int RB = row_rb(N);
    set_smem(k_rowpass<N, RB, 32 * RB, T>, 0);
    if (n_images > 65535) return set_error(BLINK_ERR_UNSUPPORTED, "wave of more than 65535 images");
    k_rowpass<N, RB, 32 * RB, T><<<dim3(N / RB, n_images), 32 * RB, 0, st>>>(static_cast<const T*>(H), ldh, has_nyq, w,
                                                                             w_mod, wm, out_first, tw, img);
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

// u columns per gather-gridding CTA: COL_CW, fewer on sides whose column tile would not fit shared memory
int col_block_width(int N) {
    int cw = COL_CW;
    while (cw > 1 && (size_t)N * cw * sizeof(float2) > (size_t)160 * 1024) cw /= 2;
    return cw;
}

namespace {
__device__ float2 unit_root(int k, int n) {     // exp(+2 pi i k / n), FP64 sincospi rounded to FP32
    double sn, cs;
    sincospi(2.0 * (double)k / (double)n, &sn, &cs);
    return make_float2((float)cs, (float)sn);
}

__device__ float2 pass_twiddle(int N, int e) {  // entry e of the per-pass table of an N-point transform
    for (int ns = 1; ns < N; ns *= radix_at(N, ns)) {
        const int R = radix_at(N, ns), sz = (R - 1) * ns;
        if (e < sz) {
            const int r = e / ns + 1, k = e % ns;
            return unit_root(k * r, ns * R);
        }
        e -= sz;
    }
    return make_float2(1.f, 0.f);
}

__global__ void k_make_twiddles(float2* out, int N) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= tws_total(N)) return;
    float2 v = make_float2(0.f, 0.f);
    if (e < tws_col(N)) {
        if (e <= N / 2) v = unit_root(e, N);
    } else if (e < tws_row(N)) {
        if (e - tws_col(N) < tw_size(N)) v = pass_twiddle(N, e - tws_col(N));
    } else if (e - tws_row(N) < tw_size(N / 2)) {
        v = pass_twiddle(N / 2, e - tws_row(N));
    }
    out[e] = v;
}
}  // namespace

blink_status make_twiddles(float2* d_out, int N, cudaStream_t st) {
    k_make_twiddles<<<(tws_total(N) + 255) / 256, 256, 0, st>>>(d_out, N);
    BLINK_CUDA(cudaGetLastError());
    return BLINK_OK;
}

blink_status launch_grid_gather(const Plan& p, const float* d_vis4, int first_image, int n_images, float* d_grid,
                                int* d_status, cudaStream_t st) {
    const size_t smem = (size_t)p.N * p.cw * sizeof(float2);
    set_smem(k_grid_gather, smem);
    const int nb = p.n_cb + 1;   // one more block for the Nyquist column u = N/2
    for (int i0 = 0; i0 < n_images; i0 += 65535) {
        const int n = std::min(65535, n_images - i0);
        k_grid_gather<<<dim3(nb, n), kGridThreads, smem, st>>>(
            d_vis4 + (int64_t)i0 * p.B * 8, p.B, p.F, first_image + i0, p.pol, p.N, p.cw, p.n_cb, p.d_ent_off,
            p.d_ent, reinterpret_cast<float2*>(d_grid) + (int64_t)i0 * p.N * (p.N / 2 + 1), d_status);
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

blink_status launch_colpass_grid(int N, int prec, const float2* d_tw, const float2* d_grid, int n_images,
                                 void* d_H, int ldh, cudaStream_t st) {
    if (prec == BLINK_PREC_BF16) {
        BLINK_DISPATCH_N(N, return (colpass_grid_n<NN, __nv_bfloat162>(d_tw, d_grid, n_images, d_H, ldh, st)));
    }
    BLINK_DISPATCH_N(N, return (colpass_grid_n<NN, float2>(d_tw, d_grid, n_images, d_H, ldh, st)));
}

blink_status launch_rowpass(int N, int prec, const float2* d_tw, const void* d_H, int ldh, int has_nyq,
                            const float* d_w, int w_mod, WaveMap wm, int n_images, int out_first, float* d_img,
                            cudaStream_t st) {
    if (prec == BLINK_PREC_BF16) {
        BLINK_DISPATCH_N(N, return (rowpass_n<NN, __nv_bfloat162>(d_tw, d_H, ldh, has_nyq, d_w, w_mod, wm, n_images,
                                                                   out_first, d_img, st)));
    }
    BLINK_DISPATCH_N(N, return (rowpass_n<NN, float2>(d_tw, d_H, ldh, has_nyq, d_w, w_mod, wm, n_images, out_first,
                                                       d_img, st)));
}

}  // namespace blink
