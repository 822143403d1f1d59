// Internal declarations of the GB300 dirty-imaging library (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/blink.h"

namespace blink {

// ------------------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------------------
blink_status set_error(blink_status s, const std::string& msg);
blink_status cuda_error(cudaError_t e, const char* what);

#define BLINK_CUDA(call)                                                     \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return ::blink::cuda_error(e_, #call);        \
    } while (0)

#define BLINK_TRY(call)                                                      \
    do {                                                                     \
        blink_status s_ = (call);                                            \
        if (s_ != BLINK_OK) return s_;                                       \
    } while (0)

// device status word bits
enum : int { DEV_ERR_INDEX = 1, DEV_ERR_TIMEOUT = 2 };

constexpr uint32_t CELL_NONE = 0x80008000u;   // flagged or outside the grid

// ------------------------------------------------------------------------------------------------
// plan: everything that depends only on (array, channels, imaging), built once and cached
// ------------------------------------------------------------------------------------------------
struct Plan {
    uint64_t key = 0;
    int n_tiles = 0, n_fine = 0, chan_avg = 1, F = 0, N = 0, pol = 0, autos = 1;
    int64_t B = 0;
    int cw = 16, n_cb = 0;                 // column-block width and count of the u >= 0 half plane
    double du = 0.0;
    int64_t n_cells = 0, n_contrib = 0, n_dropped = 0;
    std::vector<double> out_freq;          // [F]
    std::vector<float> W;                  // [F] sum of weights per output channel
    // device
    short2* d_bl = nullptr;                // [B] (i, j)
    uint8_t* d_flags = nullptr;            // [n_tiles]
    double* d_enu = nullptr;               // [n_tiles][3]
    double* d_freq = nullptr;              // [F]
    uint32_t* d_cells = nullptr;           // [F][B]
    int* d_cell_off = nullptr;             // [F][n_cb + 1] -> index into cell arrays
    uint32_t* d_cell_key = nullptr;        // [n_cells] (v << 16) | u
    int* d_cell_beg = nullptr;             // [n_cells + 1] -> index into contrib
    uint32_t* d_contrib = nullptr;         // [n_contrib] (b << 1) | conj
    float* d_W = nullptr;                  // [F]
    float2* d_tw = nullptr;                // [N] exp(+2 pi i k / N)
    double* d_uvw = nullptr;               // [F][B][3] (kept for blink_cells)
};

struct Workspace {
    void* ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace blink

struct blink_context {
    int device = 0;
    int n_sm = 0;
    int* d_status = nullptr;
    std::vector<blink::Plan*> plans;       // most recent last
    blink::Workspace ws[4];
    float2* tw[16] = {};                   // twiddle tables by log2(side)
    // per-stage profiling (blink_set_profiling): recorded (stage, start, stop) event pairs and a free pool
    bool profiling = false;
    struct Rec { int stage; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
};

namespace blink {

blink_status get_plan(blink_context* ctx, const blink_array* a, const blink_obs* o, const blink_imaging* im,
                      bool need_gather, cudaStream_t st, Plan** out);
blink_status workspace(blink_context* ctx, int slot, size_t bytes, void** out);
blink_status twiddles(blink_context* ctx, int N, float2** out);

// Brackets one stage launch with profiling events when profiling is on.
struct StageTimer {
    blink_context* ctx;
    int stage;
    cudaStream_t st;
    cudaEvent_t b = nullptr;
    StageTimer(blink_context* c, int s, cudaStream_t stream);
    ~StageTimer();
};

// ---- kernel launchers (defined next to their kernels) --------------------------------------------
void launch_cells(const Plan& p, cudaStream_t st);
blink_status launch_corr_fp32(int out_kind, const uint8_t* d_volt, int64_t sample_stride_bytes, const Plan& p,
                              int ns, int first_item, int n_items, void* out, int64_t out_item_stride,
                              int* d_status, cudaStream_t st);
blink_status launch_corr_fp8(int out_kind, const uint8_t* d_volt, int64_t sample_stride_bytes, const Plan& p,
                             int ns, int first_item, int n_items, void* out, int64_t out_item_stride,
                             int* d_status, int n_sm, cudaStream_t st);
blink_status launch_grid_gather(const Plan& p, const float* d_vis4, int first_image, int n_images, float* d_grid,
                                int* d_status, cudaStream_t st);
blink_status launch_grid_atomic(const Plan& p, const float2* d_visI, int image, float2* d_grid_full,
                                cudaStream_t st);
blink_status launch_colpass_gather(const Plan& p, int prec, const float2* d_visI, int64_t vis_stride,
                                   int first_image, int n_images, void* d_H, int ldh, int* d_status,
                                   cudaStream_t st);
blink_status launch_colpass_grid(int N, int prec, const float2* d_tw, const float2* d_grid, int n_images,
                                 void* d_H, int ldh, cudaStream_t st);
blink_status launch_rowpass(int N, int prec, const float2* d_tw, const void* d_H, int ldh, int has_nyq,
                            const float* d_w, int w_offset, int w_mod, int n_images, float* d_img,
                            cudaStream_t st);

// output kinds of the correlators
enum { CORR_OUT_VIS4 = 0, CORR_OUT_STOKES_I = 1, CORR_OUT_XX = 2 };

constexpr int COL_CW = 16;                 // u columns per column-pass CTA

// ------------------------------------------------------------------------------------------------
// device helpers
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul_i(float2 a) { return make_float2(-a.y, a.x); }     // a * i
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// storage of complex values in shared or global memory: FP32 pairs or BF16 pairs
__device__ __forceinline__ float2 ld_c(const float2* p) { return *p; }
__device__ __forceinline__ float2 ld_c(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
__device__ __forceinline__ void st_c(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void st_c(__nv_bfloat162* p, float2 v) { *p = __float22bfloat162_rn(v); }

// Unnormalised inverse DFT of R points in registers: v[q] <- sum_r v[r] exp(+2 pi i r q / R).
template <int R> __device__ __forceinline__ void idft(float2* v);

template <> __device__ __forceinline__ void idft<1>(float2*) {}

template <> __device__ __forceinline__ void idft<2>(float2* v) {
    float2 a = cadd(v[0], v[1]), b = csub(v[0], v[1]);
    v[0] = a;
    v[1] = b;
}

template <> __device__ __forceinline__ void idft<4>(float2* v) {
    float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    float2 a2 = cadd(v[1], v[3]), a3 = cmul_i(csub(v[1], v[3]));
    v[0] = cadd(a0, a2);
    v[1] = cadd(a1, a3);
    v[2] = csub(a0, a2);
    v[3] = csub(a1, a3);
}

template <> __device__ __forceinline__ void idft<8>(float2* v) {
    // radix-2 split into the 4-point transforms of the even and odd samples
    float2 a0 = cadd(v[0], v[4]), a1 = csub(v[0], v[4]);
    float2 a2 = cadd(v[2], v[6]), a3 = cmul_i(csub(v[2], v[6]));
    float2 b0 = cadd(v[1], v[5]), b1 = csub(v[1], v[5]);
    float2 b2 = cadd(v[3], v[7]), b3 = cmul_i(csub(v[3], v[7]));
    float2 e0 = cadd(a0, a2), e1 = cadd(a1, a3), e2 = csub(a0, a2), e3 = csub(a1, a3);
    float2 o0 = cadd(b0, b2), o1 = cadd(b1, b3), o2 = csub(b0, b2), o3 = csub(b1, b3);
    const float r2 = 0.70710678118654752440f;
    // w^1 o1, w^2 o2 = i o2, w^3 o3 with w = exp(2 pi i / 8)
    float2 t1 = make_float2((o1.x - o1.y) * r2, (o1.x + o1.y) * r2);
    float2 t2 = cmul_i(o2);
    float2 t3 = make_float2((-o3.x - o3.y) * r2, (o3.x - o3.y) * r2);
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, t1);
    v[5] = csub(e1, t1);
    v[2] = cadd(e2, t2);
    v[6] = csub(e2, t2);
    v[3] = cadd(e3, t3);
    v[7] = csub(e3, t3);
}

// One pass of a batched, in-place Stockham autosort inverse FFT in shared memory.
// BATCH transforms of N points; point p of transform `lane` lives at s[p * PS + lane * LS].
// NS is the product of the radices of the earlier passes.  tw[k * TWS] = exp(+2 pi i k / N).
// Every butterfly reads its R inputs into registers, the block synchronises, then all write.
template <int N, int R, int NS, int BATCH, int NTHR, int PS, int LS, int TWS, typename T>
__device__ __forceinline__ void fft_pass(T* s, const float2* __restrict__ tw, int tid) {
    constexpr int NB = N / R;
    constexpr int TOT = NB * BATCH;
    constexpr int PER = (TOT + NTHR - 1) / NTHR;
    float2 v[PER][R];
#pragma unroll
    for (int m = 0; m < PER; m++) {
        const int bf = tid + m * NTHR;
        if (TOT % NTHR == 0 || bf < TOT) {
            const int lane = bf % BATCH, j = bf / BATCH;
#pragma unroll
            for (int r = 0; r < R; r++) v[m][r] = ld_c(s + (j + r * NB) * PS + lane * LS);
            if (NS > 1) {
                const int k = j % NS;
#pragma unroll
                for (int r = 1; r < R; r++) v[m][r] = cmul(v[m][r], __ldg(tw + (k * r * (N / (NS * R))) * TWS));
            }
            idft<R>(v[m]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < PER; m++) {
        const int bf = tid + m * NTHR;
        if (TOT % NTHR == 0 || bf < TOT) {
            const int lane = bf % BATCH, j = bf / BATCH;
            const int d = (j / NS) * NS * R + (j % NS);
#pragma unroll
            for (int r = 0; r < R; r++) st_c(s + (d + r * NS) * PS + lane * LS, v[m][r]);
        }
    }
    __syncthreads();
}

// The full transform: radix-8 passes, then one pass of the remaining factor (2 or 4).
template <int N, int NS, int BATCH, int NTHR, int PS, int LS, int TWS, typename T>
__device__ __forceinline__ void fft_run(T* s, const float2* __restrict__ tw, int tid) {
    if constexpr (NS < N) {
        constexpr int REM = N / NS;
        constexpr int R = (REM % 8 == 0) ? 8 : REM;
        fft_pass<N, R, NS, BATCH, NTHR, PS, LS, TWS, T>(s, tw, tid);
        fft_run<N, NS * R, BATCH, NTHR, PS, LS, TWS, T>(s, tw, tid);
    }
}

__device__ __forceinline__ void dev_fail(int* status, int code) {
    if (status) atomicOr(status, code);
}

}  // namespace blink
