// Internal declarations of the GB300 dirty-imaging library (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <type_traits>
#include <utility>
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
constexpr int kSepMaxW = 8;                  // widest kernel with a separable gather list (row weights per record)

// ------------------------------------------------------------------------------------------------
// plan: everything that depends only on (array, channels, imaging), built once and cached
// ------------------------------------------------------------------------------------------------
// Launch shape of the persistent FFT kernel, chosen by the autotuner on a plan's first batched call.
struct FftTune {
    int ring = 24, lag = 16;   // ring of column-pass results and row-task lag (images)
    int ctas_per_sm = 0;       // resident CTAs per SM (0 = as many as fit)
};

struct Plan {
    uint64_t key = 0;
    mutable FftTune tune;                  // autotuned FFT launch shape
    mutable bool tuned = false;
    mutable float tune_ms = 0.f;           // time of the chosen shape on the tuning call
    int n_tiles = 0, n_fine = 0, chan_avg = 1, F = 0, N = 0, pol = 0, autos = 1;
    int support = 0;                       // convolution kernel width in cells (0: nearest cell)
    bool phased = false;                   // off-zenith phase centre
    double basis[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};   // e_l, e_m, s0 of the pointing in (E, N, Up)
    int Ni = 0;                            // image side: N, or N / 2 with a kernel (grid side N = 2 Ni)
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
    int* d_ent_off = nullptr;              // [F][N/2 + 1]: first gather entry of each column u
    uint2* d_ent = nullptr;                // [n_contrib] {u | v << 13 | conj << 31, b}, sorted by (u, v, b)
    float* d_wt = nullptr;                 // [n_contrib] kernel weight of each entry (convolution only)
    float* d_corr = nullptr;               // [Ni] grid correction 1 / c(nu) per image pixel index (convolution only)
    // the separable form of a kernel's list (W <= kSepMaxW, the persistent kernel's sides): a record is a cross
    // visibility, its mirror (conjugate, at -g) or an autocorrelation, with its support's rows v0 .. v0 + W - 1
    // (v0 signed, rows taken mod N) and weights C(v - gv); per channel and column u, one entry for each record
    // whose support meets the column, sorted by (v0, record)
    int* d_sep_off = nullptr;              // [F][N/2 + 1] + 1: first entry of each column u
    uint4* d_sep = nullptr;                // {b | conj << 31, v0, C(u - gu) (float bits), record's weight row}
    float* d_sep_w = nullptr;              // [records][kSepMaxW]: row weights C(v0 + k - gv) (-1)^k, 0 past W
    float* d_W = nullptr;                  // [F] W, the sum of weights
    float* d_Wk = nullptr;                 // [F] W times the divisor of the correlator's raw sums (2K or K)
    float2* d_tw = nullptr;                // twiddle set of side N (tws_total(N) entries)
    double* d_uvw = nullptr;               // [F][B][3] (kept for blink_cells)
    float2* d_phase = nullptr;             // [F][B] exp(+2 pi i w) of an off-zenith phase centre, else NULL
    // gather order of the nearest-cell list: entry p of channel f (its local position in the channel's range)
    // takes baseline gsrc[f][p] (a baseline in the column u = 0 feeds two entries, itself and its mirror);
    // NULL when a baseline index does not fit 16 bits.  gphase[f][p]: the phase-centre factor in that order.
    uint16_t* d_gsrc = nullptr;            // [F][e_stride]
    float2* d_gphase = nullptr;            // [F][e_stride] off zenith, else NULL
    uint32_t* d_gpos = nullptr;            // [F][B] the inverse: entry positions p1 | p2 << 16 of baseline b
                                           //   (0xFFFF: none; the second only in the column u = 0)
    int e_stride = 0;                      // floats per plane of one gather-ordered item (>= entries per channel)
};

struct Workspace {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// Bounded dependency waits of the persistent FFT kernel: the clock-cycle budget of each wait (about a
// second by default), and an amount added to the row tasks' dependency target (0; a test sets 1 so that
// those waits cannot be met and run out).
struct FftWait {
    long long budget = 2000000000ll;
    int extra = 0;
};

}  // namespace blink

struct blink_context {
    int device = 0;
    int n_sm = 0;
    int* d_status = nullptr;
    std::vector<blink::Plan*> plans;       // most recent last
    // workspaces: 0 vis, 1 ring, 2 voltages / grid, 3 images, 4 counters, 5 plain form, 6 gains, 7 delays,
    // 8 averaged grids
    blink::Workspace ws[9];
    float2* tw[16] = {};                   // twiddle tables by log2(side)
    std::vector<std::pair<int, float2*>> tw_any;   // unit-root tables of the other sides (fft_mixed.cu)
    blink::FftWait fft_wait;               // dependency-wait budget of the persistent FFT kernel
    bool fused = false;                    // correlation inside the side-512 imaging launch (blink_set_fused)
    // per-stage profiling (blink_set_profiling): recorded (stage, start, stop) event pairs and a free pool
    bool profiling = false;
    struct Rec { int stage; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
};

namespace blink {

blink_status check_imaging(const blink_imaging* im);
blink_status nearest_only(const blink_imaging* im, const char* what);
blink_status get_plan(blink_context* ctx, const blink_array* a, const blink_obs* o, const blink_imaging* im,
                      bool need_gather, cudaStream_t st, Plan** out);
blink_status workspace(blink_context* ctx, int slot, size_t bytes, void** out);
blink_status twiddles(blink_context* ctx, int N, float2** out);
// Raise kernel `fn`'s dynamic shared-memory limit to `bytes` and prefer the largest carve-out, the first
// time a launch needs more than before; remembered per kernel (instances of one template share a type, so
// a cache keyed by type would mix them up).
blink_status kernel_smem(const void* fn, size_t bytes);

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
// Calibration of a correlation launch: complex float [channels][n_tiles][2 pol] gains, or (full) complex
// [channels][n_tiles][2][2] Jones matrices J[p][r], on the device; item channel f uses row f0 + f.
// d == NULL: none.
struct GainRef {
    const float2* d = nullptr;
    int f0 = 0;
    bool full = false;
};
// Where the imaging kinds go: each item's sums, times the phase-centre factor of their baseline and channel
// when `phase` is given, in baseline order (float2 [item][out_item_stride]); or, with `gather` (the FP8
// tensor-core form only, see corr_fp8_gathers), in the gather order of the plan's nearest-cell list, as planes
// [item][re: e_stride | im: e_stride] (floats), the factor taken from the plan's gather-ordered table.
struct ImgOut {
    const float2* phase = nullptr;         // [F][B] or NULL
    bool gather = false;
};

blink_status launch_corr_fp32(int out_kind, const uint8_t* d_volt, int64_t sample_stride_bytes, const Plan& p,
                              int ns, int first_item, int n_items, void* out, int64_t out_item_stride,
                              int* d_status, cudaStream_t st, GainRef gains = {}, ImgOut io = {});
blink_status launch_corr_fp8(int out_kind, const uint8_t* d_volt, int64_t sample_stride_bytes, const Plan& p,
                             int ns, int first_item, int n_items, void* out, int64_t out_item_stride,
                             int* d_status, int n_sm, cudaStream_t st, GainRef gains = {}, ImgOut io = {});
// Whether the FP8 form can write this plan's imaging kind in gather order (no calibration, a gather source
// table, and the item's copy fitting in shared memory beside the operands).
bool corr_fp8_gathers(const Plan& p, int ns, int out_kind, GainRef gains);
// The phase-centre factors of an off-zenith plan in gather order (Plan::d_gphase from d_phase and d_gsrc).
blink_status launch_gather_phase(const Plan& p, cudaStream_t st);
blink_status launch_dedisperse(const float* d_img, int n_out, int F, int n_pix, const int* d_delay, float* d_out,
                               cudaStream_t st);
blink_status launch_dedisperse_stream(const float* d_img, int64_t t0, int n, int F, int n_pix, const int* d_delay,
                                      int D, float* d_carry, float* d_out, int* n_out, cudaStream_t st);
blink_status launch_grid_gather(const Plan& p, const float* d_vis4, int first_image, int n_images, float* d_grid,
                                int* d_status, cudaStream_t st);
blink_status launch_grid_atomic(const Plan& p, const float2* d_visI, int image, float2* d_grid_full,
                                cudaStream_t st);
// A wave of images as a block of (channel, integration) pairs: wave-local image i is the image id
// (tau0 + i % nt) * F + f0 + i / nt.  Contiguous ids are the case F = 1, f0 = 0.
struct WaveMap {
    int F, f0, tau0, nt;
    __host__ __device__ int id(int i) const { return (tau0 + i % nt) * F + f0 + i / nt; }
};

// Gridding + both FFT passes of images [tau0, tau0 + n_tau) x all channels in one persistent launch;
// d_H holds fft_ring_images_max() column-pass results, d_counters 2 + 2 * F * n_tau ints.
int fft_ring_images_max();
// The fused form of the side-512 launch: correlation tasks inside the persistent kernel (FP8 tensor cores,
// Stokes I or XX, no calibration) writing each image's sums into an L2-resident ring of gather-ordered slots.
struct FusedIn {
    const uint8_t* d_volt = nullptr;       // the call's voltage block
    int64_t sample_stride = 0;             // bytes between samples
    int ns = 0;                            // samples per integration
    int kind = 0;                          // CORR_OUT_STOKES_I or CORR_OUT_XX
    float* d_vring = nullptr;              // fused_ring_floats(p) floats
};
// Whether this plan and request can run fused, and the floats its vis ring needs.
bool fft_fused_ok(const Plan& p, int ns, int kind, const uint8_t* d_volt, int64_t sample_stride);
size_t fused_ring_floats(const Plan& p);
// d_vis holds the correlation sums of images [vis_first, ...): float2 [image][vis_stride] in baseline order, or,
// when `gathered`, gather-ordered planes of p.e_stride floats each (vis_stride = p.e_stride float2 per image).
// With `fused` (and gathered) the launch correlates the images itself and d_vis is unused; d_counters then
// holds 2 + 3 * F * n_tau ints.
blink_status launch_fft_persistent(const Plan& p, const FftTune& tune, int prec, const float2* d_vis,
                                   int64_t vis_stride, int vis_first, int tau0, int n_tau, void* d_H, int* d_counters,
                                   float* d_img, int out_first, int* d_status, int n_sm, cudaStream_t st,
                                   const FftWait& wait, bool gathered = false, const FusedIn* fused = nullptr);
// Whether the persistent kernel can read gather-ordered sums for this plan (side 512, nearest cell).
bool fft_takes_gathered(const Plan& p);
// Candidate launch shapes the autotuner times for a plan.
std::vector<FftTune> fft_tune_candidates(const Plan& p);
// Constant-memory twiddles of the persistent kernel for side N on the current device (once per plan).
blink_status fft_constants(int N);

// ---- sides outside the side-specialised kernels (fft_mixed.cu) -------------------------------------
// Power-of-two sides in [64, 2048] run the side-specialised kernels; every other even side whose only
// prime factors are 2, 3 and 5, up to 8192, runs the mixed-radix column and row passes.
inline bool fast_side(int N) { return N >= 64 && N <= 2048 && (N & (N - 1)) == 0; }
bool mixed_side_ok(int N);
// exp(+2 pi i k / N) for k < N (the mixed-radix passes' twiddle table)
blink_status make_unit_roots(float2* d_out, int N, cudaStream_t st);
// complex elements per row of the mixed column-pass result H
size_t mixed_h_row(int N);
struct MixedIn {
    int N = 0;                             // grid side
    const float2* tw = nullptr;            // make_unit_roots(N)
    const float2* grid = nullptr;          // stored half-plane grids [n][N][N/2 + 1] (the Nyquist column included) ...
    const float2* vis = nullptr;           // ... or per-item sums in baseline order, item i at vis + i * vstride,
    int64_t vstride = 0;                   //     gathered through the plan's lists of channel (first + i) % F
    bool gathered = false;                 //     (gathered: in that channel's entry order, planar, e_stride real
    int e_stride = 0;                      //     parts then e_stride imaginary parts; nearest cell only);
    int first = 0, F = 1;                  //     output o (o_first + launch index) sums the fa items
    int o_first = 0, fa = 1;               //     (o / (F/fa)) F + (o % (F/fa)) fa + m, scaled by
    const float* wk = nullptr;             //     1 / (max(wk[f], 1) fa) when wk is given
    const int* ent_off = nullptr;
    const uint2* ent = nullptr;
    const float* wt = nullptr;             // kernel weights per entry, or NULL
    const float* corr = nullptr;           // kernel grid correction [N/2]: keep the central N/2 x N/2, or NULL
};
// pass 0: column pass of n_images grids into d_H (n_images * rows * mixed_h_row(N) elements of the
// storage type, rows = N, or N/2 with a correction); pass 1: row pass of d_H into images, image i written
// at d_img + (wm.id(i) - out_first) * side^2 and divided by d_w[wm.id(i) % w_mod] (d_w NULL: by 1).
blink_status launch_mixed(const MixedIn& in, int pass, int prec, int n_images, void* d_H, const float* d_w, int w_mod,
                          WaveMap wm, int out_first, float* d_img, cudaStream_t st);
// Averaged outputs over many channels: their half-plane grids [n_out][N][N/2 + 1], unshifted, summed into d_grid
// (zeroed by the caller) from in.vis / the plan's lists, for a column pass with in.grid = d_grid.
blink_status launch_avg_grid(const MixedIn& in, int n_out, float2* d_grid, cudaStream_t st);
blink_status launch_colpass_grid(int N, int prec, const float2* d_tw, const float2* d_grid, int n_images,
                                 void* d_H, int ldh, cudaStream_t st);
blink_status launch_rowpass(int N, int prec, const float2* d_tw, const void* d_H, int ldh, int has_nyq,
                            const float* d_w, int w_mod, WaveMap wm, int n_images, int out_first, float* d_img,
                            cudaStream_t st);

// output kinds of the correlators: VIS4 = the ABI visibilities V = S / K; STOKES_I and XX = the raw
// integer sums S_XX + S_YY and S_XX (as floats) that the imaging path grids, divided later with 1/W
enum { CORR_OUT_VIS4 = 0, CORR_OUT_STOKES_I = 1, CORR_OUT_XX = 2 };


constexpr int COL_CW = 8;                  // u columns per column-pass CTA (one warp per column)

// ------------------------------------------------------------------------------------------------
// device helpers
// ------------------------------------------------------------------------------------------------
// Complex sums and differences as one packed two-lane FP32 instruction (add.rn.f32x2 / sub.rn.f32x2 of
// Blackwell): each lane is the same round-to-nearest FP32 addition as the scalar form, so results are
// unchanged while the butterflies issue half as many instructions.
// (Host versions of these and of the register DFTs below exist so that transform plans can be checked on a
// CPU; they compute the same sums with scalar operations.)
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
    return __fadd2_rn(a, b);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(*reinterpret_cast<unsigned long long*>(&a)),
        "l"(*reinterpret_cast<unsigned long long*>(&b)));
    return *reinterpret_cast<float2*>(&r);
#else
    return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul_i(float2 a) { return make_float2(-a.y, a.x); }     // a * i
__host__ __device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// storage of complex values in shared or global memory: FP32 pairs or BF16 pairs
__device__ __forceinline__ float2 ld_c(const float2* p) { return *p; }
__device__ __forceinline__ float2 ld_c(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
__device__ __forceinline__ void st_c(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void st_c(__nv_bfloat162* p, float2 v) { *p = __float22bfloat162_rn(v); }

// Unnormalised inverse DFT of R points in registers: v[q] <- sum_r v[r] exp(+2 pi i r q / R).
template <int R> __host__ __device__ __forceinline__ void idft(float2* v);

template <> __host__ __device__ __forceinline__ void idft<1>(float2*) {}

template <> __host__ __device__ __forceinline__ void idft<2>(float2* v) {
    float2 a = cadd(v[0], v[1]), b = csub(v[0], v[1]);
    v[0] = a;
    v[1] = b;
}

template <> __host__ __device__ __forceinline__ void idft<4>(float2* v) {
    float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    float2 a2 = cadd(v[1], v[3]), a3 = cmul_i(csub(v[1], v[3]));
    v[0] = cadd(a0, a2);
    v[1] = cadd(a1, a3);
    v[2] = csub(a0, a2);
    v[3] = csub(a1, a3);
}

template <> __host__ __device__ __forceinline__ void idft<3>(float2* v) {
    // w = exp(2 pi i / 3) = -1/2 + i sqrt(3)/2: v1 w^q + v2 w^2q = -(v1 + v2)/2 +- i sqrt(3)/2 (v1 - v2)
    const float h = 0.86602540378443864676f;
    const float2 t = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    const float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    const float2 r = make_float2(-h * d.y, h * d.x);                      // i sqrt(3)/2 (v1 - v2)
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
}

template <> __host__ __device__ __forceinline__ void idft<5>(float2* v) {
    // w = exp(2 pi i / 5); with a1 = v1 + v4, b1 = v1 - v4, a2 = v2 + v3, b2 = v2 - v3:
    // X1, X4 = v0 + c1 a1 + c2 a2 +- i (s1 b1 + s2 b2);  X2, X3 = v0 + c2 a1 + c1 a2 +- i (s2 b1 - s1 b2)
    // where c1 = cos(2 pi/5) = (sqrt 5 - 1)/4, c2 = cos(4 pi/5) = -(sqrt 5 + 1)/4, s1 = sin(2 pi/5), s2 = sin(4 pi/5)
    const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
    const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
    const float2 a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]), a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    const float2 p1 = make_float2(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
    const float2 p2 = make_float2(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
    const float2 q1 = cmul_i(make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
    const float2 q2 = cmul_i(make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
    v[0] = cadd(v[0], cadd(a1, a2));
    v[1] = cadd(p1, q1);
    v[4] = csub(p1, q1);
    v[2] = cadd(p2, q2);
    v[3] = csub(p2, q2);
}

template <> __host__ __device__ __forceinline__ void idft<8>(float2* v) {
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

template <> __host__ __device__ __forceinline__ void idft<16>(float2* v) {
    // 4 x 4: 4-point transforms over r1 of v[4 r1 + r2], twiddles exp(2 pi i r2 q1 / 16), then 4-point
    // transforms over r2, giving v[q1 + 4 q2]
    const float c = 0.92387953251128675613f, s = 0.38268343236508977173f, h = 0.70710678118654752440f;
    float2 a[4][4];
#pragma unroll
    for (int r2 = 0; r2 < 4; r2++) {
        a[r2][0] = v[r2];
        a[r2][1] = v[4 + r2];
        a[r2][2] = v[8 + r2];
        a[r2][3] = v[12 + r2];
        idft<4>(a[r2]);
    }
    auto rot = [](float2 x, float cr, float ci) { return make_float2(x.x * cr - x.y * ci, x.x * ci + x.y * cr); };
    a[1][1] = rot(a[1][1], c, s);                                               // w^1
    a[1][2] = make_float2((a[1][2].x - a[1][2].y) * h, (a[1][2].x + a[1][2].y) * h);   // w^2
    a[1][3] = rot(a[1][3], s, c);                                               // w^3
    a[2][1] = make_float2((a[2][1].x - a[2][1].y) * h, (a[2][1].x + a[2][1].y) * h);   // w^2
    a[2][2] = cmul_i(a[2][2]);                                                  // w^4
    a[2][3] = make_float2((-a[2][3].x - a[2][3].y) * h, (a[2][3].x - a[2][3].y) * h);  // w^6
    a[3][1] = rot(a[3][1], s, c);                                               // w^3
    a[3][2] = make_float2((-a[3][2].x - a[3][2].y) * h, (a[3][2].x - a[3][2].y) * h);  // w^6
    a[3][3] = rot(a[3][3], -c, -s);                                             // w^9
#pragma unroll
    for (int q1 = 0; q1 < 4; q1++) {
        float2 t[4] = {a[0][q1], a[1][q1], a[2][q1], a[3][q1]};
        idft<4>(t);
        v[q1] = t[0];
        v[q1 + 4] = t[1];
        v[q1 + 8] = t[2];
        v[q1 + 12] = t[3];
    }
}

// 15 points in the prime-factor form (15 = 3 x 5, coprime factors, so no twiddles): input x[(5 n1 + 3 n2) mod 15]
// goes through 3-point transforms over n1 for every n2, then 5-point transforms over n2 for every k1, and the
// output of (k1, k2) is X[(10 k1 + 6 k2) mod 15] (10 = 1 mod 3, 0 mod 5; 6 = 0 mod 3, 1 mod 5).
template <> __host__ __device__ __forceinline__ void idft<15>(float2* v) {
    float2 a[5][3];
#pragma unroll
    for (int n2 = 0; n2 < 5; n2++) {
#pragma unroll
        for (int n1 = 0; n1 < 3; n1++) a[n2][n1] = v[(5 * n1 + 3 * n2) % 15];
        idft<3>(a[n2]);
    }
#pragma unroll
    for (int k1 = 0; k1 < 3; k1++) {
        float2 b[5];
#pragma unroll
        for (int n2 = 0; n2 < 5; n2++) b[n2] = a[n2][k1];
        idft<5>(b);
#pragma unroll
        for (int k2 = 0; k2 < 5; k2++) v[(10 * k1 + 6 * k2) % 15] = b[k2];
    }
}

// One pass of a batched, in-place Stockham autosort inverse FFT in shared memory.
// BATCH transforms of N points; point p of transform `lane` lives at s[p * PS + lane * LS].
// NS is the product of the radices of the earlier passes; tw is the transform's per-pass twiddle table.
// Every butterfly reads its R inputs into registers, the block synchronises, then all write: to shared
// memory, or - for the last pass - through `out(lane, position, value)` (OUT = true).
// LM selects the thread mapping: lane-major (consecutive threads take consecutive transforms, for
// column layouts with LS = 1) or position-major (consecutive threads take consecutive butterflies of one
// transform, for row layouts with PS = 1).
// ---- twiddle tables ---------------------------------------------------------------------------------
// Radix of the pass of an N-point transform that follows passes whose radices multiply to NS: radix 8
// while at least 8 points remain, then the remaining factor (2 or 4).
__host__ __device__ constexpr int radix_at(int N, int NS) { return ((N / NS) % 8 == 0) ? 8 : N / NS; }
// Offset of the pass starting at NS in the per-pass table of an N-point transform: the pass's twiddles
// exp(+2 pi i k r / (NS R)) sit at [(r - 1) * NS + k] for r in [1, R) and k in [0, NS), so that threads
// with consecutive k read consecutive entries.
__host__ __device__ constexpr int tw_off(int N, int NS) {
    int off = 0;
    for (int ns = 1; ns < NS; ns *= radix_at(N, ns)) off += (radix_at(N, ns) - 1) * ns;
    return off;
}
__host__ __device__ constexpr int tw_size(int N) { return tw_off(N, N); }
// Twiddle set of an image side N, in one array: [0, N/2] exp(+2 pi i k / N) (complex-to-real pre-twiddle),
// then the per-pass table of the N-point column transform, then that of the N/2-point row transform.
__host__ __device__ constexpr int tws_pre(int) { return 0; }
__host__ __device__ constexpr int tws_col(int N) { return (N / 2 + 1 + 7) / 8 * 8; }
__host__ __device__ constexpr int tws_row(int N) { return tws_col(N) + (tw_size(N) + 7) / 8 * 8; }
__host__ __device__ constexpr int tws_total(int N) { return tws_row(N) + (tw_size(N / 2) + 7) / 8 * 8; }
// Fill the twiddle set of side N (one kernel launch, FP64 sincospi rounded to FP32).
blink_status make_twiddles(float2* d_out, int N, cudaStream_t st);

// Padded position of point p in a transform stored with one spare slot after every 16 points: it keeps the
// stride-R writes of the Stockham passes of a single transform free of shared-memory bank conflicts.
__device__ __forceinline__ int padx(int p) { return p + (p >> 4); }

template <int N, int R, int NS, int BATCH, int NTHR, int PS, int LS, bool LM, bool OUT, bool WARP, typename T,
          typename Out, bool PAD = false>
__device__ __forceinline__ void fft_pass(T* s, const float2* tw, int tid, Out& out) {
    constexpr int NB = N / R;
    constexpr int TOT = NB * BATCH;
    constexpr int PER = (TOT + NTHR - 1) / NTHR;
    float2 v[PER][R];
#pragma unroll
    for (int m = 0; m < PER; m++) {
        const int bf = tid + m * NTHR;
        if (TOT % NTHR == 0 || bf < TOT) {
            const int lane = LM ? bf % BATCH : bf / NB, j = LM ? bf / BATCH : bf % NB;
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int q = j + r * NB;
                v[m][r] = ld_c(s + (PAD ? padx(q) : q) * PS + lane * LS);
            }
            if (NS > 1) {
                const int k = j % NS;
#pragma unroll
                for (int r = 1; r < R; r++) v[m][r] = cmul(v[m][r], tw[tw_off(N, NS) + (r - 1) * NS + k]);
            }
            idft<R>(v[m]);
        }
    }
    if (!OUT) {
        if (WARP) __syncwarp(); else __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < PER; m++) {
        const int bf = tid + m * NTHR;
        if (TOT % NTHR == 0 || bf < TOT) {
            const int lane = LM ? bf % BATCH : bf / NB, j = LM ? bf / BATCH : bf % NB;
            const int d = (j / NS) * NS * R + (j % NS);
#pragma unroll
            for (int r = 0; r < R; r++) {
                if (OUT)
                    out(lane, d + r * NS, v[m][r]);
                else
                    st_c(s + (PAD ? padx(d + r * NS) : d + r * NS) * PS + lane * LS, v[m][r]);
            }
        }
    }
    if (!OUT) {
        if (WARP) __syncwarp(); else __syncthreads();
    }
}

// The full transform: radix-8 passes, then one pass of the remaining factor (2 or 4).  With OUT = true
// the last pass hands its results to `out` instead of writing shared memory.  WARP = true: the threads
// of one warp (tid = lane, NTHR = 32) own the transforms and synchronise with __syncwarp only.
template <int N, int NS, int BATCH, int NTHR, int PS, int LS, bool LM, bool OUT, bool WARP, typename T, typename Out,
          bool PAD = false>
__device__ __forceinline__ void fft_run(T* s, const float2* tw, int tid, Out& out) {
    if constexpr (NS < N) {
        constexpr int R = radix_at(N, NS);
        constexpr bool LAST = NS * R == N;
        fft_pass<N, R, NS, BATCH, NTHR, PS, LS, LM, OUT && LAST, WARP, T, Out, PAD>(s, tw, tid, out);
        fft_run<N, NS * R, BATCH, NTHR, PS, LS, LM, OUT, WARP, T, Out, PAD>(s, tw, tid, out);
    }
}

struct NoOut {
    __device__ void operator()(int, int, float2) const {}
};

// ---- one transform per warp, padded positions, with the index arithmetic hoisted -----------------------
// Layout of a pass's buffer: point p at padq<C>(p) = p + C * (p / 16), i.e. C spare slots after every 16
// points (C = 1 is padx).  Every pass reads aligned runs of 16 consecutive points per half-warp, which are
// conflict-free under any C; the writes of the pass after the first radix-8 pass (stride 8 within groups of
// 64) are conflict-free only with C = 2, the others with C = 1, so that pass writes with C = 2 and the next
// reads with it.  Transforms start and end in the C = 1 layout.
// A position p = A(lane) + K, where K is a compile-time multiple of 16 or stays inside A's run of 16, has
// padq<C>(p) = padq<C>(A) + K + C * (K / 16): each lane computes its base once per pass and every element
// address is that plus a constant.  Sides whose radix-8 passes would not fit these decompositions (fewer
// than 32 butterflies per pass) fall back to the generic fft_pass.
template <int C> __device__ __forceinline__ int padq(int p) { return p + C * (p >> 4); }
// Slots a warp transform of n points needs (room for the C = 2 layout when the hoisted form is used).
__host__ __device__ constexpr int wfft_slots(int n) { return n >= 256 ? n + n / 8 : n + n / 16; }

// MASKED (first pass only): point p = lane + 32 t holds data only if bit t of `occ` is set, else it reads as
// zero without a shared-memory access.
template <int N, int R, int NS, int PR, int PW, bool OUT, bool MASKED, typename T, typename Out>
__device__ __forceinline__ void wfft_pass(T* s, const float2* tw, int lane, Out& out, uint32_t occ) {
    constexpr int NB = N / R;
    constexpr int PER = NB / 32;                    // butterflies per lane
    static_assert(NB % 32 == 0, "warp transform needs at least 32 butterflies per pass");
    static_assert(NS == 1 || NS == 8 || NS % 32 == 0, "unsupported pass layout");
    static_assert(!MASKED || (NS == 1 && N <= 1024), "the occupancy mask covers the first pass of up to 1024 points");
    float2 v[PER][R];
    const int rbase = padq<PR>(lane);               // reads: j + r * NB, j = lane + 32 m, NB % 32 == 0
#pragma unroll
    for (int m = 0; m < PER; m++) {
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int t = (32 * m + r * NB) / 32;   // the point's index over the lanes
            if (!MASKED || ((occ >> t) & 1u))
                v[m][r] = ld_c(s + rbase + (32 * m + r * NB) * (16 + PR) / 16);
            else
                v[m][r] = make_float2(0.f, 0.f);
        }
        if (NS > 1) {
            // k = j % NS
            const int k = (NS % 32 == 0) ? (lane + (32 * m) % NS) : (lane & (NS - 1));
#pragma unroll
            for (int r = 1; r < R; r++) v[m][r] = cmul(v[m][r], tw[tw_off(N, NS) + (r - 1) * NS + k]);
        }
        idft<R>(v[m]);
    }
    if (!OUT) __syncwarp();
    // writes: d + r * NS with d = (j / NS) * NS * R + j % NS
    int wbase;
    if (NS == 1) {
        wbase = R * lane + PW * ((R * lane) >> 4);  // d = R j = R lane + 32 m R
    } else if (NS == 8) {
        wbase = (64 + 4 * PW) * (lane >> 3) + (lane & 7);   // d = 64 (lane >> 3) + (lane & 7) + 256 m
    } else {
        wbase = padq<PW>(lane);                     // d = lane + const (NS % 32 == 0)
    }
#pragma unroll
    for (int m = 0; m < PER; m++) {
        const int j0 = 32 * m;                      // the lane-independent part of j
#pragma unroll
        for (int r = 0; r < R; r++) {
            if (OUT) {
                const int j = lane + j0;
                out(0, (j / NS) * NS * R + (j % NS) + r * NS, v[m][r]);
            } else {
                int c;
                if (NS == 1) c = 32 * m * R + r;
                else if (NS == 8) c = 256 * m + 8 * r;
                else c = (j0 / NS) * NS * R + (j0 % NS) + r * NS;
                st_c(s + wbase + c + PW * (c / 16), v[m][r]);
            }
        }
    }
    if (!OUT) __syncwarp();
}

// Whole transform by one warp on a padded array; OUT: the last pass hands results to `out`.  PR is the
// layout the pass reads (C = 1 for the first); MASKED: the first pass reads only the points `occ` marks.
template <int N, int NS, int PR, bool OUT, bool MASKED, typename T, typename Out>
__device__ __forceinline__ void wfft_run(T* s, const float2* tw, int lane, Out& out, uint32_t occ) {
    if constexpr (NS < N) {
        constexpr int R = radix_at(N, NS);
        constexpr bool LAST = NS * R == N;
        constexpr int PW = (NS == 8 && !LAST) ? 2 : 1;
        wfft_pass<N, R, NS, PR, PW, OUT && LAST, MASKED && NS == 1, T, Out>(s, tw, lane, out, occ);
        wfft_run<N, NS * R, PW, OUT, false, T, Out>(s, tw, lane, out, occ);
    }
}

// Warp transform of a padded array (padx layout in and out, wfft_slots(N) slots): the hoisted form when
// every pass has at least 32 butterflies (sides of 256 and more), the generic one otherwise.
template <int N, bool OUT, typename T, typename Out>
__device__ __forceinline__ void warp_fft(T* s, const float2* tw, int lane, Out& out) {
    if constexpr (N >= 256)
        wfft_run<N, 1, 1, OUT, false, T, Out>(s, tw, lane, out, 0u);
    else
        fft_run<N, 1, 1, 32, 1, 0, OUT ? false : true, OUT, true, T, Out, true>(s, tw, lane, out);
}

// The same on a column whose points p = lane + 32 t are valid only where bit t of this lane's `occ` is set
// (the rest of the array may hold stale data).  Sides below 256 take the generic form, which needs the
// array zeroed, so callers only use this for N >= 256.
template <int N, typename T>
__device__ __forceinline__ void warp_fft_masked(T* s, const float2* tw, int lane, uint32_t occ) {
    static_assert(N >= 256, "masked warp transform needs the hoisted form");
    NoOut none;
    wfft_run<N, 1, 1, false, true, T, NoOut>(s, tw, lane, none, occ);
}

__device__ __forceinline__ void dev_fail(int* status, int code) {
    if (status) atomicOr(status, code);
}

// Column tile of a column-pass CTA: column c at s[c * col_ld(N)], point v at padx(v); the extra 2 slots
// keep the row-wise store phase free of bank conflicts.
template <int N> __host__ __device__ constexpr int col_ld() { return N + N / 16 + 2; }

// Gather entries: x = u | v << 13 | conj << 31 (cell (u, v) of the half plane, u <= 4096), y = baseline.
__device__ __forceinline__ int ent_u(uint32_t x) { return (int)(x & 0x1FFFu); }
__device__ __forceinline__ int ent_v(uint32_t x) { return (int)((x >> 13) & 0x3FFFFu); }
__device__ __forceinline__ uint32_t ent_cell(uint32_t x) { return x & 0x7FFFFFFFu; }

// Gather entry i of a column whose entries end at `end`: its cell key and visibility (conjugated for an
// entry of the mirrored half plane), times the entry's weight wt[i] when `wt` is given (a convolution
// kernel's weight); key 0xFFFFFFFF and zero past the end.  The visibility is val(b) of the entry's baseline
// b, or val(i, b) where the caller's sums are in gather order (then its load does not wait for the entry's).
template <typename Val>
__device__ __forceinline__ void gather_entry(const uint2* __restrict__ ent, const float* __restrict__ wt, int i,
                                             int end, Val val, uint32_t& key, float2& x) {
    key = 0xFFFFFFFFu;
    x = make_float2(0.f, 0.f);
    if (i < end) {
        const uint2 e = ent[i];
        key = ent_cell(e.x);
        if constexpr (std::is_invocable_v<Val, int, uint32_t>)
            x = val(i, e.y);
        else
            x = val(e.y);
        if (e.x >> 31) x.y = -x.y;
        if (wt) {
            const float w = wt[i];
            x = make_float2(x.x * w, x.y * w);
        }
    }
}

// Grid one column with one warp: sum its gather entries [beg, end) (sorted by v, then baseline) into the
// column's cells s[idx(u, v)], which the caller has zeroed.  The warp takes the entries 32 at a time, one per
// lane, and sums runs of equal cells with a segmented scan over the lanes (keys are sorted, so lanes with
// equal keys are contiguous); the last lane of each run adds the run's sum to its cell.  A cell with many
// contributions (the autocorrelations at (0, 0)) therefore costs a few chunks, not a serial chain, and
// the order of additions is fixed, so results are reproducible.  `val(b)` is baseline b's visibility;
// with `shift` every cell is multiplied by (-1)^(u+v) (the image shift by N/2).
// (key, x) is lane's entry of the first chunk (gather_entry(ent, wt, beg + lane, ...)), loaded by the caller so
// that its latency overlaps the caller's own work; each later chunk is loaded while the previous is summed.
template <typename T, typename Val, typename Idx>
__device__ __forceinline__ void warp_gather_column(const uint2* __restrict__ ent, const float* __restrict__ wt, int beg,
                                                   int end, int lane, T* s, Val val, Idx idx, bool shift, uint32_t key,
                                                   float2 x) {
    for (int base = beg; base < end; base += 32) {
        const int i = base + lane;
        uint32_t nkey;
        float2 nx;
        gather_entry(ent, wt, i + 32, end, val, nkey, nx);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t k2 = __shfl_up_sync(0xFFFFFFFFu, key, d);
            const float xr = __shfl_up_sync(0xFFFFFFFFu, x.x, d), xi = __shfl_up_sync(0xFFFFFFFFu, x.y, d);
            if (lane >= d && k2 == key) {
                x.x += xr;
                x.y += xi;
            }
        }
        const uint32_t knext = __shfl_down_sync(0xFFFFFFFFu, key, 1);
        if (i < end && (lane == 31 || i + 1 >= end || knext != key)) {
            const int u = ent_u(key), v = ent_v(key);
            if (shift && ((u + v) & 1)) x = make_float2(-x.x, -x.y);
            T* p = s + idx(u, v);
            st_c(p, cadd(ld_c(p), x));
        }
        __syncwarp();
        key = nkey;
        x = nx;
    }
}

// The same for a column array that is not zeroed (shift always applied): each cell's first contribution is
// stored rather than added, and bit v / 32 of occ[v % 32] records that cell v holds data (occ zeroed by the
// caller).  Only the first run of a chunk can continue a cell of the previous chunk, which it then adds to.
template <typename T, typename Val, typename Idx>
__device__ __forceinline__ void warp_gather_column_occ(const uint2* __restrict__ ent, const float* __restrict__ wt,
                                                       int beg, int end, int lane, T* s, Val val, Idx idx,
                                                       uint32_t key, float2 x, uint32_t* occ) {
    uint32_t prev = 0xFFFFFFFFu;                    // the last cell of the previous chunk
    for (int base = beg; base < end; base += 32) {
        const int i = base + lane;
        uint32_t nkey;
        float2 nx;
        gather_entry(ent, wt, i + 32, end, val, nkey, nx);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t k2 = __shfl_up_sync(0xFFFFFFFFu, key, d);
            const float xr = __shfl_up_sync(0xFFFFFFFFu, x.x, d), xi = __shfl_up_sync(0xFFFFFFFFu, x.y, d);
            if (lane >= d && k2 == key) {
                x.x += xr;
                x.y += xi;
            }
        }
        const uint32_t knext = __shfl_down_sync(0xFFFFFFFFu, key, 1);
        const uint32_t klast = __shfl_sync(0xFFFFFFFFu, key, min(31, end - 1 - base));
        if (i < end && (lane == 31 || i + 1 >= end || knext != key)) {
            const int u = ent_u(key), v = ent_v(key);
            if ((u + v) & 1) x = make_float2(-x.x, -x.y);
            T* p = s + idx(u, v);
            if (key == prev) x = cadd(ld_c(p), x);
            st_c(p, x);
            atomicOr(occ + (v & 31), 1u << (v >> 5));
        }
        prev = klast;
        __syncwarp();
        key = nkey;
        x = nx;
    }
}

// The same over the entries [beg, end) of several consecutive columns (the keys carry u, so runs never span
// two columns), with the entries and their visibilities loaded NB chunks of 32 at a time.  val(i, b) is the
// value of entry i, whose baseline is b: with sums in baseline order it depends on the entry's load (two
// dependent round trips per NB chunks), with gather-ordered sums only on i (one).  occ(u, v) is the
// occupancy word of cell (u, v) (bit v / 32 of the word of v % 32 in its column).  Every run's sum is
// multiplied by `scale` before it is stored (or added to the cell's earlier part).  hook() runs once, while the
// first batch's loads are in flight.  With `wt` every entry's value is first multiplied by its weight wt[i] (a
// convolution kernel's), loaded with the entry.
template <int NB, typename T, typename Val, typename Idx, typename Occ, typename Hook>
__device__ __forceinline__ void warp_gather_occ_batched(const uint2* __restrict__ ent, int beg, int end, int lane, T* s,
                                                        Val val, Idx idx, Occ occ, float scale, Hook hook,
                                                        const float* __restrict__ wt = nullptr) {
    uint32_t prev = 0xFFFFFFFFu;                    // the last cell of the previous chunk
    for (int base = beg; base < end; base += 32 * NB) {
        uint32_t key[NB], bl[NB];
        float2 x[NB];
        float w[NB];
#pragma unroll
        for (int q = 0; q < NB; q++) {
            const int i = base + 32 * q + lane;
            key[q] = 0xFFFFFFFFu;
            bl[q] = 0u;
            w[q] = 1.0f;
            if (i < end) {
                const uint2 e = ent[i];
                key[q] = e.x;
                bl[q] = e.y;
                if (wt) w[q] = wt[i];
            }
        }
        // the values' loads are guarded by the entry index alone, so that with gather-ordered sums (val
        // independent of the baseline) they are in flight together with the entries' loads
#pragma unroll
        for (int q = 0; q < NB; q++) {
            const int i = base + 32 * q + lane;
            x[q] = i < end ? val(i, bl[q]) : make_float2(0.f, 0.f);
        }
        if (base == beg) hook();                    // the first batch's loads are in flight
#pragma unroll
        for (int q = 0; q < NB; q++) {
            if (key[q] != 0xFFFFFFFFu) {
                if (key[q] >> 31) x[q].y = -x[q].y;
                if (wt) x[q] = make_float2(x[q].x * w[q], x[q].y * w[q]);
                key[q] = ent_cell(key[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < NB; q++) {
            const int cb = base + 32 * q;
            if (cb >= end) break;
            const int i = cb + lane;
            uint32_t k = key[q];
            float2 y = x[q];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t k2 = __shfl_up_sync(0xFFFFFFFFu, k, d);
                const float yr = __shfl_up_sync(0xFFFFFFFFu, y.x, d), yi = __shfl_up_sync(0xFFFFFFFFu, y.y, d);
                if (lane >= d && k2 == k) {
                    y.x += yr;
                    y.y += yi;
                }
            }
            const uint32_t knext = __shfl_down_sync(0xFFFFFFFFu, k, 1);
            const uint32_t klast = __shfl_sync(0xFFFFFFFFu, k, min(31, end - 1 - cb));
            if (i < end && (lane == 31 || i + 1 >= end || knext != k)) {
                const int u = ent_u(k), v = ent_v(k);
                const float sc = ((u + v) & 1) ? -scale : scale;
                y = __fmul2_rn(y, make_float2(sc, sc));
                T* p = s + idx(u, v);
                if (k == prev) y = cadd(ld_c(p), y);
                st_c(p, y);
                atomicOr(occ(u, v), 1u << (v >> 5));
            }
            prev = klast;
            __syncwarp();
        }
    }
}

// The same, loading the first chunk itself.
template <typename T, typename Val, typename Idx>
__device__ __forceinline__ void warp_gather_column(const uint2* __restrict__ ent, const float* __restrict__ wt, int beg,
                                                   int end, int lane, T* s, Val val, Idx idx, bool shift) {
    uint32_t key;
    float2 x;
    gather_entry(ent, wt, beg + lane, end, val, key, x);
    warp_gather_column(ent, wt, beg, end, lane, s, val, idx, shift, key, x);
}

}  // namespace blink
