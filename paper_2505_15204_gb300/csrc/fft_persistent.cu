// Gridding and the batched 2D inverse FFT of a whole correlated chunk in one persistent launch.
//
// The work is two kinds of task per image (Sec. 5.2.4, Eq. 4):
//   column task (image k, column block cb): gather-grid the block's 8 u-columns in shared memory and
//       transform each along v (one warp per column; a side of 512 in a radix-16 and a radix-32 pass, other
//       sides in radix-8 passes), then write the block to the image's slot of a small ring of intermediates
//       (kept in L2);
//   row task (image k, row block rb): once all column tasks of image k are done, transform 32 rows
//       along u (complex to real) and scale by 1 / (W * 2K) (side 512 with nearest-cell gridding scales the
//       gridded cells instead), writing the image rows with streaming stores (they are not read back, so
//       they should not displace the ring from L2).
// Side 512 (nearest cell) keeps the ring column-major, [u][v] with v contiguous: each column warp stores its
// transformed column straight from registers as whole 128-byte lines, and a row task reads 32 consecutive
// rows v of one column u per warp instruction, so that lane l holds row y0 + l.  Its first radix-16 pass
// (the 256-point row transform is 16 x 16) then runs in registers with the rows across the lanes: warp w
// takes the butterflies j and 16 - j (0 and 8 for warp 0), whose points u = j + 16 r and 256 - u are exactly
// the pairs the complex-to-real pre-twiddle combines, and every twiddle it needs is the same for the whole
// warp (read from constant memory).  One exchange through shared memory hands the 16 x 16 intermediate of
// each row to the second pass, two rows per warp, whose outputs are consecutive pixels of one row.  Other
// sides (and gridding with a kernel) keep the row-major ring: a column task transposes its block through
// shared memory into ring rows, and a row task transforms whole rows in shared memory.
// CTAs take task tickets in order from a global counter.  The ticket stream is cut into segments of
// (column tasks of image s) + (row tasks of image s - lag), so an image's row tasks come `lag` segments
// after its column tasks.  Dependencies are per-image counters: a row task waits for the image's column
// tasks, and a column task that reuses a ring slot waits for the previous occupant's row tasks.  A task
// only ever waits on tasks with smaller tickets, which resident CTAs already hold, so the waits always
// end; they are nevertheless bounded, and on expiry the launch records BLINK_ERR_TIMEOUT and every CTA
// stops taking tickets.
#include <algorithm>
#include <type_traits>
#include <cmath>

#include "blink_internal.cuh"
#include "tc_ptx.cuh"

namespace blink {

namespace {

constexpr int kW = 8;                            // warps per CTA: columns per column task, rows per row task
constexpr int kPT = 32 * kW;                     // threads
constexpr int kCW = kW;                          // u columns per column task (one per warp)
constexpr int kRPW = 2;                          // rows per warp in a row batch
constexpr int kRB = kW * kRPW;                   // rows per row batch
constexpr int kRowBatches = 2;                   // row batches per row task
constexpr int kVisAhead = 8;                     // images ahead whose visibilities a column task prefetches
constexpr int kRowLd = 257;                      // side 512: float2 pitch of a row's 16 x 16 intermediate (odd:
                                                 //   lanes = rows write it without bank conflicts)

// The twiddles of the side-512 row tasks, per warp w (which always takes the butterflies jA, jB of the first
// pass): [0, 9) the pre-twiddles exp(2 pi i u / 512) of its A points, [9, 17) those of its B points, [17, 32)
// and [32, 47) the first pass's exp(2 pi i 2 j k1 / 512), k1 = 1 .. 15, for j = jA and jB.  A warp reads its
// row at a warp-uniform base with constant offsets, so no index arithmetic is spent on them.
constexpr int kRowTw = 48;
__constant__ float2 c_rowtw512[kW * kRowTw];

struct FftParams {
    const float2* vis;       // correlation sums of the chunk's images, [item][B]
    int64_t vis_stride;
    int vis_first;           // image id of vis row 0
    uint32_t vis_prefetch;   // bytes of one image's visibilities when they can be prefetched (16-byte multiple), else 0
    int F, tau0, n_tau;      // images: channel-major order k -> (f = k / n_tau, tau = tau0 + k % n_tau)
    int n_img;
    int n_cb, n_rb;          // column tasks and row tasks per image
    const int* ent_off;      // [F][N/2 + 1]
    const uint2* ent;        // gather entries
    const float* wt;         // per-entry kernel weights (convolutional gridding), else NULL
    const int* sep_off;      // the separable form of a kernel's list (FP32 storage), else NULL: [F][N/2 + 1] + 1
    const uint4* sep;        //   {b | conj << 31, v0, C(u - gu) bits, weight row}
    const float* sep_w;      //   [records][kSepMaxW] row weights C(v0 + k - gv) (-1)^k
    int sep_W;               //   kernel width (rows per record)
    const float* corr;       // [N / 2] grid correction per image pixel index (convolutional gridding), else NULL
    const float2* tw;        // twiddle set of side N
    void* H;                 // ring of column-pass results, [ring][N][ldh]
    int ldh, ring, lag;
    const float* wk;         // [F] W * 2K (or W * K)
    float* img_out;
    int out_first;           // image id of img_out's first image
    int* tickets;            // counters, zeroed before the launch: [0] ticket, [1] abort,
    int* col_done;           //   [n_img] column tasks finished per image
    int* row_done;           //   [n_img] row tasks finished per image
    int* status;
    int gathered;            // vis holds gather-ordered planes of e_stride floats (re, then im) per image
    int e_stride;
    long long wait_budget;   // clock cycles a dependency wait may take before the launch gives up
    int extra_wait;          // added to the row tasks' dependency target (0; 1 makes those waits run out)
    // fused form (side 512, gather order): a correlation task per image computes its sums into a small ring
    // of gather-ordered slots that stays in L2, instead of an earlier correlator launch writing them to memory
    int fused;
    const uint8_t* volt;     // the call's voltage block (sample 0, first channel of the call)
    int64_t sample_stride;   // bytes between consecutive samples
    int ns, cavg, n_tiles;   // samples per integration, fine channels averaged, tiles
    int ns_c, n_chunks;      // K streams through the operand tiles in chunks of ns_c samples
    int Kq, Kp, n_blk;       // a chunk's K (multiple of 4), operand row bytes, blocks of 64 tiles
    int stokes;              // Stokes I (X and Y halves of K side by side), else XX
    const uint32_t* gpos;    // [F][B]: entry positions p1 | p2 << 16 of each baseline in its channel's list
    int64_t B;
    const uint8_t* flags;    // [n_tiles]
    float* vring;            // [ring_v][2][e_stride]: the gather-ordered sums of the images in flight
    int ring_v, lead;        // its slots; segments by which an image's correlation precedes its column tasks
    int* corr_done;          // [n_img]
};

constexpr int kCorrCols = 128;                   // TMEM columns per CTA in the fused form: two block pairs

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Asynchronous copy of [p, p + bytes) from memory into L2 (a hint: nothing waits for it).  p and bytes are
// multiples of 16.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Bulk copy of `bytes` (a multiple of 16) from global to shared memory, completing on mbarrier `bar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

__device__ __forceinline__ float2 ldcg_c(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ldcg_c(const __nv_bfloat162* p) {
    const unsigned u = __ldcg(reinterpret_cast<const unsigned*>(p));
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
}

// Thread 0 waits (bounded) until *cnt reaches `target` (no wait and no load when cnt is NULL); the
// verdict is shared with the whole CTA through one barrier (s_flag is not written again before the task's
// closing barrier).
__device__ bool wait_count(const FftParams& P, const int* cnt, int target, int* s_flag) {
    if (threadIdx.x == 0) {
        int ok = 1;
        const long long t0 = clock64();
        while (cnt && ld_acquire(cnt) < target) {
            if (clock64() - t0 > P.wait_budget || ld_relaxed(P.tickets + 1)) {
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        if (!ok) {
            atomicOr(P.status, DEV_ERR_TIMEOUT);
            atomicExch(P.tickets + 1, 1);
        }
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// The same for one warp: lane 0 waits (bounded) until *cnt reaches `target`, starting from `seen`, a value of
// *cnt it acquired earlier (no wait when that already reaches the target, or when cnt is NULL); the
// warp barrier orders the other lanes' later accesses after lane 0's acquire.
__device__ bool warp_wait(const FftParams& P, const int* cnt, int target, int seen) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0 && cnt && seen < target) {
        const long long t0 = clock64();
        while (ld_acquire(cnt) < target) {
            if (clock64() - t0 > P.wait_budget || ld_relaxed(P.tickets + 1)) {
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        if (!ok) {
            atomicOr(P.status, DEV_ERR_TIMEOUT);
            atomicExch(P.tickets + 1, 1);
        }
    }
    ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
    __syncwarp();
    return ok != 0;
}

__host__ __device__ constexpr int even(int x) { return (x + 1) / 2 * 2; }
// Column tile stride (in elements) and row buffer stride: room for the warp transforms' layouts, and
// 16 / kCW mod 16 slots so that the tile's row-wise store phase (kCW columns x 16 / kCW rows per half-warp)
// is free of bank conflicts.
template <int N> __host__ __device__ constexpr int tile_ld() { return wfft_slots(N) + 16 / kCW; }

// Two 256-point inverse transforms by one warp in two radix-16 Stockham passes: rows at s and s + stride
// (padx layout), half-warp h transforms row h and lane j = lane % 16 takes butterfly j of each pass.  tw16
// holds exp(2 pi i j r / 256) at [(r - 1) * 16 + j].  Results go to out(h, position, value).
template <typename Out>
__device__ __forceinline__ void warp_fft256x2(float2* s, int stride, const float2* tw16, int lane, Out& out) {
    const int h = lane >> 4, j = lane & 15;
    float2* b = s + h * stride;
    float2 v[16];
    // pass 1: inputs j + 16 r (padded: j + 17 r), outputs 16 j + r (padded: 17 j + r); both conflict-free
#pragma unroll
    for (int r = 0; r < 16; r++) v[r] = b[j + 17 * r];
    idft<16>(v);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; r++) b[17 * j + r] = v[r];
    __syncwarp();
    // pass 2: inputs j + 16 r, twiddles of k = j, outputs j + 16 r (natural order)
#pragma unroll
    for (int r = 0; r < 16; r++) v[r] = b[j + 17 * r];
#pragma unroll
    for (int r = 1; r < 16; r++) v[r] = cmul(v[r], tw16[(r - 1) * 16 + j]);
    idft<16>(v);
#pragma unroll
    for (int r = 0; r < 16; r++) out(h, j + 16 * r, v[r]);
}

// exp(2 pi i q / 32) for a compile-time q in [0, 16): cos(k pi / 16) for k = 0 .. 8 gives both parts.
__device__ __forceinline__ float2 w32(int q) {
    constexpr float C[9] = {1.0f, 0.98078528040323044913f, 0.92387953251128675613f, 0.83146961230254523708f,
                            0.70710678118654752440f, 0.55557023301960222474f, 0.38268343236508977173f,
                            0.19509032201612826785f, 0.0f};
    return make_float2(q <= 8 ? C[q] : -C[16 - q], C[q <= 8 ? 8 - q : q - 8]);
}

// One 512-point inverse transform by one warp in two Stockham passes: radix 16 (butterfly j = lane, points
// j + 32 r), then radix 32 with twiddles of k = b (butterfly b = lane % 16, points b + 16 r), each radix-32
// butterfly split over lanes b and b + 16: lane h = lane / 16 transforms the points of r = 2 s + h with 16
// points and one exchange of the halves combines them.  Positions are padx; the first pass reads only the
// points `occ` marks (point lane + 32 r: bit r) and treats the others as zero.  tw32 holds exp(2 pi i k r / 512)
// at [r * 16 + k], r < 32, k < 16.
template <typename T>
__device__ __forceinline__ void warp_fft512(T* s, const float2* tw32, int lane, uint32_t occ) {
    float2 v[16];
    const int pj = lane + (lane >> 4);              // padx(lane + 32 r) = pj + 34 r
    // pass 1: inputs lane + 32 r, outputs 16 lane + r (padded 17 lane + r): both conflict-free
#pragma unroll
    for (int r = 0; r < 16; r++) v[r] = ((occ >> r) & 1u) ? ld_c(s + pj + 34 * r) : make_float2(0.f, 0.f);
    idft<16>(v);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; r++) st_c(s + 17 * lane + r, v[r]);
    __syncwarp();
    // pass 2: lane (b, h) reads points b + 16 (2 s + h) = lane + 32 s and twiddles them by exp(2 pi i b r / 512)
    const int b = lane & 15, h = lane >> 4;
#pragma unroll
    for (int q = 0; q < 16; q++) v[q] = cmul(ld_c(s + pj + 34 * q), tw32[32 * q + lane]);
    idft<16>(v);                                    // E (h = 0) or O (h = 1)
    __syncwarp();
    // X[q + 16 h] = E[q] + (-1)^h exp(2 pi i q / 32) O[q], at position b + 16 (q + 16 h) (padded b + 17 q + 272 h)
#pragma unroll
    for (int q = 0; q < 16; q++) {
        const float2 mine = v[q];
        const float2 other = make_float2(__shfl_xor_sync(0xFFFFFFFFu, mine.x, 16),
                                         __shfl_xor_sync(0xFFFFFFFFu, mine.y, 16));
        const float2 e = h ? other : mine, t = cmul(h ? mine : other, w32(q));
        st_c(s + b + 17 * q + 272 * h, h ? csub(e, t) : cadd(e, t));
    }
    __syncwarp();
}

// Unnormalised inverse DFT of 32 points in registers, v[q] <- sum_r v[r] exp(+2 pi i r q / 32): the 16-point
// transforms of the even and the odd points, combined with exp(2 pi i q / 32).
__device__ __forceinline__ void idft32(float2 (&v)[32]) {
    float2 e[16], o[16];
#pragma unroll
    for (int r = 0; r < 16; r++) {
        e[r] = v[2 * r];
        o[r] = v[2 * r + 1];
    }
    idft<16>(e);
    idft<16>(o);
#pragma unroll
    for (int q = 0; q < 16; q++) {
        const float2 t = cmul(o[q], w32(q));
        v[q] = cadd(e[q], t);
        v[q + 16] = csub(e[q], t);
    }
}

// First pass of the 512-point column transform by one warp on a column of kCol512Ld slots whose first 512 hold
// point v at slot v (lane = j, points n = j + 32 r): the radix-16 DFT over r, with Y[j][k1] stored at slot
// 17 j + k1, so that both these stores (lanes j, fixed k1) and the second pass's reads of Y[.][b] (lanes b,
// fixed j) touch 16 distinct 8-byte bank pairs per half-warp, at a base plus constant offsets.  The pass
// reads only the points `occ` marks (point lane + 32 r: bit r) and treats the others as zero.
constexpr int kCol512Ld = 32 * 17;
template <typename T>
__device__ __forceinline__ void col512_pass1(T* s, int lane, uint32_t occ) {
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; r++) v[r] = ((occ >> r) & 1u) ? ld_c(s + lane + 32 * r) : make_float2(0.f, 0.f);
    idft<16>(v);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; r++) st_c(s + 17 * lane + r, v[r]);
}

// Complex-to-real pre-twiddle of one pair of row points (Eq. 4 on the Hermitian half plane): from G[q] = zk
// and G[M - q] = zm, with wq = exp(2 pi i q / N), the inputs of the M-point complex transform are
//   Z[q] = A + i C,  Z[M - q] = conj(A) + i conj(C),  A = zk + conj(zm),  C = (zk - conj(zm)) wq,
// written back over zk and zm.
__device__ __forceinline__ void pretw(float2& zk, float2& zm, float2 wq) {
    const float2 A = make_float2(zk.x + zm.x, zk.y - zm.y);
    const float2 C = cmul(make_float2(zk.x - zm.x, zk.y + zm.y), wq);
    zk = make_float2(A.x - C.y, A.y + C.x);
    zm = make_float2(A.x + C.y, C.x - A.y);
}

// Column task of side 512 with the column-major ring: 16 columns u0 + c, two per warp.  Each warp grids its
// two columns (as in column_task), runs the first pass of both, then the second pass with one radix-32
// butterfly per lane (lane = b + 16 c: column c of the warp's pair, butterfly b): with n = j + 32 r and
// k = b + 16 k2,
//   X[b + 16 k2] = sum_j exp(2 pi i j k2 / 32) exp(2 pi i j b / 512) Y[j][b],
// and stores the column from registers, each half-warp writing 16 consecutive points (128 bytes) per
// instruction, once the ring slot's previous image has been read.
template <typename T, bool FUSED>
__device__ int* column_task512(const FftParams& P, int k, int cb, const float2* s_twc, unsigned char* work,
                               uint32_t* s_occ) {
    constexpr int N = 512, M = N / 2, LD = kCol512Ld;     // columns: 512 points, then Y[j][k1] at 17 j + k1
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int f = k / P.n_tau, tau = P.tau0 + k % P.n_tau, id = tau * P.F + f;
    const int slot = k % P.ring;
    // the ring slot's previous occupant, acquired while the gather's first loads are in flight (an acquire
    // holds the warp's later loads until it completes, so it must not precede them)
    const int* prev = k >= P.ring ? P.row_done + (k - P.ring) : nullptr;
    int seen = 0;
    if (kVisAhead > 0 && tid == 0 && cb == 0 && k + kVisAhead < P.n_img && P.vis_prefetch) {
        const int k2 = k + kVisAhead, f2 = k2 / P.n_tau, id2 = (P.tau0 + k2 % P.n_tau) * P.F + f2;
        prefetch_l2(P.vis + (int64_t)(id2 - P.vis_first) * P.vis_stride, P.vis_prefetch);
    }
    T* s = reinterpret_cast<T*>(work);
    // fused form: the image's sums are in its vis-ring slot once its correlation task is done
    if (FUSED && !warp_wait(P, P.corr_done + k, 1, 0)) return P.col_done + k;
    const float2* V = FUSED ? reinterpret_cast<const float2*>(P.vring + (int64_t)(k % P.ring_v) * 2 * P.e_stride)
                            : P.vis + (int64_t)(id - P.vis_first) * P.vis_stride;
    const int* off = P.ent_off + f * (M + 1);
    const int base = off[0];                          // the channel's first entry (gather order's position 0)
    const float* Vre = reinterpret_cast<const float*>(V) - base;
    const int u0 = cb * 2 * kCW + 2 * warp;           // the warp's columns u0, u0 + 1
    // 1 / (W * 2K) (or 1 / (W * K)) is applied to each gridded cell: the transforms are linear, so the image
    // comes out scaled, and a cell costs one product where an image pixel would
    const float wk = __ldg(P.wk + f);
    const float inv = 1.0f / (wk > 0.f ? wk : 1.f);
    {
        // both columns in one pass over their (contiguous) entries
        uint32_t* occ = s_occ + 2 * warp * 32;
        occ[lane] = 0u;
        occ[32 + lane] = 0u;
        __syncwarp();
        auto idx = [&](int u, int v) { return (2 * warp + (u - u0)) * LD + v; };
        auto occw = [&](int u, int v) { return occ + (u - u0) * 32 + (v & 31); };
        auto gather = [&](auto val) {
            warp_gather_occ_batched<4>(P.ent, off[u0], off[u0 + 2], lane, s, val, idx, occw, inv, [&]() {
                if (lane == 0 && prev) seen = ld_acquire(prev);
            });
        };
        // one instance per order of the sums, so that the choice stays outside the unrolled loads
        if (FUSED || P.gathered)
            gather([&](int i, uint32_t) { return make_float2(__ldcs(Vre + i), __ldcs(Vre + P.e_stride + i)); });
        else
            gather([&](int, uint32_t b) { return __ldcs(V + b); });
        __syncwarp();
        col512_pass1(s + 2 * warp * LD, lane, occ[lane]);
        col512_pass1(s + (2 * warp + 1) * LD, lane, occ[32 + lane]);
    }
    __syncwarp();
    const int b = lane & 15, c = lane >> 4;
    const T* y = s + (2 * warp + c) * LD + b;         // Y[j][b] at 17 j + b
    float2 v[32];
#pragma unroll
    for (int j = 0; j < 32; j++) v[j] = ld_c(y + 17 * j);
#pragma unroll
    for (int j = 1; j < 32; j++) v[j] = cmul(v[j], s_twc[16 * j + b]);
    idft32(v);
    if (warp_wait(P, prev, P.n_rb, seen)) {
        T* dst = static_cast<T*>(P.H) + (int64_t)slot * M * N + (int64_t)(u0 + c) * N + b;
#pragma unroll
        for (int k2 = 0; k2 < 32; k2++) st_c(dst + 16 * k2, v[k2]);
    }
    return P.col_done + k;
}

// Row task of side 512 (32 rows y0 + l, l = lane) with the column-major ring: the first radix-16 pass of the
// 256-point row transform in registers (lanes = rows), one exchange through shared memory, the second pass
// with two rows per warp.  With the point index n = j + 16 r of the row (u = n) and m = k1 + 16 k2 of the
// output pixel pair (2m, 2m + 1):
//   Y[j][k1] = exp(2 pi i j k1 / 256) sum_r Z[j + 16 r] exp(2 pi i r k1 / 16),
//   X[k1 + 16 k2] = sum_j Y[j][k1] exp(2 pi i j k2 / 16).
// The ring slot's row count is released as soon as every warp has read its rows.
template <typename T>
__device__ int* row_task512(const FftParams& P, int k, int rb, unsigned char* work) {
    constexpr int N = 512, M = N / 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int f = k / P.n_tau, tau = P.tau0 + k % P.n_tau, id = tau * P.F + f;
    const int slot = k % P.ring;
    const int y0 = rb * 32;
    float2* S = reinterpret_cast<float2*>(work);
    const bool ok = warp_wait(P, P.col_done + k, P.n_cb + P.extra_wait, 0);
    if (ok) {
        const int jA = warp == 0 ? 0 : warp, jB = warp == 0 ? 8 : 16 - warp;
        const int tb = warp * kRowTw;               // the warp's twiddle row
        auto tw = [&](int q) { return c_rowtw512[tb + q]; };
        const T* col = static_cast<const T*>(P.H) + (int64_t)slot * M * N + y0 + lane;
        float2 a[16], b[16];
#pragma unroll
        for (int r = 0; r < 16; r++) {
            a[r] = ldcg_c(col + (int64_t)(jA + 16 * r) * N);
            b[r] = ldcg_c(col + (int64_t)(jB + 16 * r) * N);
        }
        if (warp == 0) {
            // butterfly 0: u = 16 r pairs with 16 (16 - r); u = 0 with the (empty) Nyquist column, u = 128 with
            // itself.  Butterfly 8: u = 8 + 16 r pairs with 8 + 16 (15 - r).
            float2 z = make_float2(0.f, 0.f);
            pretw(a[0], z, tw(0));
#pragma unroll
            for (int r = 1; r < 8; r++) pretw(a[r], a[16 - r], tw(r));
            z = a[8];
            pretw(a[8], z, tw(8));
#pragma unroll
            for (int r = 0; r < 8; r++) pretw(b[r], b[15 - r], tw(9 + r));
        } else {
            // u = j + 16 s pairs with 256 - u = (16 - j) + 16 (15 - s); the pair's smaller index gives wq
#pragma unroll
            for (int s = 0; s < 8; s++) {
                pretw(a[s], b[15 - s], tw(s));
                pretw(b[s], a[15 - s], tw(9 + s));
            }
        }
        auto pass1 = [&](float2(&v)[16], int j, int t0) {
            idft<16>(v);
            float2* dst = S + lane * kRowLd + 16 * j;
            dst[0] = v[0];
#pragma unroll
            for (int k1 = 1; k1 < 16; k1++) dst[k1] = cmul(v[k1], tw(t0 + k1 - 1));
        };
        pass1(a, jA, 17);
        pass1(b, jB, 32);
    }
    if (__syncthreads_or(!ok)) return nullptr;
    if (tid == 0) {                                     // every warp's ring reads are done
        __threadfence();
        atomicAdd(P.row_done + k, 1);
    }
    const int h = lane >> 4, k1 = lane & 15;
#pragma unroll 1
    for (int it = 0; it < 2; it++) {
        const int rr = warp + 8 * (2 * it + h);
        const float2* src = S + rr * kRowLd + k1;
        float2 v[16];
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = src[16 * j];
        idft<16>(v);
        // the column tasks gridded the cells already scaled by 1 / (W * 2K)
        float2* out = reinterpret_cast<float2*>(P.img_out + ((int64_t)(id - P.out_first) * N + y0 + rr) * N) + k1;
#pragma unroll
        for (int k2 = 0; k2 < 16; k2++) __stcs(out + 16 * k2, v[k2]);
    }
    return nullptr;
}

// Correlation task of image k in the fused form (Eq. 2, Sec. 5.2.2): the Stokes-I (or XX) integer sums of its
// item (integration tau, output channel f) on the tensor cores, as in the standalone FP8 correlator - K in
// chunks of ns_c samples bulk-copied to shared memory, unpacked to e4m3 operand tiles (the realified complex
// product), MMAs accumulating in TMEM - with the CTA's 128 TMEM columns holding two 64 x 64 block pairs per
// round.  Each round's sums go from TMEM to the image's vis-ring slot at the gather positions of their
// baselines (two for a baseline of the column u = 0).  Returns false if a wait ran out (the launch aborts).
__device__ bool corr_task512(const FftParams& P, int k, unsigned char* work, const uint32_t* lut, const uint8_t* sflags,
                             uint32_t tmem, uint32_t bar_raw, uint32_t bar_mma, uint32_t& par_raw, uint32_t& par_mma,
                             int* s_flag) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int f = k / P.n_tau, tau = P.tau0 + k % P.n_tau;
    const int nt = P.n_tiles;
    // the vis-ring slot's previous image must have been gridded by all its column tasks
    const int* prev = k >= P.ring_v ? P.col_done + (k - P.ring_v) : nullptr;
    if (!wait_count(P, prev, P.n_cb, s_flag)) return false;
    if (smem_u32(work) & 15) return false;             // operands and bulk copies need 16-byte alignment
    const uint32_t tile_bytes = 128u * P.Kp;
    uint8_t* ops = work;
    uint8_t* raw = work + P.n_blk * tile_bytes;
    // the work area last held another task's data: zero the operand tiles, so that the K padding of every row
    // and the rows past the last tile, which the unpack never writes, contribute nothing
    for (uint32_t e = tid; e < (uint32_t)P.n_blk * tile_bytes / 16; e += kPT)
        reinterpret_cast<uint4*>(ops)[e] = make_uint4(0u, 0u, 0u, 0u);
    const uint32_t row_bytes = (uint32_t)P.cavg * nt * 2;   // one sample's c channels of all tiles
    const int n_pairs = P.n_blk * (P.n_blk + 1) / 2;
    const uint32_t idesc = idesc_e4m3(128, 64), ops_s = smem_u32(ops), sbo = (uint32_t)P.Kp * 8;
    float* vout = P.vring + (int64_t)(k % P.ring_v) * 2 * P.e_stride;
    const uint32_t* gp = P.gpos + (int64_t)f * P.B;
    // the item's raw samples, all of them, once: one bulk copy per sample of its c channels
    if (tid == 0) {
        mbar_expect_tx(bar_raw, (uint32_t)P.ns * row_bytes);
        const uint8_t* src = P.volt + (int64_t)tau * P.ns * P.sample_stride + (int64_t)f * row_bytes;
        for (int q = 0; q < P.ns; q++)
            bulk_load(smem_u32(raw) + q * row_bytes, src + (int64_t)q * P.sample_stride, row_bytes, bar_raw);
    }
    {
        bool ok = mbar_wait(bar_raw, par_raw, P.wait_budget);
        if (!ok) ok = mbar_wait(bar_raw, par_raw, P.wait_budget);          // let copies in flight land
        par_raw ^= 1;
        if (__syncthreads_or(!ok)) return false;
    }
    for (int q0 = 0; q0 < n_pairs; q0 += 2) {
        const int q1 = min(n_pairs, q0 + 2);
        for (int j = 0; j < P.n_chunks; j++) {
            const int s0 = j * P.ns_c, sn = min(P.ns_c, P.ns - s0);
            const uint8_t* rj = raw + (size_t)s0 * row_bytes;
            if (P.stokes)
                unpack_e4m3<true, false>(rj, lut, sflags, ops, tile_bytes, nt, P.Kq, P.Kp, sn * P.cavg, tid, kPT);
            else
                unpack_e4m3<false, false>(rj, lut, sflags, ops, tile_bytes, nt, P.Kq, P.Kp, sn * P.cavg, tid, kPT);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                for (int q = q0; q < q1; q++) {
                    int mb, jb;
                    pair_of(q, mb, jb);
                    const uint32_t d = tmem + (uint32_t)((q - q0) * 64);
                    const uint32_t a0 = ops_s + mb * tile_bytes, b0 = ops_s + jb * tile_bytes;
                    for (int ks = 0; ks < P.Kp / 32; ks++)
                        mma_e4m3(d, smem_desc(a0 + ks * 256, 128, sbo), smem_desc(b0 + ks * 256, 128, sbo), idesc,
                                 j > 0 || ks > 0);
                }
                mma_commit(bar_mma);
            }
            bool okm = mbar_wait(bar_mma, par_mma, P.wait_budget);
            if (!okm) okm = mbar_wait(bar_mma, par_mma, P.wait_budget);    // the MMAs still read shared memory
            par_mma ^= 1;
            if (__syncthreads_or(!okm)) return false;
            tc_fence_after();
        }
        // warps 0-3 read block pair q0, warps 4-7 pair q0 + 1: TMEM lane 32 (w % 4) + lane = unit row (re for
        // rows below 64, im above), 64 columns = units of the pair's column block
        const int q = q0 + (warp >> 2);
        if (q < q1) {
            int mb, jb;
            pair_of(q, mb, jb);
            const int row = (warp & 3) * 32 + lane;
            const int ui = mb * 64 + (row & 63);
            float* plane = vout + (row >> 6) * P.e_stride;
            const int64_t brow = (int64_t)ui * (ui + 1) / 2;
#pragma unroll 1
            for (int c0 = 0; c0 < 64; c0 += 32) {
                // the positions of 32 baselines in flight together, then their sums from TMEM
                uint32_t w[32];
#pragma unroll
                for (int cc = 0; cc < 32; cc++) {
                    const int uj = jb * 64 + c0 + cc;
                    w[cc] = (ui < nt && uj <= ui) ? __ldg(gp + brow + uj) : 0xFFFFFFFFu;
                }
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    uint32_t v[16];
                    tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((q - q0) * 64 + c0 + 16 * h), v);
#pragma unroll
                    for (int cc = 0; cc < 16; cc++) {
                        const uint32_t p1 = w[16 * h + cc] & 0xFFFFu, p2 = w[16 * h + cc] >> 16;
                        if (p1 != 0xFFFFu) plane[p1] = __uint_as_float(v[cc]);
                        if (p2 != 0xFFFFu) plane[p2] = __uint_as_float(v[cc]);
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    return true;
}

// Grid column u (zeroed by the caller) from the separable form of a kernel's list: entries [beg, end) name
// the records whose support meets the column, sorted by (v0, record).  Entry e adds its record's sum (conjugated
// for a mirror) times C(u - gu) C(v - gv) (-1)^(u + v) to each row v = v0 + k, k < W (mod N); the row weights
// carry (-1)^k.  Lanes take an entry each, two chunks of 32 loaded together (their entries, then their sums
// and weight rows).  Entries with equal v0 take turns by their rank among them, so that in each of a turn's W
// steps the lanes write different cells, and each cell's additions come in a fixed order.
template <int N, typename Cell>
__device__ __forceinline__ void warp_gather_sep(const uint4* __restrict__ ent, const float* __restrict__ wrow,
                                                const float2* __restrict__ V, int beg, int end, int W, int lane, int u,
                                                Cell cell) {
    constexpr int NB = 2;
    for (int base = beg; base < end; base += 32 * NB) {
        uint4 e[NB];
#pragma unroll
        for (int q = 0; q < NB; q++) {
            const int i = base + 32 * q + lane;
            e[q] = i < end ? __ldg(ent + i) : make_uint4(0u, 0x7FFFFFFFu, 0u, 0u);
        }
        float2 x[NB];
        float4 w0[NB], w1[NB];
#pragma unroll
        for (int q = 0; q < NB; q++) {
            x[q] = make_float2(0.f, 0.f);
            w0[q] = w1[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (base + 32 * q + lane < end) {
                x[q] = __ldg(V + (e[q].x & 0x7FFFFFFFu));
                const float4* wr = reinterpret_cast<const float4*>(wrow + e[q].w);
                w0[q] = __ldg(wr);
                w1[q] = __ldg(wr + 1);
            }
        }
#pragma unroll
        for (int q = 0; q < NB; q++) {
            if (base + 32 * q >= end) break;
            const bool ok = base + 32 * q + lane < end;
            const int v0 = (int)e[q].y;                     // 0x7FFFFFFF past the end: equal to no v0
            float2 y = x[q];
            if (e[q].x >> 31) y.y = -y.y;
            const float wu = ((u ^ v0) & 1) ? -__uint_as_float(e[q].z) : __uint_as_float(e[q].z);
            y = make_float2(y.x * wu, y.y * wu);
            const float w[kSepMaxW] = {w0[q].x, w0[q].y, w0[q].z, w0[q].w, w1[q].x, w1[q].y, w1[q].z, w1[q].w};
            const unsigned same = __match_any_sync(0xFFFFFFFFu, v0);
            const int rank = __popc(same & ((1u << lane) - 1u));
            const int turns = __reduce_max_sync(0xFFFFFFFFu, ok ? (unsigned)rank : 0u) + 1;
            for (int t = 0; t < turns; t++) {
                const bool mine = ok && rank == t;
#pragma unroll
                for (int k = 0; k < kSepMaxW; k++) {
                    if (k >= W) break;
                    if (mine) {
                        float2* c = cell((v0 + k) & (N - 1));
                        const float2 a = *c;
                        *c = make_float2(fmaf(y.x, w[k], a.x), fmaf(y.y, w[k], a.y));
                    }
                    __syncwarp();
                }
            }
        }
    }
}

// The tasks return the counter their completion increments (NULL after an abort); the caller releases it.
// With WT (gridding with a convolution kernel) every gather entry carries a weight, the grid side N is twice
// the image side, and the row tasks transform only the central N/2 rows and keep their central N/2 pixels,
// multiplied by the grid correction.
template <int N, typename T, bool WT>
__device__ int* column_task(const FftParams& P, int k, int cb, const float2* s_twc, unsigned char* work,
                            uint32_t* s_occ, int* s_flag) {
    constexpr int CW = kCW, LD = tile_ld<N>();
    const int tid = threadIdx.x;
    const int f = k / P.n_tau, tau = P.tau0 + k % P.n_tau, id = tau * P.F + f;
    const int slot = k % P.ring;
    const int warp = tid >> 5, lane = tid & 31;
    // the ring slot's previous occupant, read now so that the load overlaps the gridding and transforms
    const int* prev = k >= P.ring ? P.row_done + (k - P.ring) : nullptr;
    int prev_done = 0;
    if (tid == 0 && prev) prev_done = ld_acquire(prev);
    // the visibilities of the image kVisAhead images on, brought into L2 for its gridding
    if (kVisAhead > 0 && tid == 0 && cb == 0 && k + kVisAhead < P.n_img && P.vis_prefetch) {
        const int k2 = k + kVisAhead, f2 = k2 / P.n_tau, id2 = (P.tau0 + k2 % P.n_tau) * P.F + f2;
        prefetch_l2(P.vis + (int64_t)(id2 - P.vis_first) * P.vis_stride, P.vis_prefetch);
    }
    T* s = reinterpret_cast<T*>(work);
    T* col = s + warp * LD;                              // this warp's column
    const float2* V = P.vis + (int64_t)(id - P.vis_first) * P.vis_stride;
    auto val = [&](uint32_t b) { return __ldcs(V + b); };          // read once: do not keep in L2
    const int u = cb * CW + warp;
    auto idx = [&](int, int v) { return warp * LD + padx(v); };
    const int* off = P.ent_off + f * (N / 2 + 1);
    const int beg = off[u], end = off[u + 1];
    const float* wt = WT ? P.wt : nullptr;
    if constexpr (N >= 256 && N <= 1024) {
        uint32_t* occ = s_occ + warp * 32;
        bool sep = false;
        if constexpr (WT && std::is_same_v<T, float2>) {
            sep = P.sep != nullptr;
            if (sep) {
                // a kernel's separable list: the column zeroed, then each record's W rows added; all rows read
                for (int e = lane; e < LD; e += 32) col[e] = make_float2(0.f, 0.f);
                occ[lane] = 0xFFFFFFFFu;
                __syncwarp();
                const int* so = P.sep_off + f * (N / 2 + 1);
                warp_gather_sep<N>(P.sep, P.sep_w, V, so[u], so[u + 1], P.sep_W, lane, u,
                                   [&](int v) { return col + padx(v); });
            }
        }
        if (!sep) {
            // no zeroing: the gridding marks the cells it writes, and the first pass reads only those; the
            // entries (and weights) of four chunks are loaded together, then their sums (baseline order: after
            // the entries)
            occ[lane] = 0u;
            __syncwarp();
            // gather-ordered sums (planes of e_stride floats from the channel's first entry; nearest cell only)
            // or baseline order, one instance each
            const float* Vre = reinterpret_cast<const float*>(V) - off[0];
            auto gather = [&](auto valg) {
                warp_gather_occ_batched<4>(P.ent, beg, end, lane, s, valg, idx,
                                           [&](int, int v) { return occ + (v & 31); }, 1.0f, [] {}, wt);
            };
            if (!WT && P.gathered)
                gather([&](int i, uint32_t) { return make_float2(__ldcs(Vre + i), __ldcs(Vre + P.e_stride + i)); });
            else
                gather([&](int, uint32_t b) { return val(b); });
        }
        __syncwarp();
        if constexpr (N == 512)
            warp_fft512(col, s_twc, lane, occ[lane]);
        else
            warp_fft_masked<N, T>(col, s_twc, lane, occ[lane]);
    } else {
        bool sep = false;
        if constexpr (WT && std::is_same_v<T, float2>) {
            sep = P.sep != nullptr;
            if (sep) {
                // a kernel's separable list on the zeroed column
                for (int e = lane; e < LD; e += 32) col[e] = make_float2(0.f, 0.f);
                __syncwarp();
                const int* so = P.sep_off + f * (N / 2 + 1);
                warp_gather_sep<N>(P.sep, P.sep_w, V, so[u], so[u + 1], P.sep_W, lane, u,
                                   [&](int v) { return col + padx(v); });
            }
        }
        if (!sep) {
            uint32_t key;
            float2 x;
            gather_entry(P.ent, wt, beg + lane, end, val, key, x);    // in flight while the column is zeroed
            for (int e = lane; e < LD; e += 32) st_c(col + e, make_float2(0.f, 0.f));
            __syncwarp();
            warp_gather_column(P.ent, wt, beg, end, lane, s, val, idx, true, key, x);
        }
        __syncwarp();
        NoOut none;
        warp_fft<N, false, T, NoOut>(col, s_twc, lane, none);
    }
    // all columns transformed (the wait's barrier), and the ring slot free of its previous image
    if (!wait_count(P, prev_done >= P.n_rb ? nullptr : prev, P.n_rb, s_flag)) return nullptr;
    // with a kernel the row tasks read only the central N/2 rows, so only those are stored
    constexpr int YS = WT ? N / 4 : 0, NY = WT ? N / 2 : N;
    T* out = static_cast<T*>(P.H) + (int64_t)slot * N * P.ldh + cb * CW;
    for (int e = tid; e < NY * CW; e += kPT) {
        const int y = YS + e / CW, c = e % CW;
        out[(int64_t)y * P.ldh + c] = s[c * LD + padx(y)];
    }
    return P.col_done + k;
}

template <int N, typename T, bool WT>
__device__ int* row_task(const FftParams& P, int k, int rb, const float2* s_pre, const float2* s_twr,
                         unsigned char* work, int* s_flag) {
    constexpr int M = N / 2, LS = tile_ld<M>();
    constexpr int NI = WT ? N / 2 : N;                  // image side
    constexpr int Y0 = WT ? N / 4 : 0;                  // grid row of image row 0
    constexpr int X0 = WT ? N / 8 : 0;                  // first output pair m kept (grid pixels 2m, 2m + 1)
    const int tid = threadIdx.x, r = tid >> 5, lane = tid & 31;
    const int f = k / P.n_tau, tau = P.tau0 + k % P.n_tau, id = tau * P.F + f;
    const int slot = k % P.ring;
    if (!wait_count(P, P.col_done + k, P.n_cb + P.extra_wait, s_flag)) return nullptr;
    const float w = P.wk[f];
    const float inv = 1.0f / (w > 0.f ? w : 1.f);
#pragma unroll 1
    for (int b = 0; b < kRowBatches; b++) {
        const int y0 = Y0 + (rb * kRowBatches + b) * kRB;  // the batch's rows: y0 + h * kW + r (warp r)
#pragma unroll
        for (int h = 0; h < kRPW; h++) {
            const int y = y0 + h * kW + r;
            const T* row = static_cast<const T*>(P.H) + ((int64_t)slot * N + y) * P.ldh;
            float2* dst = reinterpret_cast<float2*>(work) + (h * kW + r) * LS;
#pragma unroll
            for (int q = lane; q <= M / 2; q += 32) {   // unrolled: every load of the rows is issued at once
                const float2 zk = ldcg_c(row + q);
                const float2 zm = (q == 0) ? make_float2(0.f, 0.f) : ldcg_c(row + (M - q));
                const float2 wq = s_pre[q];               // exp(2 pi i q / N); that of M - q is -conj(wq)
                dst[padx(q)] = cadd(cadd(zk, conjf2(zm)), cmul_i(cmul(csub(zk, conjf2(zm)), wq)));
                if (q > 0 && q < M - q)
                    dst[padx(M - q)] = cadd(cadd(zm, conjf2(zk)), cmul_i(cmul(csub(zm, conjf2(zk)), make_float2(-wq.x, wq.y))));
            }
        }
        __syncwarp();
        // image row (y - Y0) of grid row y; with a kernel each row and pixel is scaled by its grid correction
        auto row_scale = [&](int y) { return WT ? inv * __ldg(P.corr + (y - Y0)) : inv; };
        auto put = [&](float2* out, float sy, int m, float2 v) {    // streaming: the images are not read back
            if constexpr (WT) {
                if (m >= X0 && m < X0 + NI / 2) {
                    const float2 c = __ldg(reinterpret_cast<const float2*>(P.corr) + (m - X0));
                    __stcs(out + (m - X0), make_float2(v.x * sy * c.x, v.y * sy * c.y));
                }
            } else {
                __stcs(out + m, make_float2(v.x * sy, v.y * sy));
            }
        };
        if constexpr (M == 256 && kRPW == 2) {
            // both rows at once: rows h * kW + r of the buffer, grid rows y0 + h * kW + r
            float2* out = reinterpret_cast<float2*>(P.img_out + ((int64_t)(id - P.out_first) * NI + y0 - Y0 + r) * NI);
            const float s0 = row_scale(y0 + r), s1 = row_scale(y0 + kW + r);
            auto store = [&](int h, int m, float2 v) { put(out + h * kW * (NI / 2), h ? s1 : s0, m, v); };
            warp_fft256x2(reinterpret_cast<float2*>(work) + r * LS, kW * LS, s_twr, lane, store);
        } else {
#pragma unroll 1
            for (int h = 0; h < kRPW; h++) {
                const int y = y0 + h * kW + r;
                float2* dst = reinterpret_cast<float2*>(work) + (h * kW + r) * LS;
                float2* out = reinterpret_cast<float2*>(P.img_out + ((int64_t)(id - P.out_first) * NI + y - Y0) * NI);
                const float sy = row_scale(y);
                auto store = [&](int, int m, float2 v) { put(out, sy, m, v); };
                warp_fft<M, true, float2, decltype(store)>(dst, s_twr, lane, store);
            }
        }
        __syncwarp();                                   // the warp's rows are rewritten by the next batch
    }
    return P.row_done + k;
}

// Side 512 with nearest-cell gridding keeps the column-major ring and the register row pass.
template <int N, bool WT> constexpr bool ring_cm() { return N == 512 && !WT; }

template <int N, typename T, bool WT> constexpr size_t fft_smem() {
    constexpr int M = N / 2;
    constexpr size_t col = (size_t)kCW * tile_ld<N>() * sizeof(T);
    if constexpr (ring_cm<N, WT>()) {
        constexpr size_t col2 = (size_t)2 * kCW * kCol512Ld * sizeof(T);   // two columns per warp
        constexpr size_t row = (size_t)32 * kRowLd * sizeof(float2);
        return (size_t)32 * 16 * sizeof(float2) + (col2 > row ? col2 : row);
    } else {
        constexpr size_t tw = (size_t)(even(tw_size(N)) + even(M / 2 + 1) + even(tw_size(M))) * sizeof(float2);
        constexpr size_t row = (size_t)kRB * tile_ld<M>() * sizeof(float2);
        return tw + (col > row ? col : row);
    }
}

// MINB resident CTAs per SM: 4 (32 warps) for sides up to 512 in the row-major form (measured faster than 24
// warps, despite a few register spills), 2 or 3 for the side-512 column-major form (its register row pass
// holds two butterflies' 32 points per lane; the autotuner picks), 1 above 512.
// FUSED (side 512 only): the instance with correlation tasks; the others carry none of their code or shared data.
template <int N, typename T, bool WT, int MINB, bool FUSED = false>
__global__ void __launch_bounds__(kPT, MINB) k_fft_persistent(const FftParams P) {
    constexpr int M = N / 2;
    constexpr bool CM = ring_cm<N, WT>();
    static_assert(!FUSED || CM, "correlation tasks run in the side-512 column-major form only");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* s_twc = reinterpret_cast<float2*>(smem_raw);
    float2* s_pre = s_twc + (CM ? 32 * 16 : even(tw_size(N)));
    float2* s_twr = s_pre + (CM ? 0 : even(M / 2 + 1));
    unsigned char* work = reinterpret_cast<unsigned char*>(s_twr + (CM ? 0 : even(tw_size(M))));
    __shared__ int s_ticket[2], s_flag;
    __shared__ uint32_t s_occ[2 * kW * 32];        // per column of a task: its occupancy, one word per lane
    const int tid = threadIdx.x;
    if constexpr (N == 512) {
        // exp(2 pi i k r / 512) = the pre-twiddle table's entry m = k r, or minus that of m - 256
        static_assert(32 * 16 <= even(tw_size(N)), "radix-32 table must fit the column table's room");
        for (int e = tid; e < 32 * 16; e += kPT) {
            const int m = (e & 15) * (e >> 4);
            const float2 w = P.tw[tws_pre(N) + (m <= N / 2 ? m : m - N / 2)];
            s_twc[e] = m <= N / 2 ? w : make_float2(-w.x, -w.y);
        }
    } else {
        for (int e = tid; e < tw_size(N); e += kPT) s_twc[e] = P.tw[tws_col(N) + e];
    }
    if constexpr (!CM) {
        for (int e = tid; e <= M / 2; e += kPT) s_pre[e] = P.tw[tws_pre(N) + e];
        if constexpr (M == 256 && kRPW == 2) {
            // exp(2 pi i j r / 256) = exp(2 pi i m / N) with m = 2 j r: the pre-twiddle table's entry m, or minus
            // that of m - N / 2 (entries 0 .. N / 2 are stored)
            static_assert(15 * 16 <= tw_size(M), "radix-16 table must fit the row table's room");
            for (int e = tid; e < 15 * 16; e += kPT) {
                const int m = 2 * (e & 15) * (e / 16 + 1);
                const float2 w = P.tw[tws_pre(N) + (m <= N / 2 ? m : m - N / 2)];
                s_twr[e] = m <= N / 2 ? w : make_float2(-w.x, -w.y);
            }
        } else {
            for (int e = tid; e < tw_size(M); e += kPT) s_twr[e] = P.tw[tws_row(N) + e];
        }
    }
    // fused form: the CTA's TMEM columns, MMA and copy barriers, the byte -> e4m3 LUT and the flags
    __shared__ uint32_t s_lut[FUSED ? 256 : 1];
    __shared__ uint8_t s_tflags[FUSED ? 512 : 1];
    __shared__ __align__(8) uint64_t s_bars[2];
    __shared__ uint32_t s_tmem;
    uint32_t tmem = 0, par_raw = 0, par_mma = 0;
    const uint32_t bar_raw = (uint32_t)__cvta_generic_to_shared(&s_bars[0]), bar_mma = bar_raw + 8;
    if constexpr (FUSED) {
        {
            if ((tid >> 5) == 0) {
                asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                             ::"r"((uint32_t)__cvta_generic_to_shared(&s_tmem)), "r"(kCorrCols) : "memory");
                asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
            }
            if (tid == 0) {
                mbar_init(bar_raw, 1);
                mbar_init(bar_mma, 1);
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            }
            fill_e4m3_lut(s_lut, tid, kPT);
            for (int a = tid; a < P.n_tiles; a += kPT) s_tflags[a] = P.flags[a] ? 1 : 0;
            if (smem_u32(work) & 15) atomicOr(P.status, DEV_ERR_INDEX);   // (the correlation tasks then refuse)
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            tmem = s_tmem;
        }
    }
    // the ticket stream: segments of (correlation of image s, fused form only) + (column tasks of image
    // s - lead) + (row tasks of image s - lead - lag)
    constexpr int fz = FUSED ? 1 : 0;
    const int seg = fz + P.n_cb + P.n_rb;
    const int total = (P.n_img + P.lag + (fz ? P.lead : 0)) * seg;
    // Thread 0 asks for the next ticket when a task starts, so the atomic's round trip overlaps the task, and
    // publishes it in the other half of a two-entry slot (warps still reading this task's entry are not
    // disturbed).  One barrier ends each task; thread 0 releases the finished task's counter after it (the
    // fence orders the whole CTA's accesses of the task before the counter) while the other warps go on.
    // The abort flag is read with the ticket request, so that its round trip too overlaps the task.
    if (tid == 0) s_ticket[0] = atomicAdd(P.tickets, 1);
    __syncthreads();
    for (int it = 0;; it ^= 1) {
        const int t = s_ticket[it];
        if (t >= total) break;
        int nt = 0, ab = 0;
        if (tid == 0) {
            nt = atomicAdd(P.tickets, 1);
            ab = ld_relaxed(P.tickets + 1);
        }
        const int sg = t / seg, r0 = t - sg * seg;
        int* done = nullptr;
        if (fz && r0 == 0) {
            if constexpr (FUSED) {
                if (sg < P.n_img) {
                    if (corr_task512(P, sg, work, s_lut, s_tflags, tmem, bar_raw, bar_mma, par_raw, par_mma, &s_flag))
                        done = P.corr_done + sg;
                    else if (tid == 0) {
                        atomicOr(P.status, DEV_ERR_TIMEOUT);
                        atomicExch(P.tickets + 1, 1);
                    }
                }
            }
        } else {
            const int r = r0 - fz, kc = sg - (fz ? P.lead : 0);
            if (r < P.n_cb) {
                if (kc >= 0 && kc < P.n_img) {
                    if constexpr (CM)
                        done = column_task512<T, FUSED>(P, kc, r, s_twc, work, s_occ);
                    else
                        done = column_task<N, T, WT>(P, kc, r, s_twc, work, s_occ, &s_flag);
                }
            } else {
                const int k = kc - P.lag;
                if (k >= 0 && k < P.n_img) {
                    if constexpr (CM)
                        done = row_task512<T>(P, k, r - P.n_cb, work);
                    else
                        done = row_task<N, T, WT>(P, k, r - P.n_cb, s_pre, s_twr, work, &s_flag);
                }
            }
        }
        if (tid == 0) s_ticket[it ^ 1] = ab ? total : nt;
        __syncthreads();
        if (tid == 0 && done) {
            __threadfence();
            atomicAdd(done, 1);
        }
    }
    if constexpr (FUSED) {
        {
            tc_fence_before();
            __syncthreads();
            if ((tid >> 5) == 0)
                asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCorrCols) : "memory");
        }
    }
}

template <int N, typename T, bool WT, int MINB, bool FUSED = false>
blink_status launch_n(FftParams P, int n_sm, int ctas_per_sm, cudaStream_t st) {
    auto kern = k_fft_persistent<N, T, WT, MINB, FUSED>;
    const size_t smem = fft_smem<N, T, WT>();
    static int per_sm = 0;                         // attributes and occupancy once per instantiation
    if (!per_sm) {
        if (smem > 48 * 1024)
            BLINK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        BLINK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPT, smem));
    }
    if (per_sm < 1) return set_error(BLINK_ERR_UNSUPPORTED, "persistent FFT kernel does not fit on an SM");
    P.n_cb = N / 2 / (ring_cm<N, WT>() ? 2 * kCW : kCW);
    P.n_rb = (WT ? N / 2 : N) / (kRB * kRowBatches);
    const int per = ctas_per_sm > 0 ? std::min(ctas_per_sm, per_sm) : per_sm;
    kern<<<n_sm * per, kPT, smem, st>>>(P);
    BLINK_CUDA(cudaGetLastError());
    return BLINK_OK;
}

// Instantiation by resident CTAs per SM: the side-512 column-major form at 3 when asked, else 2; the others
// at their fixed bound.
template <int N, typename T, bool WT>
blink_status launch_sized(FftParams P, int n_sm, int ctas_per_sm, cudaStream_t st) {
    if constexpr (ring_cm<N, WT>()) {
        if (P.fused) {
            if constexpr (std::is_same<T, float2>::value) {
                if (ctas_per_sm == 3) return launch_n<N, T, WT, 3, true>(P, n_sm, 3, st);
                return launch_n<N, T, WT, 2, true>(P, n_sm, 2, st);
            }
            return set_error(BLINK_ERR_UNSUPPORTED, "the fused imaging launch stores its ring in FP32");
        }
        if (ctas_per_sm == 3) return launch_n<N, T, WT, 3>(P, n_sm, 3, st);
        return launch_n<N, T, WT, 2>(P, n_sm, 2, st);
    } else if constexpr (N == 1024) {
        if (ctas_per_sm == 2) return launch_n<N, T, WT, 2>(P, n_sm, 2, st);
        return launch_n<N, T, WT, 1>(P, n_sm, ctas_per_sm, st);
    } else {
        return launch_n<N, T, WT, (N <= 512 ? 32 / kW : 1)>(P, n_sm, ctas_per_sm, st);
    }
}

}  // namespace

// Ring of column-pass results and the lag (in images) between an image's column and row tasks: the row
// tasks trail by enough images that they rarely wait, and the ring is a little larger than the lag so that
// reusing a slot rarely waits either, while staying small enough to live in L2.  The autotuner picks among
// these shapes per plan.
std::vector<FftTune> fft_tune_candidates(const Plan& p) {
    if (p.N == 512 && !p.d_wt)
        return {{48, 32, 2}, {64, 32, 2}, {32, 24, 3}, {48, 32, 3}, {48, 24, 3}, {64, 32, 3}, {64, 48, 3},
                {64, 40, 3}, {56, 32, 3}};
    // a ring slot holds N x N/2 complex values: 4 MiB at side 1024, 16 MiB at 2048, so fewer slots stay in L2
    if (p.N >= 2048) return {{4, 2, 0}, {6, 4, 0}, {8, 4, 0}};
    // with a kernel only a slot's central rows are written, and longer rings (more images in flight for the
    // heavier gridding) measured faster
    if (p.N == 1024 && p.d_wt)
        return {{16, 12, 2}, {32, 24, 2}, {40, 32, 2}, {48, 32, 2}, {48, 40, 2}, {56, 32, 2}, {64, 32, 2}, {64, 48, 2}};
    if (p.N == 1024)
        return {{8, 4, 0}, {12, 8, 0}, {16, 8, 0}, {12, 8, 2}, {16, 12, 2}, {24, 16, 0}, {32, 24, 0}, {32, 24, 2}};
    return {{24, 16, 0}, {16, 8, 0}, {32, 24, 0}, {48, 32, 0}, {64, 48, 0}, {40, 32, 0}, {32, 24, 3}};
}
int fft_ring_images_max() { return 64; }

// Sums in gather order: the nearest-cell sides whose column tasks run the batched gather (256 to 1024)
bool fft_takes_gathered(const Plan& p) {
    return p.N >= 256 && p.N <= 1024 && !p.d_wt && p.d_gsrc && p.e_stride > 0;
}

namespace {
constexpr int kRingV = 128, kLead = 96;          // vis-ring slots and the correlation lead (images)

// K chunking of the fused correlation: the largest number of samples whose operand tiles fit the kernel's work
// area beside the item's whole raw block, then balanced over the chunks; 0 if none fits.
struct FusedChunk {
    int ns_c = 0, n_chunks = 0, Kq = 0, Kp = 0, n_blk = 0;
};
FusedChunk fused_chunk(const Plan& p, int ns, int kind) {
    FusedChunk c;
    const int nt = p.n_tiles, cavg = p.chan_avg;
    c.n_blk = (nt + 63) / 64;
    const size_t room = (size_t)32 * kRowLd * sizeof(float2);         // the work area of the side-512 kernel
    auto bytes = [&](int ns_c, int& Kq, int& Kp) {
        Kq = (ns_c * cavg + 3) / 4 * 4;
        const int Kr = kind == CORR_OUT_STOKES_I ? 4 * Kq : 2 * Kq;
        Kp = (Kr + 31) / 32 * 32;
        return (size_t)c.n_blk * 128 * Kp + (size_t)ns * cavg * nt * 2;
    };
    int best = 0;
    for (int ns_c = std::min(ns, 256); ns_c >= 1; ns_c--) {
        int Kq, Kp;
        if (bytes(ns_c, Kq, Kp) <= room) {
            best = ns_c;
            break;
        }
    }
    if (!best) return c;
    c.n_chunks = (ns + best - 1) / best;
    c.ns_c = (ns + c.n_chunks - 1) / c.n_chunks;
    bytes(c.ns_c, c.Kq, c.Kp);
    return c;
}
}  // namespace

bool fft_fused_ok(const Plan& p, int ns, int kind, const uint8_t* d_volt, int64_t sample_stride) {
    if (p.N != 512 || !fft_takes_gathered(p) || !p.d_gpos || p.n_tiles % 8 || p.n_tiles > 512) return false;
    if (kind != CORR_OUT_STOKES_I && kind != CORR_OUT_XX) return false;
    if (((uintptr_t)d_volt & 15) || (sample_stride % 16) || ((int64_t)p.chan_avg * p.n_tiles * 2) % 16) return false;
    const int64_t K = (int64_t)ns * p.chan_avg;
    if ((kind == CORR_OUT_STOKES_I ? 256 : 128) * K >= ((int64_t)1 << 24)) return false;   // exact FP32 sums
    return fused_chunk(p, ns, kind).ns_c > 0;
}

size_t fused_ring_floats(const Plan& p) { return (size_t)kRingV * 2 * p.e_stride; }

// The side-512 row tasks' twiddle rows into constant memory of the current device, from exp(2 pi i m / 512),
// m in [0, 512): the first octant's angles in FP64, the others by the exact symmetries of the circle, so that
// quarter turns are exact.
blink_status fft_constants(int N) {
    if (N != 512) return BLINK_OK;
    float2 t[512], rt[kW * kRowTw] = {};
    for (int m = 0; m < 512; m++) {
        const int q = m / 128, k = m % 128;
        double c = 1.0, s = 0.0;
        if (k) {
            const double a = 2.0 * 3.14159265358979323846 * k / 512.0;
            c = std::cos(a);
            s = std::sin(a);
        }
        const double x = q == 0 ? c : q == 1 ? -s : q == 2 ? -c : s;
        const double y = q == 0 ? s : q == 1 ? c : q == 2 ? -s : -c;
        t[m] = make_float2((float)x, (float)y);
    }
    for (int w = 0; w < kW; w++) {
        const int jA = w == 0 ? 0 : w, jB = w == 0 ? 8 : 16 - w;
        float2* r = rt + w * kRowTw;
        for (int q = 0; q < 9; q++) r[q] = w == 0 ? t[16 * q] : (q < 8 ? t[jA + 16 * q] : make_float2(0.f, 0.f));
        for (int q = 0; q < 8; q++) r[9 + q] = t[jB + 16 * q];
        for (int k1 = 1; k1 < 16; k1++) {
            r[17 + k1 - 1] = t[(2 * jA * k1) & 511];
            r[32 + k1 - 1] = t[(2 * jB * k1) & 511];
        }
    }
    BLINK_CUDA(cudaMemcpyToSymbol(c_rowtw512, rt, sizeof(rt)));
    return BLINK_OK;
}

blink_status launch_fft_persistent(const Plan& p, const FftTune& tune, int prec, const float2* d_vis,
                                   int64_t vis_stride, int vis_first, int tau0, int n_tau, void* d_H, int* d_counters,
                                   float* d_img, int out_first, int* d_status, int n_sm, cudaStream_t st,
                                   const FftWait& wait, bool gathered, const FusedIn* fused) {
    if (gathered && !fft_takes_gathered(p))
        return set_error(BLINK_ERR_UNSUPPORTED, "gather-ordered sums need a nearest-cell plan of side 256 to 1024");
    FftParams P{};
    if (fused) {
        if (!gathered || !fft_fused_ok(p, fused->ns, fused->kind, fused->d_volt, fused->sample_stride) || !fused->d_vring)
            return set_error(BLINK_ERR_UNSUPPORTED, "the fused imaging launch does not support this request");
        const FusedChunk c = fused_chunk(p, fused->ns, fused->kind);
        P.fused = 1;
        P.volt = fused->d_volt;
        P.sample_stride = fused->sample_stride;
        P.ns = fused->ns;
        P.cavg = p.chan_avg;
        P.n_tiles = p.n_tiles;
        P.ns_c = c.ns_c;
        P.n_chunks = c.n_chunks;
        P.Kq = c.Kq;
        P.Kp = c.Kp;
        P.n_blk = c.n_blk;
        P.stokes = fused->kind == CORR_OUT_STOKES_I ? 1 : 0;
        P.gpos = p.d_gpos;
        P.B = p.B;
        P.flags = p.d_flags;
        P.vring = fused->d_vring;
        P.ring_v = kRingV;
        P.lead = kLead;
    }
    P.gathered = gathered ? 1 : 0;
    P.e_stride = p.e_stride;
    P.wait_budget = wait.budget > 0 ? wait.budget : 1;
    P.extra_wait = wait.extra;
    P.vis = d_vis;
    P.vis_stride = vis_stride;
    P.vis_first = vis_first;
    {
        const uint64_t bytes = gathered ? (uint64_t)p.e_stride * sizeof(float2) : (uint64_t)p.B * sizeof(float2);
        const bool ok = bytes % 16 == 0 && (vis_stride * sizeof(float2)) % 16 == 0 &&
                        reinterpret_cast<uintptr_t>(d_vis) % 16 == 0 && bytes < (1ull << 31);
        P.vis_prefetch = ok ? (uint32_t)bytes : 0u;
    }
    P.F = p.F;
    P.tau0 = tau0;
    P.n_tau = n_tau;
    P.n_img = p.F * n_tau;
    P.ent_off = p.d_ent_off;
    P.ent = p.d_ent;
    P.tw = p.d_tw;
    P.H = d_H;
    P.ldh = p.N / 2;
    P.ring = std::min(tune.ring, fft_ring_images_max());
    P.lag = std::min(tune.lag, P.ring);
    P.wk = p.d_Wk;
    P.img_out = d_img;
    P.out_first = out_first;
    P.tickets = d_counters;
    P.col_done = d_counters + 2;
    P.row_done = d_counters + 2 + P.n_img;
    P.corr_done = fused ? d_counters + 2 + 2 * (int64_t)P.n_img : nullptr;
    P.status = d_status;
    if (fused) P.vis_prefetch = 0;
    BLINK_CUDA(cudaMemsetAsync(d_counters, 0, sizeof(int) * (2 + (fused ? 3 : 2) * (size_t)P.n_img), st));
    const bool bf = prec == BLINK_PREC_BF16, wt = p.d_wt != nullptr;
    P.wt = p.d_wt;
    P.corr = p.d_corr;
    if (wt && !bf && p.d_sep) {
        P.sep_off = p.d_sep_off;
        P.sep = p.d_sep;
        P.sep_w = p.d_sep_w;
        P.sep_W = p.support;
    }
    if (wt && (!p.d_corr || p.N < 128))
        return set_error(BLINK_ERR_UNSUPPORTED, "convolutional gridding needs a grid side of at least 128");
    const int c = tune.ctas_per_sm;
    switch (p.N) {
        case 64: return bf ? launch_sized<64, __nv_bfloat162, false>(P, n_sm, c, st) : launch_sized<64, float2, false>(P, n_sm, c, st);
#define BLINK_FFT_CASE(NN)                                                                                  \
        case NN:                                                                                            \
            if (wt) return bf ? launch_sized<NN, __nv_bfloat162, true>(P, n_sm, c, st) : launch_sized<NN, float2, true>(P, n_sm, c, st); \
            return bf ? launch_sized<NN, __nv_bfloat162, false>(P, n_sm, c, st) : launch_sized<NN, float2, false>(P, n_sm, c, st);
        BLINK_FFT_CASE(128)
        BLINK_FFT_CASE(256)
        BLINK_FFT_CASE(512)
        BLINK_FFT_CASE(1024)
        BLINK_FFT_CASE(2048)
#undef BLINK_FFT_CASE
    }
    return set_error(BLINK_ERR_UNSUPPORTED, "image side must be a power of two in [64, 2048]");
}

}  // namespace blink
