// Correlation on the tcgen05 tensor cores (Eq. 2; Sec. 5.2.2) with FP8 e4m3 operands and FP32
// accumulation in tensor memory.
//
// Every 4-bit component is an integer in [-8, 7] (and its negation in [-7, 8]), all exact in e4m3, and
// each product and partial sum is an integer below 2^24, so the tensor-core result equals the integer
// correlation bit for bit.
//
// The complex product is realified.  With x_u in C^K for a unit u (a tile, or a tile and polarisation),
//   P_u = [Re x_u, Im x_u],   Q_u = [Im x_u, -Re x_u]     (length 2K bytes each)
//   Re S_uv = P_u . P_v,       Im S_uv = Q_u . P_v,        S_uv = sum_k x_u[k] conj(x_v[k]).
// Units are grouped in blocks of 64.  The A operand of block m is the 128 rows [P of its 64 units;
// Q of its 64 units]; the B operand of block n is the 64 P rows of block n.  One M=128, N=64 MMA chain
// over K gives Re S (TMEM lanes 0-63) and Im S (lanes 64-127) for the 64 x 64 units of the block pair.
// Only block pairs n <= m are computed (the lower triangle).  For Stokes I the two polarisations are
// concatenated along K (units = tiles, K' = 2K), which sums S_XX + S_YY inside the MMA.
//
// Per CTA (persistent, one per SM): TMA loads an item's raw voltage block (double buffered), all
// threads unpack nibbles to e4m3 operand tiles in shared memory (K-major, no swizzle, 8x16-byte core
// matrices), one thread issues the MMAs and commits them to an mbarrier, and the 16 warps read the
// accumulators back from TMEM (four warps per 32-lane quarter, 16 columns each), stage them in shared memory
// (two buffers: the next block pair is staged while the previous one is written) and write the visibilities.  Every wait is bounded; on expiry the CTA records BLINK_ERR_TIMEOUT, waits (bounded) for
// its own copies, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "blink_internal.cuh"
#include "tc_ptx.cuh"

namespace blink {

namespace {

constexpr int kThreads = 512;                   // 16 warps: four per TMEM lane quarter
constexpr int kGatherIlp = 16;                  // gather-order pass: entries per thread in flight
constexpr int kUnitsPerBlk = 64;
constexpr int kTmemCols = 512;
constexpr int kStageLd = 65;                     // padded row of the epilogue staging tiles (floats)
constexpr int kPlane = 64 * kStageLd;            // floats of one staging plane (64 x 64 values, padded rows)
constexpr int kHalfLd = 33;                      // padded row of the half-pair staging (calibrated, gather order)
constexpr long long kWaitBudget = 2000000000ll;  // clock cycles (about a second)

struct TcParams {
    int mode;                // CORR_OUT_*
    int n_tiles, ns, c, F, K;
    int ns_c, n_chunks;      // K streams through the operand tiles in chunks of ns_c samples (ns_c * c values)
    int Kq;                  // a chunk's K rounded up to a multiple of 4 (one 32-bit word of e4m3 values)
    int units, n_blk, Kr, Kp;
    int n_pairs, n_rounds;
    int split;               // Stokes I with gains: XX and YY from separate MMA chains (per-polarisation K halves)
    int Kpol;                // split: bytes of one polarisation's part of an operand row (a multiple of 32)
    int pair_cols, pairs_per_round;   // TMEM columns per block pair (64, or 128 when split) and pairs per round
    int stage_buf;           // floats per staging buffer: 2 planes (re, im), or 4 (re, im of XX, then of YY)
    int two_stage;           // two epilogue staging buffers (else one)
    const float2* gains;     // calibration gains [channels][n_tiles][2 pol] or NULL; item channel f uses row gain_f0 + f
    int gain_f0;
    uint32_t off_gain;       // shared copy of the current item's gains [n_tiles][2]
    int first_item, n_items;
    int raw_bytes;
    uint32_t off_raw0, off_raw1, off_re, off_im, off_lut, off_flags, off_bar, off_tmem;
    const uint8_t* flags;
    void* out;
    int64_t out_item_stride;
    int* status;
    int64_t B;
    ImgOut io;               // imaging kinds in baseline order: phase-centre factor
    // imaging kinds in gather order: the item's sums go from TMEM to a baseline-ordered copy in shared memory
    // (planes re | im of B floats at off_item), then leave in gather order (p -> baseline gsrc[f][p])
    int gathered;            // 0: baseline order
    int overlay;             // the item's copy shares the operand tiles' space (set by tc_chunk)
    uint32_t off_item;       // (0 when the copy shares the operand tiles' space)
    const uint16_t* gsrc;
    const float2* gphase;
    const int* ent_off;      // [F][ent_ld]: entry range of each channel (last column's end = its count)
    int ent_ld, e_stride;
};

// One imaging-kind sum of item `local` (channel f) and baseline b in baseline order, times the phase-centre
// factor when given.  The factor is fetched first (img_fetch), so that a thread's fetches for several
// baselines are in flight together.
__device__ __forceinline__ float2 img_fetch(const TcParams& P, int f, int64_t b) {
    return P.io.phase ? __ldg(P.io.phase + (int64_t)f * P.B + b) : make_float2(1.f, 0.f);
}
__device__ __forceinline__ void put_img(const TcParams& P, int local, int64_t b, float2 ph, float re, float im) {
    if (P.io.phase) {
        const float r = re * ph.x - im * ph.y, i = re * ph.y + im * ph.x;
        re = r;
        im = i;
    }
    static_cast<float2*>(P.out)[(int64_t)local * P.out_item_stride + b] = make_float2(re, im);
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// CAL: 0 uncalibrated; 1 diagonal gains applied in the epilogue (Stokes I through split X / Y chains); 2 full
// 2x2 Jones matrices, which need all four products, so every output kind runs the four-product layout and the
// epilogue forms J_i S J_j^H.  Each is a separate instantiation.
template <int CAL>
__global__ void __launch_bounds__(kThreads, 1) k_corr_tc(const __grid_constant__ CUtensorMap tmap, const TcParams P) {
    constexpr bool GAINS = CAL > 0, FULL = CAL == 2;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* ops = smem;                                   // n_blk tiles of 128 x Kp bytes
    float* st_re = reinterpret_cast<float*>(smem + P.off_re);   // plane 0 of buffer 0; planes kPlane apart
    float* st_im = reinterpret_cast<float*>(smem + P.off_im);
    float2* s_g = reinterpret_cast<float2*>(smem + P.off_gain);
    uint32_t* lut = reinterpret_cast<uint32_t*>(smem + P.off_lut);   // raw byte -> e4m3 (re, im, im, -re)
    uint8_t* sflags = smem + P.off_flags;
    float* s_item = P.gathered ? reinterpret_cast<float*>(smem + P.off_item) : nullptr;
    const uint32_t bar_tma0 = smem_u32(smem + P.off_bar), bar_tma1 = bar_tma0 + 8, bar_mma = bar_tma0 + 16;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + P.off_tmem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (smem_u32(smem) & 1023) {                          // descriptors and TMA need an aligned base
        if (tid == 0) atomicOr(P.status, DEV_ERR_INDEX);
        return;
    }

    if (tid == 0) {
        mbar_init(bar_tma0, 1);
        mbar_init(bar_tma1, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    {
        // e4m3 of v in [-8, 8]: 0, 1, 2, ..., 8 encoded, the sign bit 0x80 for negatives
        const uint32_t pos[9] = {0x00, 0x38, 0x40, 0x44, 0x48, 0x4A, 0x4C, 0x4E, 0x50};
        auto e4m3 = [&](int v) -> uint32_t { return v >= 0 ? pos[v] : (0x80u | pos[-v]); };
        for (int b = tid; b < 256; b += kThreads) {
            const int re = (b & 15) >= 8 ? (b & 15) - 16 : (b & 15);
            const int im = (b >> 4) >= 8 ? (b >> 4) - 16 : (b >> 4);
            lut[b] = e4m3(re) | (e4m3(im) << 8) | (e4m3(im) << 16) | (e4m3(-re) << 24);
        }
        for (int a = tid; a < P.n_tiles; a += kThreads) sflags[a] = P.flags[a] ? 1 : 0;
    }
    {
        uint4* z = reinterpret_cast<uint4*>(ops);
        const int n16 = P.n_blk * 128 * P.Kp / 16;
        for (int e = tid; e < n16; e += kThreads) z[e] = make_uint4(0, 0, 0, 0);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const uint32_t ops_s = smem_u32(ops);
    const uint32_t raw_s[2] = {smem_u32(smem + P.off_raw0), smem_u32(smem + P.off_raw1)};
    const uint32_t bar_tma[2] = {bar_tma0, bar_tma1};
    uint32_t tma_par[2] = {0, 0}, mma_par = 0;
    bool pending[2] = {false, false};
    bool abort = false;
    const int total = P.first_item + P.n_items;
    const uint32_t sbo = (uint32_t)P.Kp * 8, tile_bytes = 128u * P.Kp;
    const uint32_t idesc = idesc_e4m3(128, 64);
    const float div = (float)(P.mode == CORR_OUT_STOKES_I ? 2 * P.K : P.K);
    const int per_k = 2 * P.n_tiles;

    // chunk j of an item: samples [j ns_c, j ns_c + ns_c) of its integration (the last chunk's excess is masked)
    auto issue = [&](int item, int j, int b) {
        const int tau = item / P.F, f = item - (item / P.F) * P.F;
        mbar_expect_tx(bar_tma[b], (uint32_t)P.raw_bytes);
        tma_load_3d(raw_s[b], &tmap, bar_tma[b], 0, f * P.c, tau * P.ns + j * P.ns_c);
    };
    // Steps: one per item when K fits one chunk (its TMEM rounds share the operands); else one per (item,
    // round, chunk), each round re-streaming K and accumulating its block pairs in TMEM across the chunks.
    auto advance = [&](int& i, int& r, int& j) {
        if (++j < P.n_chunks) return;
        j = 0;
        if (P.n_chunks > 1 && ++r < P.n_rounds) return;
        r = 0;
        i += gridDim.x;
    };

    int ci = P.first_item + blockIdx.x, cr = 0, cj = 0;
    if (tid == 0 && ci < total) issue(ci, 0, 0);
    pending[0] = ci < total;
    for (int buf = 0; ci < total; buf ^= 1) {
        const int it = ci;
        int ni = ci, nr = cr, nj = cj;
        advance(ni, nr, nj);
        if (ni < total) {
            if (tid == 0) issue(ni, nj, buf ^ 1);
            pending[buf ^ 1] = true;
        }
        const bool first_chunk = cj == 0, last_chunk = cj == P.n_chunks - 1;
        const int Kv = min(P.ns_c, P.ns - cj * P.ns_c) * P.c;     // values of this chunk inside the item
        const bool ok = mbar_wait(bar_tma[buf], tma_par[buf], kWaitBudget);
        tma_par[buf] ^= 1;
        pending[buf] = !ok;
        if (__syncthreads_or(!ok)) {
            abort = true;
            break;
        }
        if (GAINS && cr == 0 && first_chunk) {
            // this item's gains, read by the epilogue (after the barrier that ends the unpack)
            const int f = it - (it / P.F) * P.F;
            const int per = FULL ? 4 : 2;                        // float2 per tile: J[p][r], or g[p]
            const float2* g = P.gains + (int64_t)(P.gain_f0 + f) * P.n_tiles * per;
            for (int e = tid; e < per * P.n_tiles; e += kThreads) s_g[e] = g[e];
        }
        // ---- unpack nibbles to e4m3 operand rows, four consecutive k per 32-bit store -----------------
        // A task is (k group g, tile a, polarisation p): its four raw bytes give, through the LUT, the words
        // P_re, P_im (= Q_im) and Q_-re of four consecutive K positions of one unit row.
        const uint8_t* raw = smem + (buf ? P.off_raw1 : P.off_raw0);
        const int n_groups = P.Kq >> 2;
        // (group, row) tasks over all threads: a short K has fewer rows (2 n_tiles) than the CTA has threads
        for (int e = tid; e < n_groups * per_k; e += kThreads) {
            const int g = e / per_k, r = e - g * per_k;
            const int k0 = 4 * g;
            const int a = r >> 1, p = r & 1;
            int unit, kp, kh;
            if (GAINS && P.mode == CORR_OUT_STOKES_I && P.split) {
                unit = a; kp = p * P.Kpol + k0; kh = P.Kq;          // [re, im] of X, then of Y
            } else if (P.mode == CORR_OUT_STOKES_I && !FULL) {
                unit = a; kp = p * P.Kq + k0; kh = 2 * P.Kq;        // re X, re Y, im X, im Y
            } else if (P.mode == CORR_OUT_VIS4 || FULL) {
                unit = 2 * a + p; kp = k0; kh = P.Kq;
            } else {
                if (p) continue;
                unit = a; kp = k0; kh = P.Kq;
            }
            // a flagged tile's operand rows are zero, so every product involving it is exactly zero
            const bool live = !sflags[a];
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; i++) w[i] = (live && k0 + i < Kv) ? lut[raw[(k0 + i) * per_k + r]] : 0u;
            const uint32_t re = __byte_perm(__byte_perm(w[0], w[1], 0x0040), __byte_perm(w[2], w[3], 0x0040), 0x5410);
            const uint32_t im = __byte_perm(__byte_perm(w[0], w[1], 0x0051), __byte_perm(w[2], w[3], 0x0051), 0x5410);
            const uint32_t nre = __byte_perm(__byte_perm(w[0], w[1], 0x0073), __byte_perm(w[2], w[3], 0x0073), 0x5410);
            uint8_t* tile = ops + (unit >> 6) * tile_bytes;
            const int row = unit & 63;
            *reinterpret_cast<uint32_t*>(tile + op_off(row, kp, P.Kp)) = re;
            *reinterpret_cast<uint32_t*>(tile + op_off(row, kp + kh, P.Kp)) = im;
            *reinterpret_cast<uint32_t*>(tile + op_off(row + 64, kp, P.Kp)) = im;
            *reinterpret_cast<uint32_t*>(tile + op_off(row + 64, kp + kh, P.Kp)) = nre;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        // ---- MMA rounds of up to 8 block pairs, each followed (after the item's last chunk) by its epilogue -
        const int r_lo = P.n_chunks > 1 ? cr : 0, r_hi = P.n_chunks > 1 ? cr + 1 : P.n_rounds;
        for (int r = r_lo; r < r_hi && !abort; r++) {
            const int ppr = GAINS ? P.pairs_per_round : kTmemCols / 64;
            const int q0 = r * ppr, q1 = min(P.n_pairs, q0 + ppr);
            if (tid == 0) {
                tc_fence_after();
                const int nk = P.Kp / 32, nh = GAINS && P.split ? nk / 2 : nk;
                for (int q = q0; q < q1; q++) {
                    int mb, jb;
                    pair_of(q, mb, jb);
                    const uint32_t d = tmem + (uint32_t)((q - q0) * (GAINS ? P.pair_cols : 64));
                    const uint32_t a0 = ops_s + mb * tile_bytes, b0 = ops_s + jb * tile_bytes;
                    // one chain over all of K, or (split) the X half into columns 0-63 and the Y half into 64-127
                    for (int s = 0; s < nk; s++)
                        mma_e4m3(GAINS && s >= nh ? d + 64 : d, smem_desc(a0 + s * 256, 128, sbo),
                                 smem_desc(b0 + s * 256, 128, sbo), idesc,
                                 !first_chunk || (GAINS ? s % nh > 0 : s > 0));
                }
                mma_commit(bar_mma);
            }
            const bool okm = mbar_wait(bar_mma, mma_par, kWaitBudget);
            mma_par ^= 1;
            if (__syncthreads_or(!okm)) {
                abort = true;
                break;
            }
            tc_fence_after();
            if (!last_chunk) {                     // the accumulators go on with the next chunk
                tc_fence_before();
                __syncthreads();
                continue;
            }
            const int local = it - P.first_item;
            if (GAINS && !FULL && s_item) {
                // calibrated, gather order: each block pair in two halves of 32 columns, staged from TMEM (Re and Im
                // of a unit row sit in TMEM lanes 64 apart, so in different warps) and combined into the item's
                // copy as g_i S conj(g_j) (summed over X and Y for Stokes I); the gather pass below writes it out
                float* hs = reinterpret_cast<float*>(smem + P.off_re);   // planes [XX re, XX im, YY re, YY im]
                for (int q = q0; q < q1; q++) {
                    int mb, jb;
                    pair_of(q, mb, jb);
                    for (int h = 0; h < 2; h++) {
                        {
                            const int row = (warp & 3) * 32 + lane, g = warp >> 2;
                            const uint32_t ta = tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                                                (uint32_t)((q - q0) * P.pair_cols + 32 * h + 8 * g);
                            float* st = hs + (row >> 6) * 64 * kHalfLd + (row & 63) * kHalfLd + 8 * g;
                            uint32_t v[8];
                            tmem_ld8(ta, v);
#pragma unroll
                            for (int cc = 0; cc < 8; cc++) st[cc] = __uint_as_float(v[cc]);
                            if (P.split) {                     // YY: planes 2 and 3
                                tmem_ld8(ta + 64, v);
#pragma unroll
                                for (int cc = 0; cc < 8; cc++) st[2 * 64 * kHalfLd + cc] = __uint_as_float(v[cc]);
                            }
                        }
                        __syncthreads();
                        for (int e = tid; e < 64 * 32; e += kThreads) {
                            const int il = e >> 5, jl = e & 31;
                            const int ui = mb * 64 + il, uj = jb * 64 + 32 * h + jl;
                            if (ui >= P.n_tiles || uj > ui) continue;
                            const float2 gx = s_g[2 * ui], hx = s_g[2 * uj];
                            float sr = hs[il * kHalfLd + jl], si = hs[64 * kHalfLd + il * kHalfLd + jl];
                            float tr = gx.x * sr - gx.y * si, ti = gx.x * si + gx.y * sr;
                            float vr = tr * hx.x + ti * hx.y, vi = ti * hx.x - tr * hx.y;
                            if (P.split) {
                                const float2 gy = s_g[2 * ui + 1], hy = s_g[2 * uj + 1];
                                sr = hs[2 * 64 * kHalfLd + il * kHalfLd + jl];
                                si = hs[3 * 64 * kHalfLd + il * kHalfLd + jl];
                                tr = gy.x * sr - gy.y * si;
                                ti = gy.x * si + gy.y * sr;
                                vr += tr * hy.x + ti * hy.y;
                                vi += ti * hy.x - tr * hy.y;
                            }
                            const int64_t b = (int64_t)ui * (ui + 1) / 2 + uj;
                            s_item[b] = vr;
                            s_item[P.B + b] = vi;
                        }
                        __syncthreads();
                    }
                }
                tc_fence_before();
                __syncthreads();
                continue;
            }
            if (!GAINS && s_item) {
                // gather order: every block pair of the round from TMEM straight into the item's copy (warp w reads
                // TMEM lanes 32 (w % 4) + lane = unit row, re for lanes below 64, im above; columns 16 (w / 4) ..)
                for (int q = q0; q < q1; q++) {
                    int mb, jb;
                    pair_of(q, mb, jb);
                    const int row = (warp & 3) * 32 + lane, c0 = (warp >> 2) * 16;
                    uint32_t v[16];
                    tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((q - q0) * 64) + c0, v);
                    const int ui = mb * 64 + (row & 63);
                    if (ui < P.n_tiles) {
                        float* dst = s_item + (row >> 6) * P.B + (int64_t)ui * (ui + 1) / 2;
#pragma unroll
                        for (int cc = 0; cc < 16; cc++) {
                            const int uj = jb * 64 + c0 + cc;
                            if (uj <= ui) dst[uj] = __uint_as_float(v[cc]);
                        }
                    }
                }
                tc_fence_before();
                __syncthreads();
                continue;
            }
            const int stage_buf = GAINS ? P.stage_buf : 2 * kPlane;
            // stage block pair q into buffer sb: warp w reads TMEM lanes 32 (w % 4) + lane, columns 16 (w / 4) ..
            auto stage = [&](int q, int sb) {
                const int row = (warp & 3) * 32 + lane, c0 = (warp >> 2) * 16;
                float* st = (row < 64 ? st_re + row * kStageLd : st_im + (row - 64) * kStageLd) + sb * stage_buf;
                const uint32_t ta = tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                                    (uint32_t)((q - q0) * (GAINS ? P.pair_cols : 64)) + c0;
                uint32_t v[16];
                tmem_ld16(ta, v);
#pragma unroll
                for (int cc = 0; cc < 16; cc++) st[c0 + cc] = __uint_as_float(v[cc]);
                if (GAINS && P.split) {                        // YY: planes 2 and 3
                    tmem_ld16(ta + 64, v);
#pragma unroll
                    for (int cc = 0; cc < 16; cc++) st[2 * kPlane + c0 + cc] = __uint_as_float(v[cc]);
                }
            };
            // write block pair q from buffer sb
            auto write = [&](int q, int sb) {
                int mb, jb;
                pair_of(q, mb, jb);
                const float* sre = st_re + sb * stage_buf;
                const float* sim = st_im + sb * stage_buf;
                if (FULL) {
                    // tile pairs of this unit block pair (units 2 tile + pol): V = J_i S J_j^H from the four
                    // staged products of each pair; VIS4 writes all four / K, the imaging kinds XX (+ YY)
                    for (int e = tid; e < 32 * 32; e += kThreads) {
                        const int il = e >> 5, jl = e & 31;
                        const int ti = mb * 32 + il, tj = jb * 32 + jl;
                        if (ti >= P.n_tiles || tj > ti) continue;
                        const float2* Ji = s_g + 4 * ti;
                        const float2* Jj = s_g + 4 * tj;
                        float2 S[4];
#pragma unroll
                        for (int rs = 0; rs < 4; rs++) {
                            const int o = (2 * il + (rs >> 1)) * kStageLd + 2 * jl + (rs & 1);
                            S[rs] = make_float2(sre[o], sim[o]);
                        }
                        float2 V[4];
#pragma unroll
                        for (int pq = 0; pq < 4; pq++) {
                            const int pp = pq >> 1, qq = pq & 1;
                            float vr = 0.f, vi = 0.f;
#pragma unroll
                            for (int rs = 0; rs < 4; rs++) {
                                const float2 a = Ji[2 * pp + (rs >> 1)], c = Jj[2 * qq + (rs & 1)];
                                const float tr = a.x * S[rs].x - a.y * S[rs].y, tim = a.x * S[rs].y + a.y * S[rs].x;
                                vr += tr * c.x + tim * c.y;
                                vi += tim * c.x - tr * c.y;
                            }
                            V[pq] = make_float2(vr, vi);
                        }
                        const int64_t b = (int64_t)ti * (ti + 1) / 2 + tj;
                        if (P.mode == CORR_OUT_VIS4) {
                            float2* o = reinterpret_cast<float2*>(static_cast<float*>(P.out) +
                                                                  (int64_t)local * P.out_item_stride) + b * 4;
#pragma unroll
                            for (int pq = 0; pq < 4; pq++)
                                o[pq] = make_float2(__fdiv_rn(V[pq].x, div), __fdiv_rn(V[pq].y, div));
                        } else {
                            const float2 o = P.mode == CORR_OUT_STOKES_I ? make_float2(V[0].x + V[3].x, V[0].y + V[3].y) : V[0];
                            if (s_item) {                       // gather order: into the item's copy
                                s_item[b] = o.x;
                                s_item[P.B + b] = o.y;
                            } else {
                                put_img(P, local, b, img_fetch(P, it % P.F, b), o.x, o.y);
                            }
                        }
                    }
                    return;
                }
                // (flagged tiles need no test: their operand rows were zeroed in the unpack)
                if (P.mode == CORR_OUT_VIS4) {
                    for (int e = tid; e < 64 * 64; e += kThreads) {
                        const int il = e >> 6, jl = e & 63;
                        const int ui = mb * 64 + il, uj = jb * 64 + jl;
                        if (ui >= P.units) continue;
                        const int ai = ui >> 1, aj = uj >> 1;
                        if (aj > ai) continue;
                        float re = sre[il * kStageLd + jl], im = sim[il * kStageLd + jl];
                        if (GAINS) {                           // g_i^p S conj(g_j^q), unit u = 2 tile + pol
                            const float2 gi = s_g[ui], gj = s_g[uj];
                            const float tr = gi.x * re - gi.y * im, ti = gi.x * im + gi.y * re;
                            re = tr * gj.x + ti * gj.y;
                            im = ti * gj.x - tr * gj.y;
                        }
                        const int64_t b = (int64_t)ai * (ai + 1) / 2 + aj;
                        float* o = static_cast<float*>(P.out) + (int64_t)local * P.out_item_stride +
                                   (b * 4 + 2 * (ui & 1) + (uj & 1)) * 2;
                        *reinterpret_cast<float2*>(o) = make_float2(__fdiv_rn(re, div), __fdiv_rn(im, div));
                    }
                } else {
                    // imaging kinds: the exact integer sums (the 1/K or 1/2K is applied with 1/W).  Each thread
                    // keeps one column jl and steps down the rows, so consecutive lanes write consecutive
                    // baselines of a row.
                    constexpr int kRowStep = kThreads / 64;
                    const int jl = tid & 63, uj = jb * 64 + jl;
                    const int fch = it % P.F;
                    const float* pre = sre + jl;
                    const float* pim = sim + jl;
                    if (!GAINS) {
                        // the rows il = tid / 64 + kRowStep r: their baselines' data fetched together, then stored
                        constexpr int kR = 64 / kRowStep;
                        float2 ax[kR];
#pragma unroll
                        for (int r = 0; r < kR; r++) {
                            const int il = (tid >> 6) + kRowStep * r, ui = mb * 64 + il;
                            ax[r] = (ui < P.n_tiles && uj <= ui) ? img_fetch(P, fch, (int64_t)ui * (ui + 1) / 2 + uj)
                                                                 : make_float2(1.f, 0.f);
                        }
#pragma unroll
                        for (int r = 0; r < kR; r++) {
                            const int il = (tid >> 6) + kRowStep * r, ui = mb * 64 + il;
                            if (ui >= P.n_tiles || uj > ui) continue;
                            put_img(P, local, (int64_t)ui * (ui + 1) / 2 + uj, ax[r], pre[il * kStageLd],
                                    pim[il * kStageLd]);
                        }
                    } else {
                        // calibrated: g_i^X S_XX conj(g_j^X) (+ g_i^Y S_YY conj(g_j^Y) for Stokes I, split)
                        const int ujc = uj < P.n_tiles ? uj : 0;
                        const float2 hx = s_g[2 * ujc], hy = s_g[2 * ujc + 1];
                        for (int il = tid >> 6; il < 64; il += kRowStep) {
                            const int ui = mb * 64 + il;
                            if (ui >= P.n_tiles || uj > ui) continue;
                            const float2 gx = s_g[2 * ui];
                            float sr = pre[il * kStageLd], si = pim[il * kStageLd];
                            float tr = gx.x * sr - gx.y * si, ti = gx.x * si + gx.y * sr;
                            float vr = tr * hx.x + ti * hx.y, vi = ti * hx.x - tr * hx.y;
                            if (P.split) {
                                const float2 gy = s_g[2 * ui + 1];
                                sr = pre[2 * kPlane + il * kStageLd];
                                si = pim[2 * kPlane + il * kStageLd];
                                tr = gy.x * sr - gy.y * si;
                                ti = gy.x * si + gy.y * sr;
                                vr += tr * hy.x + ti * hy.y;
                                vi += ti * hy.x - tr * hy.y;
                            }
                            const int64_t b = (int64_t)ui * (ui + 1) / 2 + uj;
                            put_img(P, local, b, img_fetch(P, fch, b), vr, vi);
                        }
                    }
                }
            };
            if (P.two_stage) {
                stage(q0, 0);
                __syncthreads();
                for (int q = q0; q < q1; q++) {
                    if (q + 1 < q1) stage(q + 1, (q + 1 - q0) & 1);
                    write(q, (q - q0) & 1);
                    __syncthreads();
                }
            } else {
                for (int q = q0; q < q1; q++) {
                    stage(q, 0);
                    __syncthreads();
                    write(q, 0);
                    __syncthreads();
                }
            }
            tc_fence_before();
            __syncthreads();
        }
        if (abort) break;
        ci = ni;
        cr = nr;
        cj = nj;
        if (s_item && last_chunk && (P.n_chunks == 1 || r_lo == P.n_rounds - 1)) {
            // the item in gather order: entry p of channel f takes baseline gsrc[f][p] (times the factor
            // gphase[f][p] off zenith), kGatherIlp entries per thread in flight (a 144-tile item's 10,440
            // entries in two round trips), coalesced stores of both planes
            const int f = it % P.F;
            const int* eo = P.ent_off + (int64_t)f * P.ent_ld;
            const int n_f = eo[P.ent_ld - 1] - eo[0];
            const uint16_t* src = P.gsrc + (int64_t)f * P.e_stride;
            const float2* gph = P.gphase ? P.gphase + (int64_t)f * P.e_stride : nullptr;
            float* o = static_cast<float*>(P.out) + (int64_t)(it - P.first_item) * 2 * P.e_stride;
            for (int p0 = tid; p0 < n_f; p0 += kGatherIlp * kThreads) {
                uint32_t bb[kGatherIlp];
                float2 w[kGatherIlp];
#pragma unroll
                for (int k = 0; k < kGatherIlp; k++) {
                    const int pp = p0 + k * kThreads;
                    bb[k] = pp < n_f ? __ldg(src + pp) : 0u;
                    w[k] = (gph && pp < n_f) ? __ldg(gph + pp) : make_float2(1.f, 0.f);
                }
#pragma unroll
                for (int k = 0; k < kGatherIlp; k++) {
                    const int pp = p0 + k * kThreads;
                    if (pp >= n_f) break;
                    float re = s_item[bb[k]], im = s_item[P.B + bb[k]];
                    if (gph) {
                        const float r = re * w[k].x - im * w[k].y, i = re * w[k].y + im * w[k].x;
                        re = r;
                        im = i;
                    }
                    o[pp] = re;
                    o[P.e_stride + pp] = im;
                }
            }
            if (P.overlay) {
                // the copy lay over the operand tiles: zero them again for the next item (the unpack writes only
                // the live rows and K positions)
                __syncthreads();
                uint4* z = reinterpret_cast<uint4*>(smem);
                const int n16 = (int)((2 * P.B * sizeof(float) + 15) / 16);
                for (int e = tid; e < n16; e += kThreads) z[e] = make_uint4(0, 0, 0, 0);
            }
        }
    }
    if (abort) {
        if (tid == 0) {
            atomicOr(P.status, DEV_ERR_TIMEOUT);
            for (int b = 0; b < 2; b++)
                if (pending[b]) mbar_wait(bar_tma[b], tma_par[b], kWaitBudget);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// Shared-memory layout of a launch whose chunks hold ns_c samples: operand tiles for the chunk's K, two raw
// chunks (TMA, double buffered), the epilogue's staging buffers or the item's baseline-ordered copy (gather
// order), gains, LUT, flags, barriers.  Fills the chunk-dependent fields of P; returns the bytes needed.
size_t tc_layout(TcParams& P, int ns_c, bool gather, GainRef gains, int64_t B) {
    const int nt = P.n_tiles;
    const int Kc = ns_c * P.c;
    P.ns_c = ns_c;
    P.n_chunks = (P.ns + ns_c - 1) / ns_c;
    P.Kq = (Kc + 3) / 4 * 4;
    P.Kpol = (2 * P.Kq + 31) / 32 * 32;
    const bool four = P.units == 2 * nt;
    P.Kr = (P.mode == CORR_OUT_STOKES_I && !four) ? 4 * P.Kq : 2 * P.Kq;
    P.Kp = P.split ? 2 * P.Kpol : (P.Kr + 31) / 32 * 32;
    P.raw_bytes = ns_c * P.c * nt * 2;
    // P.overlay (gather order, one round of block pairs, chosen by tc_chunk when K does not fit otherwise): the
    // item's baseline-ordered copy is written only after the item's last MMAs have completed and read before
    // the next item's unpack, so it can share the operand tiles' space (longer chunks: fewer barriers per item);
    // the kernel zeroes that space again after reading the copy, since the unpack never writes the tiles'
    // padding
    const bool overlay = gather && P.n_rounds == 1 && P.overlay;
    const uint32_t ops_bytes = (uint32_t)P.n_blk * 128u * P.Kp;
    uint32_t off = align_up(overlay ? std::max(ops_bytes, (uint32_t)(8 * B)) : ops_bytes, 1024);
    P.off_raw0 = off;
    off = align_up(off + P.raw_bytes, 128);
    P.off_raw1 = off;
    off = align_up(off + P.raw_bytes, 128);
    P.off_re = off;                                // buffer b: planes from off_re + b * stage_buf, kPlane apart
    P.off_im = off + kPlane * 4;
    const uint32_t gain_bytes = gains.d ? (uint32_t)nt * (gains.full ? 32 : 16) : 0;
    const uint32_t tail = 256 * 4 + align_up((uint32_t)nt, 16) + 32 + (gains.d ? gain_bytes + 16 : 0);
    P.off_item = 0;
    P.gathered = gather ? 1 : 0;
    if (overlay) {
        P.off_item = 0;
        P.two_stage = 0;
        if (gains.d) {                             // the calibrated epilogue's staging
            P.off_re = off;
            P.off_im = off + kPlane * 4;
            off = align_up(off + (gains.full ? P.stage_buf * 4 : 4 * 64 * kHalfLd * 4), 16);
        }
    } else if (gather && gains.d) {
        // calibrated: half-pair staging (four planes of 64 x kHalfLd floats at off_re), or with Jones matrices one
        // whole-pair staging buffer (two planes: the four products of 32 x 32 tile pairs), then the item's copy
        P.off_re = off;
        P.off_im = off + kPlane * 4;
        off = align_up(off + (gains.full ? P.stage_buf * 4 : 4 * 64 * kHalfLd * 4), 16);
        P.off_item = off;
        off = align_up(off + (uint32_t)(8 * B), 16);
        P.two_stage = 0;
    } else if (gather) {
        // gather order: the item's baseline-ordered copy takes the staging buffers' place
        P.off_item = off;
        off = align_up(off + (uint32_t)(8 * B), 16);
        P.two_stage = 0;
    } else {
        P.two_stage = off + 2 * P.stage_buf * 4 + tail <= 227 * 1024;
        off = align_up(off + (P.two_stage ? 2 : 1) * P.stage_buf * 4, 16);
    }
    P.off_gain = off;                              // [n_tiles][2] (or [n_tiles][4] Jones) float2 when given
    if (gains.d) off = align_up(off + gain_bytes, 16);
    P.off_lut = off;
    off += 256 * 4;
    P.off_flags = off;
    off = align_up(off + nt, 16);
    P.off_bar = off;
    off += 24;
    P.off_tmem = off;
    off += 8;
    if ((uint32_t)P.Kp * 8 >= (1u << 18)) return (size_t)1 << 30;
    return std::max<size_t>(off, 120 * 1024);      // one CTA per SM: it owns all 512 TMEM columns
}

// The launch parameters that do not depend on the chunking; false when the form cannot run this request.
bool tc_setup(TcParams& P, int out_kind, const Plan& p, int ns, GainRef gains) {
    const int nt = p.n_tiles, c = p.chan_avg;
    if (nt % 8 || c > 256 || ns < 1) return false;
    P.mode = out_kind;
    P.n_tiles = nt;
    P.ns = ns;
    P.c = c;
    P.F = p.F;
    P.K = ns * c;
    const bool four = out_kind == CORR_OUT_VIS4 || (gains.d && gains.full);   // all four products
    P.units = four ? 2 * nt : nt;
    P.n_blk = (P.units + kUnitsPerBlk - 1) / kUnitsPerBlk;
    P.gains = gains.d;
    P.gain_f0 = gains.f0;
    P.split = gains.d && !gains.full && out_kind == CORR_OUT_STOKES_I;
    P.n_pairs = P.n_blk * (P.n_blk + 1) / 2;
    P.pair_cols = P.split ? 128 : 64;
    P.pairs_per_round = kTmemCols / P.pair_cols;
    P.n_rounds = (P.n_pairs + P.pairs_per_round - 1) / P.pairs_per_round;
    P.stage_buf = (P.split ? 4 : 2) * kPlane;
    // exactness: the FP32 accumulator holds integers below 2^24; |S| <= 128 K per product, and Stokes I without
    // split chains sums XX and YY in one accumulator
    const int64_t bound = (out_kind == CORR_OUT_STOKES_I && !P.split && !four) ? 256 : 128;
    return bound * P.K < ((int64_t)1 << 24);
}

// The chunk (samples, at most 256: the TMA box) of the fewest chunks whose layout fits; 0 if none does.
int tc_chunk(TcParams& P, bool gather, GainRef gains, int64_t B) {
    P.overlay = 0;
    if (tc_layout(P, std::min(P.ns, 256), gather, gains, B) <= 227 * 1024) return std::min(P.ns, 256);
    P.overlay = gather && P.n_rounds == 1 ? 1 : 0;
    // the longest chunk that fits, then the same number of chunks balanced (equal lengths but the last)
    for (int ns_c = std::min(P.ns, 256); ns_c >= 1; ns_c--) {
        if (tc_layout(P, ns_c, gather, gains, B) <= 227 * 1024) {
            const int n = (P.ns + ns_c - 1) / ns_c;
            return (P.ns + n - 1) / n;
        }
    }
    return 0;
}

}  // namespace

// Whether the gather-order form runs for this plan: no calibration, a gather source table, and a chunking
// whose operands fit beside the item's copy (2 B floats) in shared memory.
bool corr_fp8_gathers(const Plan& p, int ns, int out_kind, GainRef gains) {
    if (out_kind == CORR_OUT_VIS4 || !p.d_gsrc) return false;
    TcParams P{};
    if (!tc_setup(P, out_kind, p, ns, gains)) return false;
    return tc_chunk(P, true, gains, p.B) > 0;
}

blink_status launch_corr_fp8(int out_kind, const uint8_t* d_volt, int64_t sample_stride, const Plan& p, int ns,
                             int first_item, int n_items, void* out, int64_t out_item_stride, int* d_status, int n_sm,
                             cudaStream_t st, GainRef gains, ImgOut io) {
    if (n_items <= 0) return BLINK_OK;
    const int nt = p.n_tiles, c = p.chan_avg;
    if (nt % 8 || c > 256 || ((uintptr_t)d_volt & 15) || (sample_stride % 16))
        return set_error(BLINK_ERR_UNSUPPORTED,
                         "FP8 tensor-core correlation needs n_tiles % 8 == 0, chan_avg <= 256 and a 16-byte aligned "
                         "voltage block");
    TcParams P{};
    if (!tc_setup(P, out_kind, p, ns, gains))
        return set_error(BLINK_ERR_UNSUPPORTED, "FP8 tensor-core correlation: K too large for exact FP32 accumulation "
                                                "(128 K, or 256 K for Stokes I, must stay below 2^24)");
    if (io.gather && !corr_fp8_gathers(p, ns, out_kind, gains))
        return set_error(BLINK_ERR_UNSUPPORTED, "FP8 correlation: gather order not available for this plan");
    const int ns_c = tc_chunk(P, io.gather, gains, p.B);
    if (!ns_c)
        return set_error(BLINK_ERR_UNSUPPORTED, "FP8 tensor-core correlation: operands do not fit shared memory");
    const size_t smem = tc_layout(P, ns_c, io.gather, gains, p.B);
    if (io.gather) {
        P.gsrc = p.d_gsrc;
        P.gphase = p.d_gphase;
        P.ent_off = p.d_ent_off;
        P.ent_ld = p.N / 2 + 1;
        P.e_stride = p.e_stride;
    }
    P.first_item = first_item;
    P.n_items = n_items;
    P.flags = p.d_flags;
    P.out = out;
    P.out_item_stride = out_item_stride;
    P.status = d_status;
    P.B = p.B;
    if (out_kind != CORR_OUT_VIS4 && !io.gather) P.io = io;

    auto encode = encode_fn();
    if (!encode) return set_error(BLINK_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const int last_tau = (first_item + n_items - 1) / p.F;
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)(nt / 2), (cuuint64_t)p.n_fine, (cuuint64_t)(last_tau + 1) * ns};
    const cuuint64_t strides[2] = {(cuuint64_t)nt * 2, (cuuint64_t)sample_stride};
    const cuuint32_t box[3] = {(cuuint32_t)(nt / 2), (cuuint32_t)c, (cuuint32_t)ns_c};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<uint8_t*>(d_volt), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(BLINK_ERR_CUDA, "cuTensorMapEncodeTiled failed for the voltage block");
    static size_t smem_set = 0;                   // raise the kernel's limit once (not during a capture)
    if (smem > smem_set) {
        BLINK_CUDA(cudaFuncSetAttribute(k_corr_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        BLINK_CUDA(cudaFuncSetAttribute(k_corr_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        BLINK_CUDA(cudaFuncSetAttribute(k_corr_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        smem_set = 227 * 1024;
    }
    const int grid = std::min(n_items, n_sm);
    if (gains.d && gains.full)
        k_corr_tc<2><<<grid, kThreads, smem, st>>>(map, P);
    else if (gains.d)
        k_corr_tc<1><<<grid, kThreads, smem, st>>>(map, P);
    else
        k_corr_tc<0><<<grid, kThreads, smem, st>>>(map, P);
    BLINK_CUDA(cudaGetLastError());
    return BLINK_OK;
}

}  // namespace blink
