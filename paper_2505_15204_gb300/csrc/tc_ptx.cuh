// Inline-PTX helpers of the tcgen05 correlation (Blackwell): shared-memory addresses, mbarriers, the
// tensor-core MMA with FP8 e4m3 operands and FP32 accumulation in tensor memory, and tensor-memory loads.
// Shared by the standalone correlator and the correlation tasks of the fused imaging kernel.
#pragma once

#include <stdint.h>

namespace blink {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of parity `parity` to complete; false if `budget` clock cycles ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long budget) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, no swizzle.  lbo = byte distance of core matrices adjacent
// along K, sbo = byte distance of 8-row groups; bits 46-47 hold the descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f8f6f4: D = F32, A = B = E4M3, both K-major, dense.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 8 consecutive TMEM columns of this warp's 32 lanes, then the wait
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// byte offset of (row, kbyte) inside a 128-row operand tile of Kp bytes per row
__device__ __forceinline__ int op_off(int row, int kb, int Kp) {
    return (row >> 3) * (Kp * 8) + (kb >> 4) * 128 + (row & 7) * 16 + (kb & 15);
}

__device__ __forceinline__ void pair_of(int q, int& mb, int& jb) {
    mb = 0;
    while ((mb + 1) * (mb + 2) / 2 <= q) mb++;
    jb = q - mb * (mb + 1) / 2;
}


// One item's FP8 operand rows from its raw 4+4-bit samples: task (k group g of four consecutive K positions,
// tile a, polarisation p) turns four raw bytes (through the byte -> e4m3 LUT) into the words P_re, P_im (= Q_im)
// and Q_-re of one unit row.  raw[k * per_k + r] is the byte of sample position k and r = 2 a + p; positions
// k >= Kv and flagged tiles give zero rows.  Layout (K-major, no swizzle, 8 x 16-byte core matrices) of 128-row
// tiles of Kp bytes, unit u in tile u / 64 (row u % 64 for P, u % 64 + 64 for Q); Stokes I puts the X and Y
// halves of K side by side (units = tiles, K' = 2 Kq), the four-product layout has units 2 a + p, XX only X.
template <bool STOKES_I, bool FOUR>
__device__ __forceinline__ void unpack_e4m3(const uint8_t* raw, const uint32_t* lut, const uint8_t* sflags,
                                            uint8_t* ops, uint32_t tile_bytes, int n_tiles, int Kq, int Kp, int Kv,
                                            int tid, int n_threads) {
    const int per_k = 2 * n_tiles;
    const int n_groups = Kq >> 2;
    for (int e = tid; e < n_groups * per_k; e += n_threads) {
        const int g = e / per_k, r = e - g * per_k;
        const int k0 = 4 * g, a = r >> 1, p = r & 1;
        int unit, kp, kh;
        if (STOKES_I) {
            unit = a; kp = p * Kq + k0; kh = 2 * Kq;        // re X, re Y, im X, im Y
        } else if (FOUR) {
            unit = 2 * a + p; kp = k0; kh = Kq;
        } else {
            if (p) continue;
            unit = a; kp = k0; kh = Kq;
        }
        const bool live = !sflags[a];
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; i++) w[i] = (live && k0 + i < Kv) ? lut[raw[(k0 + i) * per_k + r]] : 0u;
        const uint32_t re = __byte_perm(__byte_perm(w[0], w[1], 0x0040), __byte_perm(w[2], w[3], 0x0040), 0x5410);
        const uint32_t im = __byte_perm(__byte_perm(w[0], w[1], 0x0051), __byte_perm(w[2], w[3], 0x0051), 0x5410);
        const uint32_t nre = __byte_perm(__byte_perm(w[0], w[1], 0x0073), __byte_perm(w[2], w[3], 0x0073), 0x5410);
        uint8_t* tile = ops + (unit >> 6) * tile_bytes;
        const int row = unit & 63;
        *reinterpret_cast<uint32_t*>(tile + op_off(row, kp, Kp)) = re;
        *reinterpret_cast<uint32_t*>(tile + op_off(row, kp + kh, Kp)) = im;
        *reinterpret_cast<uint32_t*>(tile + op_off(row + 64, kp, Kp)) = im;
        *reinterpret_cast<uint32_t*>(tile + op_off(row + 64, kp + kh, Kp)) = nre;
    }
}

// The byte -> e4m3 LUT: a byte's nibbles re (low), im (high) in [-8, 7] give the words (re, im, im, -re).
__device__ __forceinline__ void fill_e4m3_lut(uint32_t* lut, int tid, int n_threads) {
    const uint32_t pos[9] = {0x00, 0x38, 0x40, 0x44, 0x48, 0x4A, 0x4C, 0x4E, 0x50};   // e4m3 of 0 .. 8
    for (int b = tid; b < 256; b += n_threads) {
        const int re = (b & 15) >= 8 ? (b & 15) - 16 : (b & 15);
        const int im = (b >> 4) >= 8 ? (b >> 4) - 16 : (b >> 4);
        auto e4m3 = [&](int v) -> uint32_t { return v >= 0 ? pos[v] : (0x80u | pos[-v]); };
        lut[b] = e4m3(re) | (e4m3(im) << 8) | (e4m3(im) << 16) | (e4m3(-re) << 24);
    }
}

}  // namespace blink
