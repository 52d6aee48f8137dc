// Device-side building blocks of the Falcon kernels (sm_103a).
//
// Work decomposition: one warp per chunk of B <= 1025 values.  Lane l owns the 32
// consecutive delta columns 32l .. 32l+31 (column c holds z_{c+2}, Eq. 5), so a 32x32
// bit transpose in registers turns each bit plane into one 32-bit word whose
// little-endian bytes are row bytes 4l .. 4l+3 of that plane (Sec. 3.3, Fig. 8).
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "falcon_internal.h"

#define FALCON_TABLE_QUAL static __constant__ const
#include "falcon_tables.h"

namespace falcon {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Value kinds of the kernels: D = 0 FP64, 1 FP32, 2 FP16 (binary16, R18).  U holds a value's
// bit pattern and every integer derived from it (G, Z) modulo 2^W.
constexpr int kD64 = 0, kD32 = 1, kD16 = 2;
template <int D> struct Traits;
template <> struct Traits<kD64> {
    using U = uint64_t;
    static constexpr int W = 64;            // bits per value
    static constexpr int S = 8;             // bytes per value
    static constexpr int Z1B = 8;           // bytes of z_1 in a record
    static constexpr int A_MAX = 22;        // Case 1: alpha_max <= 22 (Thm 3)
    static constexpr int B_MAX = 15;        // Case 1: beta_hat_max <= 15 (Thm 2)
    static constexpr int A_SENT = 23;       // Case-2 header sentinels
    static constexpr int B_SENT = 16;
    static constexpr int UNITS = 16;        // 16-byte units per lane (32 values)
};
template <> struct Traits<kD32> {
    using U = uint32_t;
    static constexpr int W = 32;
    static constexpr int S = 4;
    static constexpr int Z1B = 4;
    static constexpr int A_MAX = 10;        // 5^10 < 2^24: 10^alpha exact in FP32
    static constexpr int B_MAX = 7;         // 10^7 < 2^24
    static constexpr int A_SENT = 11;
    static constexpr int B_SENT = 8;
    static constexpr int UNITS = 8;
};
template <> struct Traits<kD16> {
    using U = uint16_t;
    static constexpr int W = 16;
    static constexpr int S = 2;
    static constexpr int Z1B = 2;
    static constexpr int A_MAX = 4;         // 5^4 < 2^11: 10^alpha exact in binary16
    static constexpr int B_MAX = 3;         // 10^3 < 2^11
    static constexpr int A_SENT = 5;
    static constexpr int B_SENT = 4;
    static constexpr int UNITS = 4;
};

// --------------------------------------------------------------------------------------
// small helpers
// --------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most the most recently committed group is still in flight
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_none() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Bulk (TMA) copy of `bytes` from shared to global memory, both 16-byte aligned, bytes a
// multiple of 16, tracked in the issuing thread's bulk groups.  The writers of the shared
// bytes must have executed fence_proxy_async() first.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_addr(ssrc)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared source of every committed bulk copy has been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed bulk copy has completed
__device__ __forceinline__ void bulk_wait() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ uint64_t zigzag(uint64_t x) { return (x << 1) ^ (uint64_t)((int64_t)x >> 63); }
__device__ __forceinline__ uint32_t zigzag(uint32_t x) { return (x << 1) ^ (uint32_t)((int32_t)x >> 31); }
__device__ __forceinline__ uint64_t unzigzag(uint64_t z) { return (z >> 1) ^ (0ull - (z & 1ull)); }
__device__ __forceinline__ uint32_t unzigzag(uint32_t z) { return (z >> 1) ^ (0u - (z & 1u)); }
__device__ __forceinline__ uint16_t zigzag(uint16_t x) {
    return (uint16_t)(((uint32_t)x << 1) ^ (uint32_t)((int32_t)(int16_t)x >> 15));
}
__device__ __forceinline__ uint16_t unzigzag(uint16_t z) { return (uint16_t)((z >> 1) ^ (0u - (z & 1u))); }

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src) {
    return ((uint64_t)__shfl_sync(kFull, (uint32_t)(v >> 32), src) << 32) |
           __shfl_sync(kFull, (uint32_t)v, src);
}
__device__ __forceinline__ uint64_t shfl_down_u64(uint64_t v, int d) {
    return ((uint64_t)__shfl_down_sync(kFull, (uint32_t)(v >> 32), d) << 32) |
           __shfl_down_sync(kFull, (uint32_t)v, d);
}
__device__ __forceinline__ uint64_t shfl_up_u64(uint64_t v, int d) {
    return ((uint64_t)__shfl_up_sync(kFull, (uint32_t)(v >> 32), d) << 32) |
           __shfl_up_sync(kFull, (uint32_t)v, d);
}
__device__ __forceinline__ uint32_t shfl_x(uint32_t v, int src) { return __shfl_sync(kFull, v, src); }
__device__ __forceinline__ uint64_t shfl_x(uint64_t v, int src) { return shfl_u64(v, src); }
__device__ __forceinline__ uint32_t shfl_down_x(uint32_t v, int d) { return __shfl_down_sync(kFull, v, d); }
__device__ __forceinline__ uint64_t shfl_down_x(uint64_t v, int d) { return shfl_down_u64(v, d); }
__device__ __forceinline__ uint32_t shfl_up_x(uint32_t v, int d) { return __shfl_up_sync(kFull, v, d); }
__device__ __forceinline__ uint64_t shfl_up_x(uint64_t v, int d) { return shfl_up_u64(v, d); }
__device__ __forceinline__ uint16_t shfl_x(uint16_t v, int src) { return (uint16_t)__shfl_sync(kFull, (uint32_t)v, src); }
__device__ __forceinline__ uint16_t shfl_down_x(uint16_t v, int d) {
    return (uint16_t)__shfl_down_sync(kFull, (uint32_t)v, d);
}
__device__ __forceinline__ uint16_t shfl_up_x(uint16_t v, int d) { return (uint16_t)__shfl_up_sync(kFull, (uint32_t)v, d); }

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += ((uint64_t)__shfl_xor_sync(kFull, (uint32_t)(v >> 32), o) << 32) |
                                          __shfl_xor_sync(kFull, (uint32_t)v, o);
    return v;
}
__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
    uint32_t hi = __reduce_max_sync(kFull, (uint32_t)(v >> 32));
    uint32_t lo = __reduce_max_sync(kFull, ((uint32_t)(v >> 32) == hi) ? (uint32_t)v : 0u);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint32_t warp_max_x(uint32_t v) { return __reduce_max_sync(kFull, v); }
__device__ __forceinline__ uint64_t warp_max_x(uint64_t v) { return warp_max_u64(v); }
__device__ __forceinline__ uint32_t warp_or_x(uint32_t v) { return __reduce_or_sync(kFull, v); }
__device__ __forceinline__ uint16_t warp_max_x(uint16_t v) { return (uint16_t)__reduce_max_sync(kFull, (uint32_t)v); }
__device__ __forceinline__ uint16_t warp_or_x(uint16_t v) { return (uint16_t)__reduce_or_sync(kFull, (uint32_t)v); }
__device__ __forceinline__ uint64_t warp_or_x(uint64_t v) {
    return ((uint64_t)__reduce_or_sync(kFull, (uint32_t)(v >> 32)) << 32) | __reduce_or_sync(kFull, (uint32_t)v);
}
// exclusive prefix sum of a 64-bit lane value over the warp
__device__ __forceinline__ uint64_t warp_exclusive_u64(uint64_t v, int lane) {
    uint64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = shfl_up_u64(incl, o);
        if (lane >= o) incl += t;
    }
    return incl - v;
}

// number of zero bytes of a 32-bit word (exact)
__device__ __forceinline__ int zero_bytes(uint32_t x) {
    uint32_t y = (x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu;
    y = ~(y | x | 0x7F7F7F7Fu);
    return __popc(y);
}
// 4-bit mask, bit (3-i) set iff byte i of x is non-zero
__device__ __forceinline__ uint32_t nonzero_nibble(uint32_t x) {
    uint32_t y = (x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu;
    y = (y | x) & 0x80808080u;          // bit 8i+7 set iff byte i != 0
    return ((y >> 4) & 8u) | ((y >> 13) & 4u) | ((y >> 22) & 2u) | ((y >> 31) & 1u);
}

// --------------------------------------------------------------------------------------
// 32x32 bit transpose in registers: afterwards bit j of a[i] = old bit i of a[j].
// Recursive exchange of the off-diagonal blocks (Hacker's Delight, Sec. 7-3).
// --------------------------------------------------------------------------------------
__device__ __forceinline__ void transpose32(uint32_t (&a)[32]) {
    // 16- and 8-bit block exchanges are byte permutations (one PRMT per output word)
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint32_t x = a[k], y = a[k + 16];
        a[k] = __byte_perm(x, y, 0x5410);
        a[k + 16] = __byte_perm(x, y, 0x7632);
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        if ((k & 8) == 0) {
            const uint32_t x = a[k], y = a[k + 8];
            a[k] = __byte_perm(x, y, 0x6240);
            a[k + 8] = __byte_perm(x, y, 0x7351);
        }
    }
#define FALCON_TSTEP(h, mask)                                                       \
    _Pragma("unroll") for (int k = 0; k < 32; ++k) {                               \
        if ((k & (h)) == 0) {                                                       \
            uint32_t t = ((a[k] >> (h)) ^ a[k + (h)]) & (mask);                     \
            a[k + (h)] ^= t;                                                        \
            a[k] ^= t << (h);                                                       \
        }                                                                           \
    }
    FALCON_TSTEP(4, 0x0F0F0F0Fu)
    FALCON_TSTEP(2, 0x33333333u)
    FALCON_TSTEP(1, 0x55555555u)
#undef FALCON_TSTEP
}

// --------------------------------------------------------------------------------------
// Shared-memory staging of a chunk's values, swizzled so that lane l's 16-byte units
// (values 32l .. 32l+31) are read conflict-free: unit u of lane L sits at L*UNITS + (u^(L&7)).
// --------------------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ uint32_t unit_swizzle(uint32_t L, uint32_t u) {
    // lane L's unit u: every 8 consecutive lanes reading their unit u hit 8 distinct 16-byte
    // bank groups (FP16 has 4 units per lane, so lanes L and L + 4 differ by the XOR)
    constexpr int UN = Traits<D>::UNITS;
    return u ^ (UN >= 8 ? (L & 7u) : ((L >> 1) & 3u));
}
template <int D>
__device__ __forceinline__ uint32_t phys_unit(uint32_t q) {
    constexpr int UN = Traits<D>::UNITS;
    uint32_t L = q / UN, u = q % UN;
    return L * UN + unit_swizzle<D>(L, u);
}
template <int D>
__device__ __forceinline__ uint32_t phys_elem_byte(uint32_t e) {
    constexpr int S = Traits<D>::S;
    constexpr int PER = 16 / S;       // values per unit
    return phys_unit<D>(e / PER) * 16u + (e % PER) * S;
}

// Starts loading m values (m <= 1025) from global src into a warp staging buffer
// (cp.async; the caller commits and waits).
template <int D>
__device__ __forceinline__ void stage_values_async(const uint8_t *src, uint32_t m, uint8_t *wsm, int lane) {
    constexpr int S = Traits<D>::S;
    const uint32_t base = smem_addr(wsm);
    const uint32_t nbytes = m * S;
    uint32_t done = 0;
    if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
        const uint32_t nunits = nbytes >> 4;
        constexpr uint32_t FULL_UNITS = 1024u * S / 16u;    // a whole 1024-value chunk
        if (nunits >= FULL_UNITS) {
            // unit q = lane + 32 i belongs to lane L = q / UNITS, slot u = q % UNITS
#pragma unroll
            for (uint32_t i = 0; i < FULL_UNITS / 32u; ++i) {
                const uint32_t q = lane + 32u * i;
                cp_async16(base + phys_unit<D>(q) * 16u, src + 16u * q);
            }
            for (uint32_t q = FULL_UNITS + lane; q < nunits; q += 32) cp_async16(base + phys_unit<D>(q) * 16u, src + 16u * q);
        } else {
            for (uint32_t q = lane; q < nunits; q += 32) cp_async16(base + phys_unit<D>(q) * 16u, src + 16u * q);
        }
        done = (nunits * 16u) / S;
    }
    for (uint32_t e = done + lane; e < m; e += 32) {
        if constexpr (D == kD64) cp_async8(base + phys_elem_byte<D>(e), src + (size_t)e * S);
        else if constexpr (D == kD32) cp_async4(base + phys_elem_byte<D>(e), src + (size_t)e * S);
        else                                     // no 2-byte cp.async: a plain copy (visible at the next __syncwarp)
            *reinterpret_cast<uint16_t *>(wsm + phys_elem_byte<D>(e)) = *reinterpret_cast<const uint16_t *>(src + (size_t)e * S);
    }
}

// Lane reads its 32 values (indices 32*lane + k); indices >= m read as +0.
template <int D>
__device__ __forceinline__ void read_own(const uint8_t *wsm, int lane, uint32_t m,
                                         typename Traits<D>::U (&v)[32]) {
    using U = typename Traits<D>::U;
    constexpr int UN = Traits<D>::UNITS;
    constexpr int PER = 32 / UN;
#pragma unroll
    for (int u = 0; u < UN; ++u) {
        const uint4 q = *reinterpret_cast<const uint4 *>(wsm + (lane * UN + unit_swizzle<D>(lane, u)) * 16);
        if constexpr (D == kD64) {
            v[PER * u + 0] = ((U)q.y << 32) | q.x;
            v[PER * u + 1] = ((U)q.w << 32) | q.z;
        } else if constexpr (D == kD16) {
            const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                v[PER * u + 2 * h] = (U)(w4[h] & 0xFFFFu);
                v[PER * u + 2 * h + 1] = (U)(w4[h] >> 16);
            }
        } else {
            v[PER * u + 0] = q.x;
            v[PER * u + 1] = q.y;
            v[PER * u + 2] = q.z;
            v[PER * u + 3] = q.w;
        }
    }
    if (m < 1024u) {                              // a tail chunk: values past m read as +0
#pragma unroll
        for (int k = 0; k < 32; ++k)
            if ((uint32_t)(32 * lane + k) >= m) v[k] = 0;
    }
}

template <int D>
__device__ __forceinline__ typename Traits<D>::U read_elem(const uint8_t *wsm, uint32_t e) {
    using U = typename Traits<D>::U;
    return *reinterpret_cast<const U *>(wsm + phys_elem_byte<D>(e));
}

// --------------------------------------------------------------------------------------
// Classification (R1: -0, NaN, inf, subnormals are exceptions)
// --------------------------------------------------------------------------------------
__device__ __forceinline__ bool is_special(uint64_t u) {
    const uint64_t a = u & 0x7FFFFFFFFFFFFFFFull;
    return (u != 0) && (a - 0x0010000000000000ull >= 0x7FE0000000000000ull);
}
__device__ __forceinline__ bool is_special(uint32_t u) {
    const uint32_t a = u & 0x7FFFFFFFu;
    return (u != 0) && (a - 0x00800000u >= 0x7F000000u);
}
__device__ __forceinline__ bool is_special(uint16_t u) {
    const uint32_t a = u & 0x7FFFu;
    return (u != 0) && (a - 0x0400u >= 0x7800u);
}

// floor(log10 a) as the largest k with a >= fl(10^k), for a normal, positive, with binary
// exponent in the table's reach (checked by the caller).
__device__ __forceinline__ int floor_log10(uint64_t a) {
    const int e2 = (int)(a >> 52) - 1023;
    int k = (e2 * 78913) >> 18;        // floor(e2 * log10 2) up to +-1
    if (a >= FALCON_P10_F64[k + 1 - FALCON_P10_F64_LO]) ++k;
    else if (a < FALCON_P10_F64[k - FALCON_P10_F64_LO]) --k;
    return k;
}
__device__ __forceinline__ int floor_log10(uint32_t a) {
    const int e2 = (int)(a >> 23) - 127;
    int k = (e2 * 78913) >> 18;
    if (a >= FALCON_P10_F32[k + 1 - FALCON_P10_F32_LO]) ++k;
    else if (a < FALCON_P10_F32[k - FALCON_P10_F32_LO]) --k;
    return k;
}
__device__ __forceinline__ int floor_log10(uint16_t a) {
    const int e2 = (int)(a >> 10) - 15;
    int k = (e2 * 78913) >> 18;
    if (k < FALCON_P10_F16_HI && a >= FALCON_P10_F16[k + 1 - FALCON_P10_F16_LO]) ++k;
    else if (a < FALCON_P10_F16[k - FALCON_P10_F16_LO]) --k;
    return k;
}
// binary-exponent window where floor_log10 is defined and Case 1 is reachable
__device__ __forceinline__ bool log10_in_range(uint64_t a) {
    const uint32_t be = (uint32_t)(a >> 52);
    return be >= 1023u - 90u && be < 1023u + 50u;
}
__device__ __forceinline__ bool log10_in_range(uint32_t a) {
    const uint32_t be = a >> 23;
    return be >= 127u - 40u && be < 127u + 24u;
}
__device__ __forceinline__ bool log10_in_range(uint16_t) { return true; }   // every normal binary16

// --------------------------------------------------------------------------------------
// The per-value test of Alg. 2 at decimal place a, in exact integer arithmetic.
//
// Alg. 2 accepts a for v when v (x) 10^a lies within |x| 2^-52 of an integer (eps <= mu)
// and round(x) / 10^a gives back v.  With v = m 2^E, P = m 5^a and F = -(E + a), the exact
// product is X = P / 2^F; for |X| < 2^50 both conditions together are equivalent to
//   fl(N / 10^a) == v   with N = round(X),
// i.e. |N 2^F - P| < 5^a / 2 (5^a / 4 below a power of two), because the rounding interval
// of v scaled by 10^a is exactly that wide.  The same holds for FP32 (exact x, R14).
// Callers only ask for a with |X| < 10^15 (FP32: < 10^7).
// --------------------------------------------------------------------------------------
__device__ __forceinline__ bool q_test(uint64_t u, int a) {
    const uint64_t au = u & 0x7FFFFFFFFFFFFFFFull;
    if (au == 0) return true;
    const int E = (int)(au >> 52) - 1075;
    const uint64_t m = (au & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const int F = -(E + a);
    if (F <= 0) return true;
    if (F >= 128) return false;
    const uint64_t p5 = FALCON_POW5[a];
    if (F <= 64) {
        // the low F bits of P are the low bits of the 64-bit product: no 128-bit arithmetic
        const uint64_t mask = (F == 64) ? ~0ull : ((1ull << F) - 1ull);
        const uint64_t r = (m * p5) & mask;
        const uint64_t lim = p5 >> 1;
        if (r > (mask >> 1)) return (mask - r) + 1ull <= lim;          // r >= 2^(F-1)
        return r <= ((m == 0x0010000000000000ull) ? ((p5 - 1) >> 2) : lim);
    }
    const unsigned __int128 P = (unsigned __int128)m * p5;
    const unsigned __int128 one = 1;
    const unsigned __int128 r = P & ((one << F) - 1);
    const unsigned __int128 half = one << (F - 1);
    const uint64_t lim = p5 >> 1;
    if (r >= half) return ((one << F) - r) <= lim;
    return r <= ((m == 0x0010000000000000ull) ? ((p5 - 1) >> 2) : lim);
}
__device__ __forceinline__ bool alg2_step_f32(uint32_t u, int a, bool &rt);
__device__ __forceinline__ bool q_test(uint32_t u, int a) {
    bool rt;
    (void)alg2_step_f32(u, a, rt);
    return rt;
}

// Alg. 2's first test alone (eps <= mu) for FP32, on the exact product x = v * 10^a (R14):
// the distance of X = P / 2^F to the nearest integer is at most X * 2^-23.
__device__ __forceinline__ bool eps_le_mu(uint32_t u, int a) {
    const uint32_t au = u & 0x7FFFFFFFu;
    if (au == 0) return true;
    const int E = (int)(au >> 23) - 150;
    const uint64_t m = (au & 0x007FFFFFu) | 0x00800000u;
    const int F = -(E + a);
    if (F <= 0) return true;
    if (F >= 64) return false;
    const uint64_t P = m * FALCON_POW5[a];
    const uint64_t r = P & ((1ull << F) - 1);
    const uint64_t rc = (1ull << F) - r;
    const uint64_t dist = r < rc ? r : rc;
    return dist <= (P >> 23);
}

// Both tests of Alg. 2 for FP32 at decimal place a, from one product: eps <= mu (returned)
// and the round trip (rt), as eps_le_mu and q_test compute them.  P = m 5^a < 2^48 comes from
// one 32 x 32 -> 64 multiply; for F < 32 the remainder and both bounds are 32-bit.
__device__ __forceinline__ bool alg2_step_f32(uint32_t u, int a, bool &rt) {
    const uint32_t au = u & 0x7FFFFFFFu;
    const int F = 150 - (int)(au >> 23) - a;
    if (au == 0 || F <= 0) { rt = true; return true; }
    if (F >= 64) { rt = false; return false; }
    const uint32_t m = (au & 0x007FFFFFu) | 0x00800000u;
    const uint32_t p5 = (uint32_t)FALCON_POW5[a];          // 5^a < 2^24 for a <= 10
    const uint64_t P = (uint64_t)m * p5;
    const uint32_t lim = p5 >> 1, lim_low = (m == 0x00800000u) ? ((p5 - 1u) >> 2) : lim;
    const uint32_t mu = (uint32_t)(P >> 23);                // < 2^25
    if (F < 32) {
        const uint32_t mask = (1u << F) - 1u;
        const uint32_t r = (uint32_t)P & mask, rc = mask - r + 1u;
        rt = (r > (mask >> 1)) ? (rc <= lim) : (r <= lim_low);
        return (r < rc ? r : rc) <= mu;
    }
    const uint64_t mask = (1ull << F) - 1ull;
    const uint64_t r = P & mask, rc = mask - r + 1ull;
    rt = (r > (mask >> 1)) ? (rc <= lim) : (r <= lim_low);
    return (r < rc ? r : rc) <= mu;
}

// FP32 decimal place of one value as Alg. 2 finds it, restricted to [0, atop]: the first a
// with eps <= mu, accepted only if the round trip holds there; -1 otherwise (an exception
// or a decimal place beyond atop, both of which make the chunk Case 2).  The 24-bit
// significand leaves no margin for Thm 4 at beta = 7, so early spurious passes are real
// and must be reproduced value by value.
__device__ __forceinline__ int first_pass_f32(uint32_t u, int atop) {
    if ((u & 0x7FFFFFFFu) == 0) return 0;
    for (int a = 0; a <= atop; ++a)
        if (eps_le_mu(u, a)) return q_test(u, a) ? a : -1;
    return -1;
}

// g = round(v (x) 10^a) (Eq. 4, Case 1) for a value that passed q_test at a.  Passing means
// X = v 10^a lies within 5^a / 2^(F+1) <= 1/8 of the integer g (the rounding interval of v,
// scaled), so an approximation of X closer than 3/8 rounds to g: with m and 5^a both
// normalised to 64 bits, mulhi(m 2^11, 5^a 2^(63-d)) = floor(X 2^sh), sh = F + 10 - d >= 13,
// is X within 2^-13, and rounding it at bit sh gives g.  One 64-bit high product per value.
__device__ __forceinline__ uint64_t case1_g(uint64_t u, int a) {
    const uint64_t au = u & 0x7FFFFFFFFFFFFFFFull;
    if (au == 0) return 0;
    const int E = (int)(au >> 52) - 1075;
    const uint64_t m = (au & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const int sh = -(E + a) + 10 - (int)FALCON_LOG2_POW5[a];
    const uint64_t t = __umul64hi(m << 11, FALCON_POW5_NORM[a]);
    const uint64_t N = ((t >> (sh - 1)) + 1ull) >> 1;
    return (u >> 63) ? (0ull - N) : N;
}
__device__ __forceinline__ uint32_t case1_g(uint32_t u, int a) {
    const uint32_t au = u & 0x7FFFFFFFu;
    if (au == 0) return 0;
    const int E = (int)(au >> 23) - 150;
    const uint64_t m = (au & 0x007FFFFFu) | 0x00800000u;
    const int F = -(E + a);
    const uint64_t P = m * FALCON_POW5[a];
    uint64_t N;
    if (F <= 0) N = P << (-F);
    else N = (P + (1ull << (F - 1))) >> F;
    return (u >> 31) ? (0u - (uint32_t)N) : (uint32_t)N;
}

// binary16 (R18): both tests of Alg. 2 at decimal place a from one product, as for FP32:
// v = m 2^E with an 11-bit m, P = m 5^a < 2^21, F = -(E + a) <= 24; eps <= mu is
// dist(P, 2^F Z) <= P 2^-10 and the round trip |N 2^F - P| < 5^a / 2 (5^a / 4 below a power
// of two, where the ulp below v is half as wide).
__device__ __forceinline__ bool alg2_step_f16(uint16_t u, int a, bool &rt) {
    const uint32_t au = u & 0x7FFFu;
    const int F = 25 - (int)(au >> 10) - a;
    if (au == 0 || F <= 0) { rt = true; return true; }
    const uint32_t m = (au & 0x3FFu) | 0x400u;
    const uint32_t p5 = (uint32_t)FALCON_POW5[a];            // 5^a <= 625
    const uint32_t P = m * p5;
    const uint32_t lim = p5 >> 1, lim_low = (m == 0x400u) ? ((p5 - 1u) >> 2) : lim;
    const uint32_t mask = (1u << F) - 1u;
    const uint32_t r = P & mask, rc = mask - r + 1u;
    rt = (r > (mask >> 1)) ? (rc <= lim) : (r <= lim_low);
    return (r < rc ? r : rc) <= (P >> 10);
}
__device__ __forceinline__ bool q_test(uint16_t u, int a) {
    bool rt;
    (void)alg2_step_f16(u, a, rt);
    return rt;
}
// Alg. 2's decimal place of one binary16 value within [0, atop]: the first a with eps <= mu,
// -1 if the round trip fails there (an early stop) or no a passes
__device__ __forceinline__ int first_pass_f16(uint16_t u, int atop) {
    if ((u & 0x7FFFu) == 0) return 0;
    for (int a = 0; a <= atop; ++a) {
        bool rt;
        if (alg2_step_f16(u, a, rt)) return rt ? a : -1;
    }
    return -1;
}
__device__ __forceinline__ uint16_t case1_g(uint16_t u, int a) {
    const uint32_t au = u & 0x7FFFu;
    if (au == 0) return 0;
    const int F = 25 - (int)(au >> 10) - a;
    const uint32_t P = ((au & 0x3FFu) | 0x400u) * (uint32_t)FALCON_POW5[a];
    const uint32_t N = F <= 0 ? (P << (-F)) : ((P + (1u << (F - 1))) >> F);
    return (uint16_t)((u >> 15) ? (0u - N) : N);
}

// fl(g / 10^a), correctly rounded (nearest, ties to even), for |g| < 2^53 and 0 <= a <= 22, in
// integer arithmetic (the inverse of Eq. 4, Case 1).  g / 10^a = (g / 5^a) 2^-a and the
// scaling by 2^-a is exact (no result is subnormal), so the work is one correctly rounded
// division by 5^a: with G = |g| normalised to [2^63, 2^64), d = floor(log2 5^a) and the
// reciprocal R = floor(2^(64+d) / 5^a), T = mulhi(G, R) is floor(G 2^d / 5^a) or one less
// (division by an invariant integer, Granlund and Montgomery, PLDI 1994); the remainder,
// below 2 * 5^a, is exact in 64-bit arithmetic and corrects T.  T has 63 or 64 significant
// bits; its top 53 bits, the next bit and a sticky bit (lower bits or a non-zero remainder)
// round to the IEEE significand.  Returns the bits of the double.
__device__ __forceinline__ uint64_t div_pow10_exact(int64_t g, int a) {
    if (g == 0) return 0;
    const uint64_t sign = (uint64_t)g & 0x8000000000000000ull;
    const uint64_t ag = g < 0 ? 0ull - (uint64_t)g : (uint64_t)g;
    const int s = __clzll((long long)ag);
    const uint64_t G = ag << s;
    uint64_t T = G, r = 0;
    int d = 0;
    if (a > 0) {
        d = FALCON_LOG2_POW5[a];
        const uint64_t D = FALCON_POW5[a];
        T = __umul64hi(G, FALCON_RECIP5[a]);
        r = (G << d) - T * D;                   // true remainder in [0, 2 D): exact mod 2^64
        if (r >= D) { r -= D; ++T; }
    }
    const int lz = __clzll((long long)T);       // 0 or 1
    const uint64_t Tn = T << lz;
    uint64_t mant = Tn >> 11;
    const uint32_t rest = (uint32_t)Tn & 0x7FFu;
    const bool sticky = (rest & 0x3FFu) != 0u || r != 0;
    if ((rest & 0x400u) && (sticky || (mant & 1ull))) ++mant;
    int e2 = 11 - lz - d - s - a;               // the value is mant * 2^e2
    if (mant == (1ull << 53)) { mant >>= 1; ++e2; }
    return sign | ((uint64_t)(e2 + 52 + 1023) << 52) | (mant & 0x000FFFFFFFFFFFFFull);
}

__device__ __forceinline__ void set_status(unsigned long long *result, uint32_t code) {
    atomicCAS(&result[1], 0ull, (unsigned long long)code);
}

// block-wide exclusive scan of one u64 per thread (1024 threads); returns the block total
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t &total, uint64_t *warp_sums) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t incl = v + warp_exclusive_u64(v, lane);
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint64_t ws = warp_sums[lane];
        const uint64_t wincl = ws + warp_exclusive_u64(ws, lane);
        warp_sums[lane] = wincl - ws;
        if (lane == 31) warp_sums[32] = wincl;
    }
    __syncthreads();
    const uint64_t r = warp_sums[warp] + incl - v;
    total = warp_sums[32];
    __syncthreads();
    return r;
}

// Exclusive prefix of a stream's u32 size array per 64-chunk tile, into tile_off[0 ..
// tile_count(nc)) (one 1024-thread block, thread t owning tile t of each step of 1024 tiles).
// Returns the total of all sizes (every thread).  A warp whose 32 tiles are all whole reads
// their 8 KB of sizes coalesced (16-byte unit 32 k + lane, i.e. tiles 2k and 2k + 1 in the
// two half-warps) and adds each tile up with half-warp shuffles in 32-bit arithmetic; a step
// in which some 16-byte unit adds up to 2^26 or more (only in a malformed stream) falls back
// to 64-bit sums per thread.
__device__ __forceinline__ uint64_t tile_prefix(const uint32_t *sizes, uint64_t nc, unsigned long long *tile_off,
                                                uint64_t *warp_sums) {
    const uint64_t ntiles = tile_count(nc);
    const uint64_t full_tiles = nc / kTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t carry = 0;
    for (uint64_t b = 0; b < ntiles; b += 1024) {
        const uint64_t tile = b + threadIdx.x;
        const uint64_t wt0 = b + 32u * (uint64_t)warp;
        uint64_t sum = 0;
        bool done = false;
        if (wt0 + 32u <= full_tiles) {
            const uint4 *q = reinterpret_cast<const uint4 *>(sizes + wt0 * kTile);
            uint32_t mine = 0;
            bool big = false;
#pragma unroll 4
            for (int k = 0; k < 16; ++k) {
                const uint4 x = q[32 * k + lane];
                const uint64_t s64 = (uint64_t)x.x + x.y + x.z + x.w;
                big |= s64 >= (1ull << 26);
                uint32_t s = (uint32_t)s64;
                s += __shfl_xor_sync(kFull, s, 8);
                s += __shfl_xor_sync(kFull, s, 4);
                s += __shfl_xor_sync(kFull, s, 2);
                s += __shfl_xor_sync(kFull, s, 1);
                const uint32_t lo = __shfl_sync(kFull, s, 0), hi = __shfl_sync(kFull, s, 16);
                if (lane == 2 * k) mine = lo;
                if (lane == 2 * k + 1) mine = hi;
            }
            done = !__any_sync(kFull, big);
            sum = mine;
        }
        if (!done && tile < ntiles) {
            sum = 0;
            const uint64_t c0 = tile * kTile;
            const uint64_t c1 = (c0 + kTile <= nc) ? c0 + kTile : nc;
            for (uint64_t c = c0; c < c1; ++c) sum += sizes[c];
        }
        uint64_t total;
        const uint64_t ex = carry + block_exclusive_scan(sum, total, warp_sums);
        if (tile < ntiles) tile_off[tile] = ex;
        carry += total;
    }
    return carry;
}

// Where chunk c's record starts (relative to the first record): its tile's offset plus the
// sizes of the earlier chunks of the tile.  load_pos issues the loads (every lane), resolve_pos
// adds them up (warp-collective) once they are needed, so their latency can be hidden.
struct ChunkPos {
    uint64_t tile;
    uint32_t s0, s1, size;
};
__device__ __forceinline__ ChunkPos load_pos(const uint32_t *sizes, const unsigned long long *tile_off, uint64_t c,
                                             int lane) {
    const uint64_t t0 = c & ~(kTile - 1);
    ChunkPos p;
    p.tile = tile_off[c / kTile];
    p.size = sizes[c];
    p.s0 = (t0 + (uint64_t)lane < c) ? sizes[t0 + lane] : 0u;
    p.s1 = (t0 + 32u + (uint64_t)lane < c) ? sizes[t0 + 32u + lane] : 0u;
    return p;
}
__device__ __forceinline__ uint64_t resolve_pos(const ChunkPos &p) {
    return p.tile + __reduce_add_sync(kFull, p.s0 + p.s1);       // a tile holds < 2^20 bytes
}

// Finds the job that owns global ticket t (jobs sorted by chunk_begin).
__device__ __forceinline__ int find_job(const Job *jobs, int njobs, uint64_t t) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].chunk_begin <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Chunk tickets (Control): take_ticket issues lane 0's atomic add and returns its raw result
// (valid in lane 0 only); ticket_of broadcasts it.  Issuing the atomic a chunk before its result
// is read hides the atomic's latency behind the current chunk; the add is predicated on lane 0
// into a register zeroed beforehand, so no instruction selects between the two and waits for it.
__device__ __forceinline__ unsigned long long take_ticket(Control *ctl, int which, int lane) {
    unsigned long long r;
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.eq.s32 p, %1, 0;\n\tmov.b64 %0, 0;\n\t"
        "@p atom.global.add.u64 %0, [%2], 1;\n\t}"
        : "=l"(r)
        : "r"(lane), "l"(&ctl->ticket[which])
        : "memory");
    return r;
}
__device__ __forceinline__ uint64_t ticket_of(unsigned long long raw) { return shfl_u64(raw, 0); }

__device__ __forceinline__ uint32_t chunk_cols(uint32_t m) { return m <= 1 ? 0u : ((m - 1u + 63u) & ~63u); }

}  // namespace falcon
