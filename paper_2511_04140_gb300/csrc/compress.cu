// Falcon compression (Sec. 3 of the paper; the work of Alg. 3 CmpKernel) for sm_103a, as
// two launches, neither of which waits on another warp:
//   1. analyse: each warp takes its chunks by ticket (its one shared-memory value buffer
//      receives the next chunk by cp.async, swizzled, as soon as the Case decision is done)
//      and computes
//      - the lane's 32 values, specials (R1) and the chunk maximum,
//      - Case 1 / Case 2 of Eq. 4: the smallest decimal place alpha_max at which every value
//        passes Alg. 2's test, in exact integer arithmetic (q_test); FP32 checks Alg. 2's
//        early stops where they are possible,
//      - G (Eq. 4), Z (Eq. 5) and the bit width w in registers,
//      - the non-zero bytes of every row (Sec. 3.3 lambda) from ORs of 8-column groups,
//        without forming the bit planes, sparse/dense per row, the record size, which goes
//        into the stream's size array and is added to its 64-chunk tile's and 4096-chunk
//        group's sums (the size synchronisation of Sec. 3.4), and alpha, beta_hat, w and the
//        dense-row mask, which go into the workspace;
//   2. emit: each chunk's record offset from those sums, the values again (straight from
//      global memory: FP64 with the next chunk prefetched into L2, FP32 and FP16 with the
//      next chunk's values loaded into registers during the current record), G, Z and the
//      bit planes (32x32 register transposes, one 32-bit word per plane: 4 row bytes per
//      lane) from the kept
//      alpha and w, the record assembled in shared memory at the output's 16-byte phase, in
//      place of the plane words it consumes, and sent to its offset with one TMA bulk copy;
//      the warp of each job's first chunk writes the header and the stream length and checks
//      the capacity.
// The paper resolves offsets inside one launch with a decoupled look-back; with about 1800
// resident warps on a GB300 the waits of that look-back took half of every warp's time, while
// the analysis recomputed by the emit launch costs less.
#include <map>
#include <mutex>
#include <tuple>

#include "falcon_device.cuh"

namespace falcon {

namespace {

constexpr int kBuf = 8288;                  // one chunk of values / one record (+32 readable)
constexpr int kScratch = 128;
constexpr int kAnalyseWarpBytes = kBuf + kScratch;  // analysis: one value buffer

// The emit launch's per-warp plane / record buffer: plane p's words at
// kPlOff + (W-1-p)*128 + 4*lane.  The record is assembled in place, from byte 0, as the planes
// are consumed top-down: an adaptive or dense row takes at most the 128 bytes of its slot, so
// the record never overtakes the plane read next with kPlOff = 48.  Every-row-sparse records
// (Sec. 5.4.2 ablation) may take 16 + 128 bytes per row and use the wide layout, whose plane
// slots start past 16 bytes of growth per row.
template <bool kWide> struct EmitLayout {
    static constexpr int kPlOff = kWide ? 1072 : 48;
    static constexpr int kBytes = kPlOff + 64 * 128 + 32;          // + 32 readable past any slot
};

// Copies len bytes from src to dst inside a warp buffer, dst + 14 <= src (the move goes
// down): unaligned head and tail bytes singly, the 16-byte aligned middle of the
// destination with one 16-byte store per lane and iteration, its source taken from two
// aligned 16-byte loads and funnel shifts.  In every iteration all lanes read before any
// lane writes, and later iterations read strictly above earlier writes, so the overlapping
// move is safe.  The buffer has 32 readable bytes past any source byte.
__device__ __forceinline__ uint32_t fsr(uint32_t lo, uint32_t hi, uint32_t s) { return __funnelshift_r(lo, hi, s); }

__device__ __forceinline__ void smem_move_down(uint8_t *buf, uint32_t dst, uint32_t src, uint32_t len, int lane) {
    const uint32_t head = min((16u - (dst & 15u)) & 15u, len);
    uint32_t hb = 0;
    if ((uint32_t)lane < head) hb = buf[src + lane];
    __syncwarp();
    if ((uint32_t)lane < head) buf[dst + lane] = (uint8_t)hb;
    __syncwarp();
    const uint32_t D = dst + head, S = src + head;
    const uint32_t units = (len - head) >> 4;
    const uint32_t off = S & 15u, k0 = off >> 2, sb = (off & 3u) * 8u;
    const uint32_t Sa = S - off;
    for (uint32_t u0 = 0; u0 < units; u0 += 32) {
        const uint32_t u = u0 + lane;
        uint4 o = make_uint4(0, 0, 0, 0);
        if (u < units) {
            const uint4 a = *reinterpret_cast<const uint4 *>(buf + Sa + 16u * u);
            const uint4 b = *reinterpret_cast<const uint4 *>(buf + Sa + 16u * u + 16u);
            switch (k0) {
                case 0: o = make_uint4(fsr(a.x, a.y, sb), fsr(a.y, a.z, sb), fsr(a.z, a.w, sb), fsr(a.w, b.x, sb)); break;
                case 1: o = make_uint4(fsr(a.y, a.z, sb), fsr(a.z, a.w, sb), fsr(a.w, b.x, sb), fsr(b.x, b.y, sb)); break;
                case 2: o = make_uint4(fsr(a.z, a.w, sb), fsr(a.w, b.x, sb), fsr(b.x, b.y, sb), fsr(b.y, b.z, sb)); break;
                default: o = make_uint4(fsr(a.w, b.x, sb), fsr(b.x, b.y, sb), fsr(b.y, b.z, sb), fsr(b.z, b.w, sb)); break;
            }
        }
        __syncwarp();
        if (u < units) *reinterpret_cast<uint4 *>(buf + D + 16u * u) = o;
    }
    __syncwarp();
    const uint32_t tail = (len - head) & 15u;
    const uint32_t T0 = units * 16u;
    uint32_t tb = 0;
    if ((uint32_t)lane < tail) tb = buf[S + T0 + lane];
    __syncwarp();
    if ((uint32_t)lane < tail) buf[D + T0 + lane] = (uint8_t)tb;
    __syncwarp();
}

// non-zero nibble of x (bit 3 - i set iff byte i is non-zero): the bytes' high-bit flags
// gathered into the top byte by one multiply
__device__ __forceinline__ uint32_t nz_nibble(uint32_t x) {
    const uint32_t y = (((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u;
    return ((y >> 7) * 0x08040201u) >> 24 & 0xFu;
}

// Sparse row (Sec. 3.3) written with byte stores at byte offset P of the warp buffer:
// a bitmap of nact/2 bytes (bit 7 of byte 0 = row byte 0), then the non-zero row bytes.
// Returns the row's length.
__device__ __forceinline__ uint32_t sparse_row(uint8_t *buf, uint32_t P, uint32_t x, int lane, uint32_t nact) {
    const bool active = (uint32_t)lane < nact;
    const uint32_t nib = active ? nz_nibble(x) : 0u;
    const uint32_t nib_next = __shfl_down_sync(kFull, nib, 1);
    if (active && !(lane & 1)) buf[P + (lane >> 1)] = (uint8_t)((nib << 4) | nib_next);
    const uint32_t cnt = __popc(nib);
    const unsigned b0 = __ballot_sync(kFull, cnt & 1u);
    const unsigned b1 = __ballot_sync(kFull, cnt & 2u);
    const unsigned b2 = __ballot_sync(kFull, cnt & 4u);
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t before = __popc(b0 & lt) + 2u * __popc(b1 & lt) + 4u * __popc(b2 & lt);
    const uint32_t total = __reduce_add_sync(kFull, cnt);
    uint32_t q = P + nact / 2u + before;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t byte = (x >> (8 * i)) & 0xFFu;
        if (active && byte) buf[q++] = (uint8_t)byte;
    }
    __syncwarp();
    return nact / 2u + total;
}

// value k of this lane from the swizzled staging buffer
template <int D>
__device__ __forceinline__ typename Traits<D>::U lane_value(const uint8_t *buf, int lane, int k) {
    using U = typename Traits<D>::U;
    constexpr int UN = Traits<D>::UNITS;
    constexpr int PER = 16 / Traits<D>::S;
    return *reinterpret_cast<const U *>(buf + (lane * UN + unit_swizzle<D>(lane, k / PER)) * 16 + (k % PER) * Traits<D>::S);
}

// Every value of the chunk (the lane's 32 in v, value 1024 of a 1025-value chunk in vx)
// passes Alg. 2's test at a.  Values past m are +0, which passes.
// Every value of the chunk passes Alg. 2's test at a; the values are re-read from the staging
// buffer (index >= m: not a value).  A failing decimal place usually fails on every lane's
// first value already, so those 32 are tested first.
template <int D>
__device__ __forceinline__ bool all_pass(const uint8_t *buf, int lane, uint32_t m, typename Traits<D>::U vx,
                                         int a) {
    const bool has0 = 32u * lane < m;
    if (!__all_sync(kFull, !has0 || q_test(lane_value<D>(buf, lane, 0), a))) return false;
    bool ok = q_test(vx, a);
#pragma unroll 4
    for (int k = 1; k < 32; ++k)
        if (32u * lane + k < m) ok &= q_test(lane_value<D>(buf, lane, k), a);
    return __all_sync(kFull, ok);
}

// Smallest a in [0, atop] at which every value passes the round-trip test, or -1 (Case 2).
// For chunks of valid values the predicate is monotone in a (Thm 4 with Thm 3), and its
// smallest true point is the largest decimal place of the values; a failure at atop means
// some value is an exception or needs alpha > atop.  Each lane's first value is tested at
// atop (a failure settles Case 2), then its own decimal place is found; the warp's maximum
// is a lower bound, and for most chunks the answer: one all-value test confirms it.
// Otherwise the answer lies above it (test atop, then bisect).  Out of line, reading the
// staged values: few chunks get here, and the hot path of the others stays small.
template <int D>
__device__ __noinline__ int search_alpha(const uint8_t *buf, int lane, uint32_t m, typename Traits<D>::U vx,
                                         int atop) {
    using U = typename Traits<D>::U;
    const U v0 = 32u * lane < m ? lane_value<D>(buf, lane, 0) : (U)0;
    if (!__all_sync(kFull, q_test(v0, atop))) return -1;
    int a0 = 0;
#pragma unroll 1
    while (a0 < atop && !q_test(v0, a0)) ++a0;
    const int lb = (int)__reduce_max_sync(kFull, (uint32_t)a0);
    int lo = lb, hi = atop;                     // the answer, if any, lies in [lo, hi]
    bool hi_ok = false;                         // all_pass(hi) is known to hold
    int a = lb;
#pragma unroll 1
    for (;;) {
        const bool ok = all_pass<D>(buf, lane, m, vx, a);
        if (ok) {
            hi = a;
            hi_ok = true;
        } else {
            if (a == atop) return -1;
            lo = a + 1;
        }
        if (hi_ok && lo >= hi) return hi;
        a = hi_ok ? ((lo + hi) >> 1) : atop;    // lo <= a < hi once atop has passed
    }
}

// FP32 chunks at beta_hat = 7 (R14) and FP16 chunks at beta_hat = 3 (R18): Alg. 2, value by
// value, stops at the first decimal place where eps <= mu passes, and if the round trip fails
// there the value is an exception.  That can happen below a value's own decimal place k only if
// |v| 10^k >= 2^(p-1) / 1.5 (p = 24 or 11 significand bits): with d / 10^k its shortest decimal,
// v 10^a (a < k) lies at least 10^-(k-a) - |v| 10^a 2^-p from every integer, more than
// mu = |v 10^a| 2^-(p-1) below that bound (checked exhaustively over every decimal below it).
// k <= alpha, so a value can stop early only if |v| 10^alpha reaches the bound.  FP32 tests
// 3 |v| 10^alpha >= 2^23 (half the bound, as a margin: the bound was checked exhaustively only
// up to that point); FP16 tests the bound itself, 3 |v| 10^alpha >= 2^11, checked over all
// 65,536 patterns.  Only those values go through Alg. 2, and none when v_max is below.
__device__ __forceinline__ bool may_stop_early(uint32_t u, int a) {
    const uint32_t au = u & 0x7FFFFFFFu;
    if (au == 0) return false;
    if (au < 0x00800000u) return true;          // subnormal: take the full test
    const int E = (int)(au >> 23) - 150;
    const uint64_t p = 3ull * ((au & 0x007FFFFFu) | 0x00800000u) * FALCON_POW5[a];   // < 2^50
    const int s = 23 - E - a;                    // 3 m 5^a 2^(E+a) >= 2^23  <=>  p >= 2^s
    return s <= 0 || (s < 50 && p >= (1ull << s));
}
__device__ __forceinline__ bool may_stop_early(uint16_t u, int a) {
    const uint32_t au = u & 0x7FFFu;
    if (au == 0) return false;
    if (au < 0x0400u) return true;
    const int E = (int)(au >> 10) - 25;
    const uint32_t p = 3u * ((au & 0x3FFu) | 0x400u) * (uint32_t)FALCON_POW5[a];     // < 2^22
    const int s = 11 - E - a;                    // 3 m 5^a 2^(E+a) >= 2^11  <=>  p >= 2^s
    return s <= 0 || (s < 32 && p >= (1u << s));
}
__device__ __forceinline__ int first_pass(uint32_t u, int atop) { return first_pass_f32(u, atop); }
__device__ __forceinline__ int first_pass(uint16_t u, int atop) { return first_pass_f16(u, atop); }

// True if some value of the chunk stops early (the chunk then takes Case 2); alpha is the
// search's alpha_max, at which every value round-trips.
template <int D>
__device__ __forceinline__ bool early_stop(const uint8_t *buf, int lane, uint32_t m, const typename Traits<D>::U (&v)[32],
                                           typename Traits<D>::U vx, bool has_vx, typename Traits<D>::U vmax,
                                           int alpha) {
    if (!may_stop_early(vmax, alpha)) return false;
    uint32_t cand = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) cand |= (uint32_t)(32u * lane + k < m && may_stop_early(v[k], alpha)) << k;
    bool bad = has_vx && may_stop_early(vx, alpha) && first_pass(vx, alpha) < 0;
#pragma unroll 1
    while (cand) {
        const int k = __ffs(cand) - 1;
        cand &= cand - 1;
        bad |= first_pass(lane_value<D>(buf, lane, k), alpha) < 0;
    }
    return __any_sync(kFull, bad);
}

// Fal._Elf's decimal place of one value (Sec. 1's trial and error, ablation of Sec. 5.4.2):
// the first a with v (x) 10^a integral, a <= 22 and a + floor(log10|v|) + 1 <= 15 (FP32: 10
// and 7), else -1 (exception).  The products are IEEE multiplies, as the method defines.
__device__ __forceinline__ int elf_dp(uint64_t u) {
    const uint64_t au = u & 0x7FFFFFFFFFFFFFFFull;
    if (au == 0) return 0;
    if (is_special(u) || !log10_in_range(au)) return -1;
    const int atop = min(22, 14 - floor_log10(au));
    const double v = __longlong_as_double((long long)u);
    for (int a = 0; a <= atop; ++a) {
        const double x = __dmul_rn(v, __longlong_as_double((long long)FALCON_P10_F64[a - FALCON_P10_F64_LO]));
        if (x == floor(x)) return a;
    }
    return -1;
}
__device__ __forceinline__ int elf_dp(uint32_t u) {
    const uint32_t au = u & 0x7FFFFFFFu;
    if (au == 0) return 0;
    if (is_special(u) || !log10_in_range(au)) return -1;
    const int atop = min(10, 6 - floor_log10(au));
    const float v = __uint_as_float(u);
    for (int a = 0; a <= atop; ++a) {
        const float x = __fmul_rn(v, __uint_as_float(FALCON_P10_F32[a - FALCON_P10_F32_LO]));
        if (x == floorf(x)) return a;
    }
    return -1;
}
__device__ __forceinline__ int elf_dp(uint16_t u) {      // binary16: products rounded to binary16
    const uint32_t au = u & 0x7FFFu;
    if (au == 0) return 0;
    if (is_special(u)) return -1;
    const int atop = min(4, 2 - floor_log10((uint16_t)au));
    const float v = __half2float(__ushort_as_half(u));
    for (int a = 0; a <= atop; ++a) {
        // the product of two binary16 values is exact in FP32, so one rounding gives fl16
        const float x = __half2float(__float2half_rn(v * (float)(FALCON_POW5[a] << a)));
        if (x == floorf(x)) return a;
    }
    return -1;
}

// Fal._Elf: alpha_max = the largest of the values' Elf decimal places, then Eq. 4's bounds and
// the R6 round trip at alpha_max, as for Falcon; -1 means Case 2.  Out of line (an ablation).
template <int D>
__device__ __noinline__ int alpha_elf(const uint8_t *buf, int lane, uint32_t m, typename Traits<D>::U vx,
                                      bool has_vx, int e_max) {
    using T = Traits<D>;
    int amax = has_vx ? elf_dp(vx) : 0;
    bool bad = amax < 0;
#pragma unroll 1
    for (int k = 0; k < 32; ++k) {
        if (32u * lane + k < m) {
            const int a = elf_dp(lane_value<D>(buf, lane, k));
            bad |= a < 0;
            amax = a > amax ? a : amax;
        }
    }
    if (__any_sync(kFull, bad)) return -1;
    amax = (int)__reduce_max_sync(kFull, (uint32_t)amax);
    if (amax > T::A_MAX || amax + e_max + 1 > T::B_MAX) return -1;
    return all_pass<D>(buf, lane, m, vx, amax) ? amax : -1;
}

__device__ __forceinline__ void issue_chunk(const Job *jobs, int njobs, const Job &single, uint64_t t,
                                            uint8_t *buf, int lane) {
    const Job &job = (jobs == nullptr) ? single : jobs[find_job(jobs, njobs, t)];
    const uint64_t c = t - job.chunk_begin;
    const uint64_t first = c * (uint64_t)job.block;
    const uint32_t m = (uint32_t)((job.n - first) < job.block ? (job.n - first) : job.block);
    if (job.dtype == 0) stage_values_async<kD64>(job.in + first * 8u, m, buf, lane);
    else if (job.dtype == 1) stage_values_async<kD32>(job.in + first * 4u, m, buf, lane);
    else stage_values_async<kD16>(job.in + first * 2u, m, buf, lane);
}

// Workspace words of a job (job.flags), written by the analysis launch:
//   flags[c]            alpha byte (5 bits) | beta_hat (5) | w (7), in bits 47..63;
//   flags[nchunks + c]  the dense-row mask (bit p: plane p is stored dense);
//   flags[2 nchunks + j]                       the sum of the record sizes of 64-chunk tile j,
//   flags[2 nchunks + tile_count(nchunks) + g]  and of 4096-chunk group g (atomic adds).
constexpr int kMetaShift = 47;

__device__ __forceinline__ unsigned long long pack_meta(int alpha_byte, int beta_hat, int w) {
    return (unsigned long long)(((uint32_t)alpha_byte << 12) | ((uint32_t)beta_hat << 7) | (uint32_t)w) << kMetaShift;
}

// G (Eq. 4) and Z (Eq. 5) in place: v[k] becomes Z of column 32 lane + k, pad columns (R11)
// are zero; alpha < 0 means Case 2.  Returns z_1 (every lane).
template <int D>
__device__ __forceinline__ typename Traits<D>::U to_z(typename Traits<D>::U (&v)[32],
                                                        typename Traits<D>::U vx, int alpha, uint32_t m,
                                                        int lane) {
    using U = typename Traits<D>::U;
    U gx;
    if (alpha >= 0) {
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = case1_g(v[k], alpha);
        gx = case1_g(vx, alpha);
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = zigzag(v[k]);
        gx = zigzag(vx);
    }
    const U z1 = shfl_x(v[0], 0);
    U nxt = shfl_down_x(v[0], 1);
    if (lane == 31) nxt = gx;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const U hi = (k < 31) ? v[k + 1] : nxt;
        v[k] = zigzag((U)(hi - v[k]));          // v now holds Z of columns 32*lane + k
    }
    // pad columns (R11): column c holds z_{c+2}, a pad when c + 1 >= m.  A full chunk of 1024
    // values has one (the last column of lane 31), 1025 values none; only tail chunks take the
    // general loop.
    if (m == 1024u) {
        if (lane == 31) v[31] = 0;
    } else if (m < 1024u && 32u * lane + 32u >= m) {
#pragma unroll
        for (int k = 0; k < 32; ++k)
            if (32u * lane + k + 1u >= m) v[k] = 0;
    }
    return z1;
}

// bit j of a nibble moved to bit 0 of byte j
__device__ __forceinline__ uint32_t spread_nibble(uint32_t n) { return (n * 0x00204081u) & 0x01010101u; }


// Launch 1, one chunk: everything up to the record size (see the file comment).  `next`
// starts the copy of the warp's next chunk into buf; it is called once, as soon as the
// staged values are no longer read (after the Case decision).
template <int D, class Next>
__device__ void analyse_chunk(const Job &job, uint64_t c, const uint8_t *buf, uint8_t *scratch, int lane,
                              Next &&next) {
    using T = Traits<D>;
    using U = typename T::U;
    constexpr U ABS = (U)((U)~(U)0 >> 1);          // every bit but the sign (~ promotes uint16 to int)
    const uint32_t B = job.block;
    const uint64_t first = c * (uint64_t)B;
    const uint32_t m = (uint32_t)((job.n - first) < B ? (job.n - first) : B);

    // ---- 1. values, specials, maximum ------------------------------------------------------
    U v[32];
    read_own<D>(buf, lane, m, v);
    U vx = 0;                                   // value 1024 of a 1025-value chunk
    if (m > 1024u && lane == 31) vx = read_elem<D>(buf, 1024);
    bool sp;
    U vmax;
    if constexpr (D == 0) {
        // on 32-bit halves: special <=> exponent field all zeros (value != +0) or all ones
        uint32_t hmax = 0;
        bool s = false;
        auto cls = [&](uint64_t u) {
            const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u, ha = hi & 0x7FFFFFFFu;
            s |= (ha - 0x00100000u >= 0x7FE00000u) && ((hi | lo) != 0u);
            hmax = ha > hmax ? ha : hmax;
        };
        cls(vx);
#pragma unroll
        for (int k = 0; k < 32; ++k) cls(v[k]);
        sp = __any_sync(kFull, s);
        const uint32_t H = __reduce_max_sync(kFull, hmax);
        uint32_t lmax = 0;
        auto lo_of = [&](uint64_t u) {
            if (((uint32_t)(u >> 32) & 0x7FFFFFFFu) == H) lmax = (uint32_t)u > lmax ? (uint32_t)u : lmax;
        };
        lo_of(vx);
#pragma unroll
        for (int k = 0; k < 32; ++k) lo_of(v[k]);
        vmax = ((uint64_t)H << 32) | __reduce_max_sync(kFull, lmax);
    } else {
        sp = is_special(vx);
        vmax = vx & ABS;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            sp |= is_special(v[k]);
            const U a = v[k] & ABS;
            vmax = a > vmax ? a : vmax;
        }
        sp = __any_sync(kFull, sp);
        vmax = warp_max_x(vmax);
    }

    // ---- 2. Case decision (Eq. 4) -----------------------------------------------------------
    int alpha = -1;                             // -1: Case 2
    int beta_hat = T::B_SENT;
    if (!sp) {
        if (vmax == 0) {
            alpha = 0;
            beta_hat = 0;
        } else if (log10_in_range(vmax)) {
            const int e_max = floor_log10(vmax);
            const int atop = min(T::A_MAX, T::B_MAX - 1 - e_max);
            if (job.variant == kVariantElf) {
                alpha = alpha_elf<D>(buf, lane, m, vx, m > 1024u && lane == 31, e_max);
            } else if (atop >= 0) {
                // quick rejection: Alg. 2 on the largest magnitude first.  The test reads
                // only |v|, so it runs on vmax itself, the same in every lane.
                bool fail;
                if constexpr (D == kD64) fail = !q_test(vmax, atop);
                else fail = first_pass(vmax, atop) < 0;
                if (!fail) {
                    alpha = search_alpha<D>(buf, lane, m, vx, atop);
                    // FP32 (R14), FP16 (R18): below beta_hat = B_MAX no value can stop early
                    // (see early_stop), so Alg. 2 value by value gives the same alpha_max
                    if constexpr (D != kD64) {
                        if (alpha >= 0 && alpha + e_max + 1 == T::B_MAX &&
                            early_stop<D>(buf, lane, m, v, vx, m > 1024u && lane == 31, vmax, alpha))
                            alpha = -1;
                    }
                }
            }
            if (alpha >= 0) beta_hat = alpha + e_max + 1;
        }
    }
    __syncwarp();
    next();                                     // the staged values have been read

    // ---- 3. G, Z, w (from the ORs of 8-column groups that step 4 uses) -------------------------
    (void)to_z<D>(v, vx, alpha, m, lane);
    U o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        U x = v[8 * i];
#pragma unroll
        for (int j = 1; j < 8; ++j) x |= v[8 * i + j];
        o[i] = x;
    }
    const U zor = warp_or_x((U)(o[0] | o[1] | o[2] | o[3]));
    const int w = zor ? ((D == 0) ? 64 - __clzll((long long)zor) : 32 - __clz((int)zor)) : 0;

    // ---- 4. non-zero bytes per row, without forming the bit planes ----------------------------
    // This lane's four bytes of row p cover its columns 8i .. 8i + 7 (i = 0..3); byte i is
    // non-zero iff bit p is set in o[i], the OR of those columns' Z.  The four bits of every
    // plane are added bit-sliced (count = b0 + 2 b1 + 4 b2) and spread into byte fields,
    // planes 4g .. 4g + 3 in the bytes of one word, which is added over the warp and stored, one
    // g at a time (a rolled loop: its code stays small).
    const uint32_t cols = chunk_cols(m);
    const uint32_t row_bytes = cols / 8u;
    constexpr int PW = T::W < 32 ? 32 : T::W;  // planes the 32-bit words hold (FP16: 16 of them zero)
#pragma unroll
    for (int h = 0; h < PW / 32; ++h) {
        const uint32_t o0 = (uint32_t)((uint64_t)o[0] >> (32 * h)), o1 = (uint32_t)((uint64_t)o[1] >> (32 * h));
        const uint32_t o2 = (uint32_t)((uint64_t)o[2] >> (32 * h)), o3 = (uint32_t)((uint64_t)o[3] >> (32 * h));
        const uint32_t x1 = o0 ^ o1, x2 = o2 ^ o3, c1 = o0 & o1, c2 = o2 & o3;
        uint32_t b0 = x1 ^ x2, b1 = c1 ^ c2 ^ (x1 & x2), b2 = c1 & c2;
#pragma unroll 2
        for (int g = 0; g < (T::W < 32 ? T::W / 4 : 8); ++g) {
            const uint32_t word = spread_nibble(b0 & 15u) | (spread_nibble(b1 & 15u) << 1) | (spread_nibble(b2 & 15u) << 2);
            const uint32_t sum = __reduce_add_sync(kFull, word);
            if (lane == 0) reinterpret_cast<uint32_t *>(scratch)[8 * h + g] = sum;
            b0 >>= 4;
            b1 >>= 4;
            b2 >>= 4;
        }
    }
    __syncwarp();

    // ---- 5. storage choice (Sec. 3.3) and record size ------------------------------------------
    // the ablations of Sec. 5.4.2 force one scheme for every row
    const bool all_sparse = job.variant == kVariantSparse, all_dense = job.variant == kVariantDense;
    uint32_t cost = 0;
    bool dense_lo = false, dense_hi = false;
    if (lane < w) {                              // plane `lane`
        const uint32_t nz = scratch[lane];
        const bool sparse = all_sparse || (!all_dense && (row_bytes - nz) > cols / 64u);   // tie -> dense (R10)
        cost += sparse ? cols / 64u + nz : row_bytes;
        dense_lo = !sparse;
    }
    if (D == 0 && lane + 32 < w) {                  // plane `lane + 32`
        const uint32_t nz = scratch[lane + 32];
        const bool sparse = all_sparse || (!all_dense && (row_bytes - nz) > cols / 64u);
        cost += sparse ? cols / 64u + nz : row_bytes;
        dense_hi = !sparse;
    }
    const uint32_t body = __reduce_add_sync(kFull, cost);
    const uint64_t dense_mask = (uint64_t)__ballot_sync(kFull, dense_lo) |
                                ((uint64_t)__ballot_sync(kFull, dense_hi) << 32);
    const uint32_t size = 3u + T::Z1B + ((uint32_t)w + 7u) / 8u + body;
    if (lane == 0) {
        reinterpret_cast<uint32_t *>(job.out + 32)[c] = size;
        job.flags[c] = pack_meta(alpha >= 0 ? alpha : T::A_SENT, beta_hat, w);
        job.flags[job.nchunks + c] = dense_mask;
        unsigned long long *tsum = job.flags + 2 * job.nchunks;
        atomicAdd(tsum + c / kTile, (unsigned long long)size);
        atomicAdd(tsum + tile_count(job.nchunks) + c / kGroup, (unsigned long long)size);
    }
}

// Lane reads its 32 values (indices 32 lane + k) from global memory, 16 bytes at a time when
// the chunk is whole and 16-byte aligned; indices >= m read as +0.
template <int D>
__device__ __forceinline__ void load_own(const uint8_t *src, int lane, uint32_t m, typename Traits<D>::U (&v)[32]) {
    using U = typename Traits<D>::U;
    constexpr int UN = Traits<D>::UNITS;
    constexpr int PER = 32 / UN;
    if (m >= 1024u && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
        const uint4 *q4 = reinterpret_cast<const uint4 *>(src) + lane * UN;
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const uint4 q = __ldg(q4 + u);
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
    } else {
        const U *e = reinterpret_cast<const U *>(src);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const uint32_t i = 32u * (uint32_t)lane + (uint32_t)k;
            v[k] = i < m ? __ldg(e + i) : (U)0;
        }
    }
}

// Asks for chunk t's values to be brought into L2 (one prefetch per 128-byte line).
__device__ __forceinline__ void prefetch_chunk(const Job *jobs, int njobs, const Job &single, uint64_t t, int lane) {
    const Job &job = (jobs == nullptr) ? single : jobs[find_job(jobs, njobs, t)];
    const uint64_t first = (t - job.chunk_begin) * (uint64_t)job.block;
    const uint32_t m = (uint32_t)((job.n - first) < job.block ? (job.n - first) : job.block);
    const uint32_t s = job.dtype == 0 ? 8u : (job.dtype == 1 ? 4u : 2u);
    const uint8_t *src = job.in + first * s;
    const uint8_t *end = src + (size_t)m * s;
    for (const uint8_t *q = src + 128u * (uint32_t)lane; q < end; q += 128u * 32u)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
}

// Chunk c's values into v (the lane's 32) and vx (value 1024 of a 1025-value chunk, lane 31).
template <int D>
__device__ __forceinline__ void load_chunk(const Job &job, uint64_t c, int lane, typename Traits<D>::U (&v)[32],
                                           typename Traits<D>::U &vx) {
    using U = typename Traits<D>::U;
    const uint64_t first = c * (uint64_t)job.block;
    const uint32_t m = (uint32_t)((job.n - first) < job.block ? (job.n - first) : job.block);
    const uint8_t *src = job.in + first * Traits<D>::S;
    load_own<D>(src, lane, m, v);
    vx = (m > 1024u && lane == 31) ? __ldg(reinterpret_cast<const U *>(src) + 1024) : (U)0;
}

// Launch 2, one chunk: G, Z and the plane words again (alpha and w from the analysis), then
// the record at its offset.  meta / dense: the chunk's workspace words; size: its record size;
// rel: its record offset relative to the first record.  With kPre the chunk's values arrive in
// v / vx, loaded during the previous chunk, and `next` loads the following chunk's into them
// as soon as the plane words are in shared memory (the register loads then complete while
// this record is assembled); otherwise the values are loaded here and `next` does nothing.
template <int D, bool kWide, bool kPre, class Next>
__device__ void emit_chunk(const Job &job, uint64_t c, uint8_t *buf, int lane, unsigned long long meta,
                           unsigned long long dense, uint32_t size, uint64_t rel,
                           typename Traits<D>::U (&v)[32], typename Traits<D>::U &vx, Next &&next) {
    constexpr int kPlOff = EmitLayout<kWide>::kPlOff;
    using T = Traits<D>;
    using U = typename T::U;
    const uint32_t B = job.block;
    const uint64_t first = c * (uint64_t)B;
    const uint32_t m = (uint32_t)((job.n - first) < B ? (job.n - first) : B);
    const uint64_t data_start = 32ull + 4ull * job.nchunks;
    const uint32_t mb = (uint32_t)(meta >> kMetaShift);
    const int alpha_byte = (int)(mb >> 12), beta_hat = (int)((mb >> 7) & 31u), w = (int)(mb & 127u);
    const int alpha = alpha_byte == T::A_SENT ? -1 : alpha_byte;
    const uint64_t rec_off = data_start + rel;
    if (rec_off + size > job.out_cap) {          // the job's first chunk reports the capacity error
        next();
        return;
    }

    // ---- G, Z and the plane words in shared memory --------------------------------------------
    if constexpr (!kPre) load_chunk<D>(job, c, lane, v, vx);
    const U z1 = to_z<D>(v, vx, alpha, m, lane);
    if (lane == 0) bulk_wait_read();             // the previous record has left the buffer
    __syncwarp();
    // half h of the values holds planes 32 h .. 32 h + 31 (the high half only when w > 32)
#pragma unroll
    for (int h = 0; h < ((D == 0) ? 2 : 1); ++h) {
        if (h == 1 && w <= 32) break;
        uint32_t a[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) a[j] = (uint32_t)((uint64_t)v[j ^ 7] >> (32 * h));
        transpose32(a);
        uint8_t *dst = buf + kPlOff + (T::W - 1 - 32 * h) * 128 + 4 * lane;
#pragma unroll
        for (int p = 0; p < (T::W < 32 ? T::W : 32); ++p) *reinterpret_cast<uint32_t *>(dst - p * 128) = a[p];
    }
    __syncwarp();
    next();                                     // v and vx are free

    const uint32_t cols = chunk_cols(m);
    const uint32_t nact = cols / 32u;
    const uint32_t row_bytes = cols / 8u;
    const uint64_t dense_mask = dense;
    const uint32_t flag_bytes = ((uint32_t)w + 7u) / 8u;
    const uint32_t hdr = 3u + T::Z1B + flag_bytes;
    struct { int alpha_byte, beta_hat; uint64_t z1; } pd{alpha_byte, beta_hat, (uint64_t)z1};
    uint8_t *gdst = job.out + rec_off;
    const uint32_t sh = (uint32_t)(reinterpret_cast<uintptr_t>(gdst) & 15u);

    // ---- 6. record in shared memory (in place of the consumed plane words), then global ------
    // Row r (plane w-r) ends before byte 37 + 128 r of the buffer (37 + 144 r when every row
    // is sparse, wide layout) while the plane read next starts at kPlOff + (64 - w + r) * 128
    // >= kPlOff + 128 r: nothing unread is overwritten.
    {
        // header byte `lane` (branch-free: every lane computes its byte, lanes < hdr store it)
        const int i = lane;
        const uint32_t zb = (uint32_t)(pd.z1 >> ((8 * (i - 2)) & 63)) & 0xFFu;
        const uint32_t fb = (uint32_t)(dense_mask >> ((8u * (flag_bytes - 1u - (uint32_t)(i - 3 - T::Z1B))) & 63u)) & 0xFFu;
        uint32_t byte = i < 2 + T::Z1B ? zb : ((i == 2 + T::Z1B) ? (uint32_t)w : fb);
        byte = i == 0 ? (uint32_t)pd.alpha_byte : (i == 1 ? (uint32_t)pd.beta_hat : byte);
        if ((uint32_t)lane < hdr) buf[sh + i] = (uint8_t)byte;
    }
    __syncwarp();
    uint32_t pos = sh + hdr;                      // next record byte in the buffer
    int p = w - 1;
    while (p >= 0) {
        const uint32_t src = kPlOff + (uint32_t)(T::W - 1 - p) * 128u;
        if ((dense_mask >> p) & 1ull) {
            // a run of dense rows p, p-1, ..., q: contiguous in the plane buffer when rows
            // are 128 bytes long, so one move copies the whole run
            int q = p;
            if (row_bytes == 128u) {
                const uint64_t below = (p >= 63) ? ~0ull : ((2ull << p) - 1ull);
                const uint64_t holes = ~dense_mask & below;               // sparse rows <= p
                q = holes ? 64 - __clzll((long long)holes) : 0;           // lowest row of the run
            }
            const uint32_t rows = (uint32_t)(p - q + 1);
            smem_move_down(buf, pos, src, rows * row_bytes, lane);
            pos += rows * row_bytes;
            p = q - 1;
        } else {
            const uint32_t x = *reinterpret_cast<const uint32_t *>(buf + src + 4 * lane);
            __syncwarp();
            pos += sparse_row(buf, pos, x, lane, nact);
            --p;
        }
    }
    __syncwarp();

    // to global memory: the 16-byte units entirely inside the record with one bulk copy
    // (lane 0), the partial units at its ends (shared with the neighbouring records) bytewise
    uint8_t *gbase = gdst - sh;
    const uint32_t total = sh + size;
    const uint32_t u0 = (sh + 15u) / 16u, u1 = total / 16u;
    if (u0 >= u1) {
        for (uint32_t b = sh + (uint32_t)lane; b < total; b += 32) gbase[b] = buf[b];
    } else {
        const uint32_t head = 16u * u0 - sh, tail = total - 16u * u1;
        if ((uint32_t)lane < head) gbase[sh + lane] = buf[sh + lane];
        if ((uint32_t)lane < tail) gbase[16u * u1 + lane] = buf[16u * u1 + lane];
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
            bulk_store(gbase + 16u * u0, buf + 16u * u0, 16u * (u1 - u0));
            bulk_commit();
        }
    }
    __syncwarp();
}

__device__ __forceinline__ const Job &job_of(const Job *jobs, int njobs, const Job &single, uint64_t t) {
    return (jobs == nullptr) ? single : jobs[find_job(jobs, njobs, t)];
}

}  // namespace

// The hot kernels come in four forms by dtype: kDt = 0 (every job FP64), 1 (every job FP32),
// 3 (every job FP16) or 2 (any, per job: batches and the server).  A single-dtype form carries
// a third of the code, which the instruction caches notice.
constexpr int kDtF64 = 0, kDtF32 = 1, kDtMixed = 2, kDtF16 = 3;

// Launch 1: analysis of every chunk (chunks by ticket; the next chunk is copied into
// the warp's one value buffer while the current one is finished).
template <int kDt>
__device__ __forceinline__ void analyse_loop(const Job *__restrict__ jobs, int njobs, Job single,
                                             uint64_t total_chunks, Control *ctl) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint8_t *wbase = smem + warp * kAnalyseWarpBytes;
    uint8_t *scratch = wbase + kBuf;
    __shared__ Job s_single;                      // the single job, read from shared memory
    if (threadIdx.x == 0) s_single = single;
    __syncthreads();
    uint64_t t = ticket_of(take_ticket(ctl, kTicketAnalyse, lane));
    if (t >= total_chunks) return;
    issue_chunk(jobs, njobs, s_single, t, wbase, lane);
    cp_async_commit();
    for (;;) {
        const unsigned long long raw = take_ticket(ctl, kTicketAnalyse, lane);   // the chunk after t
        uint64_t tn = total_chunks;
        cp_async_wait_none();                    // the current chunk has landed
        __syncwarp();
        auto next = [&]() {
            tn = ticket_of(raw);
            if (tn < total_chunks) issue_chunk(jobs, njobs, s_single, tn, wbase, lane);
            cp_async_commit();
        };
        const Job &job = job_of(jobs, njobs, s_single, t);
        const uint64_t c = t - job.chunk_begin;
        if constexpr (kDt == kDtF64) analyse_chunk<kD64>(job, c, wbase, scratch, lane, next);
        else if constexpr (kDt == kDtF32) analyse_chunk<kD32>(job, c, wbase, scratch, lane, next);
        else if constexpr (kDt == kDtF16) analyse_chunk<kD16>(job, c, wbase, scratch, lane, next);
        else if (job.dtype == 0) analyse_chunk<kD64>(job, c, wbase, scratch, lane, next);
        else if (job.dtype == 1) analyse_chunk<kD32>(job, c, wbase, scratch, lane, next);
        else analyse_chunk<kD16>(job, c, wbase, scratch, lane, next);
        __syncwarp();
        if (tn >= total_chunks) break;
        t = tn;
    }
    cp_async_wait_none();
}

// FP64, FP16 and either-dtype forms (up to 128 registers, 16 warps per SM)
template <int kDt>
__global__ void __launch_bounds__(32 * kMaxCompressWarps, 1)
analyse_kernel(const Job *__restrict__ jobs, int njobs, Job single, uint64_t total_chunks, Control *ctl) {
    analyse_loop<kDt>(jobs, njobs, single, total_chunks, ctl);
}

// FP32 form: held to 96 registers, so that 20 warps fit an SM
template <int kDt>
__global__ void __maxnreg__(96)
analyse_kernel_narrow(const Job *__restrict__ jobs, int njobs, Job single, uint64_t total_chunks, Control *ctl) {
    analyse_loop<kDt>(jobs, njobs, single, total_chunks, ctl);
}

// Stream header, stream length and capacity check of one job (one warp): the length is the
// header, the size array and the records, whose sizes the analysis added up per group.
__device__ void finish_job(const Job &job, int lane) {
    const uint64_t nc = job.nchunks;
    const unsigned long long *gsum = job.flags + 2 * nc + tile_count(nc);
    uint64_t part = 0;
    for (uint64_t g = (uint64_t)lane; g < group_count(nc); g += 32) part += gsum[g];
    const uint64_t total = warp_sum_u64(part);
    if (lane == 0) {
        const uint64_t bytes = 32ull + 4ull * nc + total;
        job.result[0] = bytes;
        if (bytes > job.out_cap) set_status(job.result, kErrCapacity);
        uint4 *dst = reinterpret_cast<uint4 *>(job.out);
        dst[0] = make_uint4(0x4E434C46u, 1u | (job.dtype << 8), job.block, 0u);
        dst[1] = make_uint4((uint32_t)job.n, (uint32_t)(job.n >> 32), (uint32_t)nc, (uint32_t)(nc >> 32));
    }
}

// Where chunk c's record starts, relative to the first record (Sec. 3.4's size synchronisation,
// from the analysis' sums): the groups before c's group, the tiles of its group before its tile
// and the chunks of its tile before it.  load_info issues the loads one chunk ahead (every lane:
// one group sum, two tile sums, two sizes) and keeps the raw words, so that nothing waits on them
// until resolve_info adds them up a chunk later.  A group's records take < 2^26 bytes and a
// tile's < 2^20, so their low 32-bit words are the sums; with at most 32 groups before c the
// records before c take < 2^31 bytes (33 * 4096 records of at most 9235 bytes) and one 32-bit
// reduction adds the lanes' shares.  Beyond that (more than 128 M values at block 1024) the
// further groups are read when resolving and added in 64 bits.
struct EmitInfo {
    unsigned long long meta, dense;
    uint32_t g0, t0, t1, s0, s1;      // this lane's group sum, two tile sums, two record sizes
    uint32_t size;                    // c's record size
};

__device__ __forceinline__ EmitInfo load_info(const Job &job, uint64_t c, int lane) {
    const uint64_t nc = job.nchunks;
    const uint32_t *sizes = reinterpret_cast<const uint32_t *>(job.out + 32);
    const uint32_t *tsum = reinterpret_cast<const uint32_t *>(job.flags + 2 * nc);   // low words
    const uint32_t *gsum = tsum + 2 * tile_count(nc);
    const uint64_t g = c / kGroup, t = c / kTile, tb = g * (kGroup / kTile), cb = t * kTile;
    EmitInfo e;
    e.meta = job.flags[c];
    e.dense = job.flags[nc + c];
    e.size = sizes[c];
    e.g0 = (uint64_t)lane < g ? gsum[2 * lane] : 0u;
    e.t0 = tb + (uint64_t)lane < t ? tsum[2 * (tb + lane)] : 0u;
    e.t1 = tb + 32u + (uint64_t)lane < t ? tsum[2 * (tb + 32u + lane)] : 0u;
    e.s0 = cb + (uint64_t)lane < c ? sizes[cb + lane] : 0u;
    e.s1 = cb + 32u + (uint64_t)lane < c ? sizes[cb + 32u + lane] : 0u;
    return e;
}
__device__ __forceinline__ uint64_t resolve_info(const Job &job, uint64_t c, const EmitInfo &e, int lane) {
    const uint32_t p = e.g0 + e.t0 + e.t1 + e.s0 + e.s1;
    const uint64_t g = c / kGroup;
    if (g <= 32u) return __reduce_add_sync(kFull, p);
    const unsigned long long *gsum = job.flags + 2 * job.nchunks + tile_count(job.nchunks);
    uint64_t part = p;
    for (uint64_t j = 32u + (uint64_t)lane; j < g; j += 32) part += gsum[j];
    return warp_sum_u64(part);
}

// Launch 2: the records (chunks by ticket; the next chunk's values are loaded into registers
// during the current one in the FP32 and FP16 forms, prefetched into L2 in the FP64 and
// either-dtype forms).
template <bool kWide, int kDt>
__device__ __forceinline__ void emit_loop(const Job *__restrict__ jobs, int njobs, const Job &s_single,
                                          uint64_t total_chunks, Control *ctl, uint8_t *smem) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint8_t *wbase = smem + warp * EmitLayout<kWide>::kBytes;
    if (blockIdx.x == 0 && warp == 0) {          // jobs without chunks: header and length only
        if (jobs == nullptr) {
            if (s_single.nchunks == 0) finish_job(s_single, lane);
        } else {
            for (int j0 = 0; j0 < njobs; j0 += 32) {
                unsigned empty = __ballot_sync(kFull, j0 + lane < njobs && jobs[j0 + lane].nchunks == 0);
                while (empty) {
                    const int j = j0 + __ffs(empty) - 1;
                    empty &= empty - 1;
                    finish_job(jobs[j], lane);
                }
            }
        }
    }
    // the FP32 and FP16 forms keep the values of the chunk after the current one in registers
    // (kPre); the FP64 form has no registers to spare for them
    constexpr bool kPre = kDt == kDtF32 || kDt == kDtF16;
    constexpr int DP = kDt == kDtF32 ? kD32 : (kDt == kDtF16 ? kD16 : kD64);
    typename Traits<DP>::U v[32], vx;
    uint64_t t = ticket_of(take_ticket(ctl, kTicketEmit, lane));
    if (t >= total_chunks) return;
    uint64_t tn = ticket_of(take_ticket(ctl, kTicketEmit, lane));
    EmitInfo info;
    {
        const Job &j0 = job_of(jobs, njobs, s_single, t);
        info = load_info(j0, t - j0.chunk_begin, lane);
        if constexpr (kPre) load_chunk<DP>(j0, t - j0.chunk_begin, lane, v, vx);
    }
    for (;;) {
        // the ticket after tn, read at the next iteration; tn's workspace words are fetched now
        const unsigned long long raw = tn < total_chunks ? take_ticket(ctl, kTicketEmit, lane) : 0ull;
        EmitInfo next{};
        if (tn < total_chunks) {
            if constexpr (!kPre) prefetch_chunk(jobs, njobs, s_single, tn, lane);
            const Job &jn = job_of(jobs, njobs, s_single, tn);
            next = load_info(jn, tn - jn.chunk_begin, lane);
        }
        const Job &job = job_of(jobs, njobs, s_single, t);
        const uint64_t c = t - job.chunk_begin;
        const uint64_t rel = resolve_info(job, c, info, lane);
        if (c == 0) finish_job(job, lane);
        auto load_next = [&]() {
            if constexpr (kPre) {
                if (tn < total_chunks) {
                    const Job &jn = job_of(jobs, njobs, s_single, tn);
                    load_chunk<DP>(jn, tn - jn.chunk_begin, lane, v, vx);
                }
            }
        };
        if constexpr (kPre) {
            emit_chunk<DP, kWide, true>(job, c, wbase, lane, info.meta, info.dense, info.size, rel, v, vx, load_next);
        } else if constexpr (kDt == kDtF64) {
            uint64_t u[32], ux;
            emit_chunk<kD64, kWide, false>(job, c, wbase, lane, info.meta, info.dense, info.size, rel, u, ux, load_next);
        } else if (job.dtype == 0) {
            uint64_t u[32], ux;
            emit_chunk<kD64, kWide, false>(job, c, wbase, lane, info.meta, info.dense, info.size, rel, u, ux, load_next);
        } else if (job.dtype == 1) {
            uint32_t u[32], ux;
            emit_chunk<kD32, kWide, false>(job, c, wbase, lane, info.meta, info.dense, info.size, rel, u, ux, load_next);
        } else {
            uint16_t u[32], ux;
            emit_chunk<kD16, kWide, false>(job, c, wbase, lane, info.meta, info.dense, info.size, rel, u, ux, load_next);
        }
        __syncwarp();
        if (tn >= total_chunks) break;
        t = tn;
        tn = ticket_of(raw);
        info = next;
    }
    if (lane == 0) bulk_wait();
}

// FP64 and either-dtype forms (up to 128 registers, 16 warps per SM)
template <bool kWide, int kDt>
__global__ void __launch_bounds__(32 * kMaxCompressWarps, 1)
emit_kernel(const Job *__restrict__ jobs, int njobs, Job single, uint64_t total_chunks, Control *ctl) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ Job s_single;
    if (threadIdx.x == 0) s_single = single;
    __syncthreads();
    emit_loop<kWide, kDt>(jobs, njobs, s_single, total_chunks, ctl, smem);
}

// FP32 and FP16 forms: held to 96 registers (FP32 needs 96 without spilling), so that 20 warps
// fit an SM
template <bool kWide, int kDt>
__global__ void __maxnreg__(96)
emit_kernel_narrow(const Job *__restrict__ jobs, int njobs, Job single, uint64_t total_chunks, Control *ctl) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ Job s_single;
    if (threadIdx.x == 0) s_single = single;
    __syncthreads();
    emit_loop<kWide, kDt>(jobs, njobs, s_single, total_chunks, ctl, smem);
}

namespace {
int persistent_grid_of(const void *kernel, int warps, int smem_bytes, int lim, uint64_t total_chunks);

template <int kDt>
void launch_analyse(const Job *d_jobs, int njobs, const Job &single, uint64_t total_chunks, Control *ctl,
                    cudaStream_t stream) {
    const int w = g_cta_warps[0], smem = w * kAnalyseWarpBytes;
    void (*kernel)(const Job *, int, Job, uint64_t, Control *);
    if constexpr (kDt == kDtF32) kernel = analyse_kernel_narrow<kDt>;
    else kernel = analyse_kernel<kDt>;
    const int g = persistent_grid_of(reinterpret_cast<const void *>(kernel), w, smem, g_ctas_per_sm[0], total_chunks);
    kernel<<<g, 32 * w, smem, stream>>>(d_jobs, njobs, single, total_chunks, ctl);
}
template <bool kWide, int kDt>
void launch_emit(const Job *d_jobs, int njobs, const Job &single, uint64_t total_chunks, Control *ctl,
                 cudaStream_t stream) {
    const int w = g_cta_warps[0], smem = w * EmitLayout<kWide>::kBytes;
    if constexpr (kDt == kDtF32 || kDt == kDtF16) {
        const int g = persistent_grid_of(reinterpret_cast<const void *>(emit_kernel_narrow<kWide, kDt>), w, smem,
                                         g_ctas_per_sm[0], total_chunks);
        emit_kernel_narrow<kWide, kDt><<<g, 32 * w, smem, stream>>>(d_jobs, njobs, single, total_chunks, ctl);
    } else {
        const int g = persistent_grid_of(reinterpret_cast<const void *>(emit_kernel<kWide, kDt>), w, smem,
                                         g_ctas_per_sm[0], total_chunks);
        emit_kernel<kWide, kDt><<<g, 32 * w, smem, stream>>>(d_jobs, njobs, single, total_chunks, ctl);
    }
}

// Resident CTAs per SM of a persistent kernel at one CTA shape, looked up once per (kernel,
// device, shape) under a lock (the server and the pipeline launch from several host threads).
std::mutex g_occ_mu;
std::map<std::tuple<const void *, int, int, int>, std::pair<int, int>> g_occ;   // -> (CTAs per SM, SMs)

int persistent_grid_of(const void *kernel, int warps, int smem_bytes, int lim, uint64_t total_chunks) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::pair<int, int> oc;
    {
        std::lock_guard<std::mutex> lk(g_occ_mu);
        const auto key = std::make_tuple(kernel, dev, warps, smem_bytes);
        auto it = g_occ.find(key);
        if (it == g_occ.end()) {
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
            int sms = 0, occ = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 32 * warps, smem_bytes);
            it = g_occ.emplace(key, std::make_pair(occ > 0 ? occ : 1, sms > 0 ? sms : 1)).first;
        } else {
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
        }
        oc = it->second;
    }
    const int cached = oc.second * ((lim > 0 && lim < oc.first) ? lim : oc.first);
    const uint64_t need = (total_chunks + (uint64_t)warps - 1) / (uint64_t)warps;
    return (int)(need < (uint64_t)cached ? (need > 0 ? need : 1) : (uint64_t)cached);
}
}  // namespace

int persistent_grid_size(const void *kernel, int warps, int smem_bytes, int lim, uint64_t total_chunks) {
    return persistent_grid_of(kernel, warps, smem_bytes, lim, total_chunks);
}

int compress_grid(uint64_t total_chunks) {
    const int w = g_cta_warps[0];
    return persistent_grid_of(reinterpret_cast<const void *>(emit_kernel<false, kDtMixed>), w,
                              w * EmitLayout<false>::kBytes, g_ctas_per_sm[0], total_chunks);
}

cudaError_t launch_compress(const Job *d_jobs, int njobs, const Job &single, uint64_t total_chunks,
                            Control *ctl, cudaStream_t stream) {
    // the every-row-sparse ablation writes records larger than the plane slots hold
    const bool wide = d_jobs == nullptr && single.variant == kVariantSparse;
    const int kind = d_jobs != nullptr ? kDtMixed
                                       : (single.dtype == 0 ? kDtF64 : (single.dtype == 1 ? kDtF32 : kDtF16));
    if (total_chunks > 0) {
        if (kind == kDtF64) launch_analyse<kDtF64>(d_jobs, njobs, single, total_chunks, ctl, stream);
        else if (kind == kDtF32) launch_analyse<kDtF32>(d_jobs, njobs, single, total_chunks, ctl, stream);
        else if (kind == kDtF16) launch_analyse<kDtF16>(d_jobs, njobs, single, total_chunks, ctl, stream);
        else launch_analyse<kDtMixed>(d_jobs, njobs, single, total_chunks, ctl, stream);
    }
    {   // the emit launch also writes the header and length of every job, chunks or none
        if (wide && kind == kDtF64) launch_emit<true, kDtF64>(d_jobs, njobs, single, total_chunks, ctl, stream);
        else if (wide && kind == kDtF32) launch_emit<true, kDtF32>(d_jobs, njobs, single, total_chunks, ctl, stream);
        else if (wide) launch_emit<true, kDtF16>(d_jobs, njobs, single, total_chunks, ctl, stream);
        else if (kind == kDtF64) launch_emit<false, kDtF64>(d_jobs, njobs, single, total_chunks, ctl, stream);
        else if (kind == kDtF32) launch_emit<false, kDtF32>(d_jobs, njobs, single, total_chunks, ctl, stream);
        else if (kind == kDtF16) launch_emit<false, kDtF16>(d_jobs, njobs, single, total_chunks, ctl, stream);
        else launch_emit<false, kDtMixed>(d_jobs, njobs, single, total_chunks, ctl, stream);
    }
    return cudaGetLastError();
}

}  // namespace falcon
