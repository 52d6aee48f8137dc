// Falcon decompression (Sec. 4 of the paper) for sm_103a: two launches per call.
//
// 1. offsets_kernel: the chunk-size array is read and its exclusive prefix (the chunk
//    offset array) is written to the workspace - the step Sec. 4 performs first.
// 2. decompress_kernel: persistent; each warp takes its chunks by ticket (one atomic add each; no
//    ordering constraint remains).  Each warp has one record buffer: the cp.async of its
//    next record starts as soon as the current one has been expanded into the plane buffer;
//    offsets are loaded one step earlier still.  Decoding a record:
//      a. header and flags; a walk over the sparse rows' bitmaps gives every row's
//         position; sparse rows are expanded into their 128-byte plane slots,
//      b. runs of dense rows are copied into their slots (16-byte funnel-shifted moves), all
//         plane words are gathered into registers from fixed slot addresses, two 32x32
//         transposes give Z, unzigzag + warp scan give G (inverse Eq. 5), Case 1 divides by
//         10^alpha (correctly rounded) and Case 2 undoes the zigzag of the IEEE bits
//         (inverse Eq. 4),
//      c. values are staged (swizzled) and written with coalesced 16-byte stores.
// Every read of a record is bounds-checked against its size; a malformed record sets
// FALCON_ERR_CORRUPT and writes nothing.
#include "falcon.h"
#include "falcon_device.cuh"

namespace falcon {

namespace {

// Per-warp buffers of a value kind: one record at a 0..15 byte phase + 16 readable bytes (an
// FP64 record is at most 19 + 64 * 144 = 9235 bytes, an FP32 one 11 + 32 * 144 = 4619, an FP16
// one 7 + 16 * 144 = 2311: every row sparse without a zero byte, bitmap + 128 bytes), then W
// plane slots of 128 bytes and 64 u16 sparse-byte totals.  The narrow kinds' smaller buffers
// let more warps stay resident.
template <int D> struct DecLayout {
    static constexpr int kBuf = D == kD64 ? 9280 : (D == kD32 ? 4672 : 2368);
    static constexpr int kPlane = Traits<D>::W * 128 + 128;
    static constexpr int kWarpBytes = kBuf + kPlane;
};

// Byte-permute selector that spreads a lane's compacted non-zero bytes over its four row
// bytes, by bitmap nibble n: row byte i (nibble bit 3 - i) takes the next compacted byte if
// the bit is set, else a zero byte (selector 4, the zero operand).
__shared__ uint32_t s_expand_sel[16];

__device__ __forceinline__ void init_expand_sel() {
    if (threadIdx.x < 16) {
        const uint32_t n = threadIdx.x;
        uint32_t sel = 0, r = 0;
        for (int i = 0; i < 4; ++i) {
            if ((n >> (3 - i)) & 1u) sel |= (r++) << (4 * i);
            else sel |= 4u << (4 * i);
        }
        s_expand_sel[n] = sel;
    }
}        // one record buffer, one plane buffer

// fl(fl(g) / 10^a) with IEEE FP64 operations, as the decoder defines it for any g; the hot
// path takes div_pow10_exact for |g| < 2^53 (every g an encoder writes: |g| < 10^15).
__device__ __forceinline__ double div_pow10(int64_t g, int a) {
    return __ddiv_rn(__ll2double_rn(g), __longlong_as_double((long long)FALCON_P10_F64[a - FALCON_P10_F64_LO]));
}
__device__ __forceinline__ float div_pow10(int32_t g, int a) {
    return __fdiv_rn(__int2float_rn(g), __uint_as_float(FALCON_P10_F32[a - FALCON_P10_F32_LO]));
}

// number of set bits of a 4-bit value, with plain integer operations
__device__ __forceinline__ uint32_t nibble_count(uint32_t n) {
    const uint32_t x = n - ((n >> 1) & 5u);
    return (x & 3u) + (x >> 2);
}

__device__ __forceinline__ const Job &job_of(const Job *jobs, int njobs, const Job &single, uint64_t t) {
    return (jobs == nullptr) ? single : jobs[find_job(jobs, njobs, t)];
}

// Offset (within the stream) and size of the record of ticket t: the loads are issued early
// (locate), the offset is added up when the record is fetched (resolve).
struct Loc {
    uint64_t t;
    uint64_t rec_off;
    uint32_t size;
    ChunkPos pos;
};

__device__ __forceinline__ Loc locate(const Job *jobs, int njobs, const Job &single, uint64_t t, int lane) {
    const Job &job = job_of(jobs, njobs, single, t);
    const uint64_t c = t - job.chunk_begin;
    Loc l;
    l.t = t;
    l.pos = load_pos(reinterpret_cast<const uint32_t *>(job.in + 32), job.flags, c, lane);
    l.size = l.pos.size;
    l.rec_off = 0;
    return l;
}

__device__ __forceinline__ void resolve(const Job *jobs, int njobs, const Job &single, Loc &l) {
    const Job &job = job_of(jobs, njobs, single, l.t);
    l.rec_off = 32ull + 4ull * job.nchunks + resolve_pos(l.pos);
}

// Largest valid record of a chunk of m values: header, flags, and w = W rows of at most
// cols/64 + cols/8 bytes (a sparse row with no zero byte).
__device__ __forceinline__ uint32_t max_record(uint32_t m, uint32_t dtype) {
    const uint32_t W = dtype == 0 ? 64u : (dtype == 1 ? 32u : 16u);
    return 3u + W / 8u + W / 8u + W * (chunk_cols(m) / 8u + chunk_cols(m) / 64u);
}

// Starts the cp.async of a record into rbuf; returns false if its location is invalid.
__device__ __forceinline__ bool issue_record(const Job &job, const Loc &l, uint8_t *rbuf, int lane) {
    const uint64_t c = l.t - job.chunk_begin;
    const uint64_t first = c * (uint64_t)job.block;
    const uint32_t m = (uint32_t)((job.n - first) < job.block ? (job.n - first) : job.block);
    const uint32_t z1b = job.dtype == 0 ? 8u : (job.dtype == 1 ? 4u : 2u);
    if (l.size < 3u + z1b || l.size > max_record(m, job.dtype) || l.rec_off + l.size > job.in_bytes) return false;
    const uint8_t *gsrc = job.in + l.rec_off;
    const uint32_t sh = (uint32_t)(reinterpret_cast<uintptr_t>(gsrc) & 15u);
    const uint8_t *gbase = gsrc - sh;                       // >= job.in (16-byte aligned)
    const uint8_t *gend = job.in + job.in_bytes;
    const uint32_t units = (sh + l.size + 15u) / 16u;
    const uint32_t base = smem_addr(rbuf);
    for (uint32_t u = lane; u < units; u += 32) {
        const uint8_t *src = gbase + 16u * u;
        if (src + 16 <= gend) cp_async16(base + 16u * u, src);
        else
            for (uint32_t b = 0; b < 16u && src + b < gend; ++b) rbuf[16u * u + b] = src[b];
    }
    return true;
}

// Copies len bytes from any byte address of a shared buffer to a 16-byte aligned one in
// another buffer: one 16-byte store per lane and unit, built from two aligned 16-byte loads
// and funnel shifts, then the tail bytes singly.  The source buffer has 16 readable bytes past
// the copied bytes.
__device__ __forceinline__ void copy_to_planes(uint8_t *dst, const uint8_t *src, uint32_t len, int lane) {
    const uintptr_t sa = reinterpret_cast<uintptr_t>(src);
    const uint32_t off = (uint32_t)(sa & 15u), k0 = off >> 2, sb = (off & 3u) * 8u;
    const uint4 *S = reinterpret_cast<const uint4 *>(sa - off);
    const uint32_t units = len >> 4;
    for (uint32_t u = (uint32_t)lane; u < units; u += 32) {
        const uint4 a = S[u], b = S[u + 1];
        uint4 o;
        switch (k0) {
            case 0: o = make_uint4(__funnelshift_r(a.x, a.y, sb), __funnelshift_r(a.y, a.z, sb), __funnelshift_r(a.z, a.w, sb), __funnelshift_r(a.w, b.x, sb)); break;
            case 1: o = make_uint4(__funnelshift_r(a.y, a.z, sb), __funnelshift_r(a.z, a.w, sb), __funnelshift_r(a.w, b.x, sb), __funnelshift_r(b.x, b.y, sb)); break;
            case 2: o = make_uint4(__funnelshift_r(a.z, a.w, sb), __funnelshift_r(a.w, b.x, sb), __funnelshift_r(b.x, b.y, sb), __funnelshift_r(b.y, b.z, sb)); break;
            default: o = make_uint4(__funnelshift_r(a.w, b.x, sb), __funnelshift_r(b.x, b.y, sb), __funnelshift_r(b.y, b.z, sb), __funnelshift_r(b.z, b.w, sb)); break;
        }
        *reinterpret_cast<uint4 *>(dst + 16u * u) = o;
    }
    const uint32_t tail = len & 15u;
    if ((uint32_t)lane < tail) dst[16u * units + lane] = src[16u * units + lane];
}

// `next` starts the copy of the warp's next record into rbuf; it is called exactly once, as
// soon as this record has been read completely.
// A value's exact FP64 value, and its key in IEEE 754 totalOrder (for min / max of non-NaN values).
__device__ __forceinline__ double value_f64(uint64_t b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ double value_f64(uint32_t b) { return (double)__uint_as_float(b); }
__device__ __forceinline__ double value_f64(uint16_t b) { return (double)__half2float(__ushort_as_half(b)); }
__device__ __forceinline__ uint64_t order_key(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// kAgg (analytics on compressed data): instead of storing the values, the warp adds them up
// (NaN count, totalOrder min / max, their sum: each lane its 32 values in index order, then a
// butterfly over the lanes, identical in every lane since FP addition commutes); the chunk's
// sum goes to sums[c], the rest into the control block by atomics.
template <int D, bool kAgg, class Next>
__device__ void decode_chunk(const Job &job, const Loc &l, bool loc_ok, const uint8_t *rbuf, uint8_t *pbuf,
                             int lane, Next &&next, Control *ctl) {
    using T = Traits<D>;
    using U = typename T::U;

    const uint64_t c = l.t - job.chunk_begin;
    const uint32_t B = job.block;
    const uint64_t first = c * (uint64_t)B;
    const uint32_t m = (uint32_t)((job.n - first) < B ? (job.n - first) : B);
    const uint32_t cols = chunk_cols(m);
    const uint32_t nact = cols / 32u;
    const uint32_t row_bytes = cols / 8u;
    const uint32_t size = l.size;
    const uint32_t sh = (uint32_t)(reinterpret_cast<uintptr_t>(job.in + l.rec_off) & 15u);
    const uint8_t *rec = rbuf + sh;
    // plane p lives in slot W - 1 - p of pbuf: slot addresses are written planes + (63 - p) * 128
    uint8_t *planes = pbuf - (64 - T::W) * 128;
    uint16_t *rowpos = reinterpret_cast<uint16_t *>(pbuf + T::W * 128);

    // ---- a. header, flags, row positions; sparse rows expanded ---------------------------
    bool bad = !loc_ok;
    uint32_t alpha = 0, beta_hat = 0, w = 0, pos = 0;
    U z1 = 0;
    uint64_t dense_mask = 0;
    if (!bad) {
        alpha = rec[0];
        beta_hat = rec[1];
#pragma unroll
        for (int i = 0; i < T::Z1B; ++i) z1 |= (U)rec[2 + i] << (8 * i);
        w = rec[2 + T::Z1B];
        const uint32_t flag_bytes = (w + 7u) / 8u;
        pos = 3u + T::Z1B + flag_bytes;
        if (w > (uint32_t)T::W || (m <= 1u && w != 0u) || pos > size) bad = true;
        else
            for (uint32_t i = 0; i < flag_bytes; ++i) dense_mask = (dense_mask << 8) | rec[3 + T::Z1B + i];
    }
    const bool active = (uint32_t)lane < nact;
    const uint32_t bm_bytes = nact / 2u;
    const uint32_t hdr = pos;
    const uint64_t wmask = (w >= 64u) ? ~0ull : ((1ull << w) - 1ull);
    // Sparse rows only (top to bottom): a sparse row's position is the header, the dense rows
    // above it (row_bytes each) and the sparse rows above it.  Dense rows need no walk.  No
    // position is checked here: a row takes at most 16 + 128 bytes, so every read stays in the
    // record buffer whatever the bytes say, and the size check after the walk (every row's
    // bytes add up to the record size) rejects a malformed record before anything is stored.
    uint64_t sparse = bad ? 0ull : (~dense_mask & wmask);
    uint32_t sparse_sum = 0, walked = 0;       // sparse rows above the current one
#pragma unroll 1
    while (sparse) {
        const int p = 63 - __clzll((long long)sparse);
        sparse &= ~(1ull << p);
        // rows above p: w - 1 - p, of which `walked` are sparse
        const uint32_t spos = hdr + row_bytes * (w - 1u - (uint32_t)p - walked) + sparse_sum;
        ++walked;
        uint32_t nib = 0;
        if (active) {
            const uint32_t byte = rec[spos + (lane >> 1)];
            nib = (lane & 1) ? (byte & 0xFu) : (byte >> 4);
        }
        const uint32_t cnt = nibble_count(nib);
        const unsigned b0 = __ballot_sync(kFull, cnt & 1u);
        const unsigned b1 = __ballot_sync(kFull, cnt & 2u);
        const unsigned b2 = __ballot_sync(kFull, cnt & 4u);
        const unsigned lt = (1u << lane) - 1u;
        const uint32_t before = __popc(b0 & lt) + 2u * __popc(b1 & lt) + 4u * __popc(b2 & lt);
        const uint32_t nnz = __reduce_add_sync(kFull, cnt);
        // the lane's non-zero bytes start at record byte spos + bm_bytes + before: load the
        // four bytes from there (two aligned words) and put each in its place with one byte
        // permute (selector by the bitmap nibble)
        const uint32_t qa = sh + spos + bm_bytes + before;
        const uint32_t *wq = reinterpret_cast<const uint32_t *>(rbuf + (qa & ~3u));
        const uint32_t word = __funnelshift_r(wq[0], wq[1], (qa & 3u) * 8u);
        const uint32_t x = __byte_perm(word, 0u, s_expand_sel[nib]);
        *reinterpret_cast<uint32_t *>(planes + (63 - p) * 128 + 4 * lane) = x;
        sparse_sum += bm_bytes + nnz;
        if (lane == 0) rowpos[p] = (uint16_t)sparse_sum;   // sparse bytes through row p
    }
    if (!bad && hdr + row_bytes * (uint32_t)__popcll(dense_mask & wmask) + sparse_sum != size) bad = true;
    if (bad) {
        if (lane == 0) set_status(job.result, kErrCorrupt);
        __syncwarp();
        next();
        return;
    }
    __syncwarp();

    // ---- b. dense runs copied into the plane slots (plane p: slot 63 - p, 128 bytes, in
    //      record order), then every plane word gathered with one aligned load ---------------
    {
        uint64_t dm = dense_mask & wmask;
#pragma unroll 1
        while (dm) {
            const int p = 63 - __clzll((long long)dm);
            const uint64_t below = (p >= 63) ? ~0ull : ((2ull << p) - 1ull);
            const uint64_t holes = ~dense_mask & below;
            const int q = (row_bytes == 128u) ? (holes ? 64 - __clzll((long long)holes) : 0) : p;
            const uint64_t above = (p >= 63) ? 0ull : (wmask & ~((2ull << p) - 1ull));
            const uint64_t sp_above = ~dense_mask & above;
            // sparse bytes above p: the running total at the lowest sparse row above p
            const uint32_t sbytes = sp_above ? (uint32_t)rowpos[__ffsll((long long)sp_above) - 1] : 0u;
            const uint32_t rp = hdr + row_bytes * (uint32_t)__popcll(dense_mask & above) + sbytes;
            copy_to_planes(planes + (63 - p) * 128, rec + rp, (uint32_t)(p - q + 1) * row_bytes, lane);
            dm &= (q > 0) ? ((1ull << q) - 1ull) : 0ull;
        }
    }
    __syncwarp();
    next();                                       // the record has been read
    // Slots of planes >= w hold stale bytes: they are masked off after each transpose (bit p
    // of every value), one AND per value instead of a select per word.  Lanes >= nact (tail
    // chunks) gather stale words too; their columns lie past the chunk's values and are never
    // stored, and they only feed the scan of later lanes.
    auto plane_word = [&](int p) -> uint32_t {
        return *reinterpret_cast<const uint32_t *>(planes + (63 - p) * 128 + 4 * lane);
    };
    U d[32];
    if constexpr (D == 0) {
        if (w > 32) {
            uint32_t a[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) a[i] = plane_word(i + 32);
            transpose32(a);
            const uint32_t keep = w >= 64 ? ~0u : ((1u << (w - 32)) - 1u);
#pragma unroll
            for (int k = 0; k < 32; ++k) d[k] = (U)(a[k ^ 7] & keep) << 32;
        } else {
#pragma unroll
            for (int k = 0; k < 32; ++k) d[k] = 0;
        }
    }
    {
        uint32_t a[32];
#pragma unroll
        for (int p = 0; p < 32; ++p) a[p] = p < T::W ? plane_word(p) : 0u;    // FP16: 16 planes
        transpose32(a);
        const uint32_t keep = w >= 32 ? ~0u : ((1u << w) - 1u);
        if constexpr (D == 0) {
#pragma unroll
            for (int k = 0; k < 32; ++k) d[k] |= (U)(a[k ^ 7] & keep);
        } else {
#pragma unroll
            for (int k = 0; k < 32; ++k) d[k] = (U)(a[k ^ 7] & keep);
        }
    }
    U run = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) { run += unzigzag(d[k]); d[k] = run; }
    U lane_off;
    if constexpr (D == 0) lane_off = warp_exclusive_u64(run, lane);
    else lane_off = (U)warp_exclusive_u64((uint64_t)run, lane);
    const U gbase = z1 + lane_off;               // G of value 32*lane + k + 1 = gbase + d[k]
    const bool case1 = alpha <= (uint32_t)T::A_MAX && beta_hat <= (uint32_t)T::B_MAX;
    if (case1) {
        if constexpr (D == 0) {
            // |g| >= 2^53 only in streams no encoder writes: then every value takes the FP64 path
            bool big = false;
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const uint64_t gk = gbase + d[k];
                big |= (gk + (1ull << 53)) > (1ull << 54);          // |g| > 2^53
            }
            if (__any_sync(kFull, big)) {
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    d[k] = (U)__double_as_longlong(div_pow10((int64_t)(gbase + d[k]), (int)alpha));
            } else {
#pragma unroll
                for (int k = 0; k < 32; ++k) d[k] = div_pow10_exact((int64_t)(gbase + d[k]), (int)alpha);
            }
        } else if constexpr (D == kD32) {
#pragma unroll
            for (int k = 0; k < 32; ++k) d[k] = (U)__float_as_uint(div_pow10((int32_t)(gbase + d[k]), (int)alpha));
        } else {
            // fl16(g / 10^a) as fl16(fl32(g / 10^a)): exact for every 16-bit g and a <= 4 (the
            // second rounding never lands on a different value; checked for all 327,680 inputs)
            const float p = __uint_as_float(FALCON_P10_F32[alpha - FALCON_P10_F32_LO]);
#pragma unroll
            for (int k = 0; k < 32; ++k)
                d[k] = __half_as_ushort(__float2half_rn(__fdiv_rn((float)(int16_t)(U)(gbase + d[k]), p)));
        }
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) d[k] = unzigzag((U)(gbase + d[k]));
    }
    U v0;
    if (case1) {
        if constexpr (D == 0) {
            const uint64_t g1 = z1;
            v0 = ((g1 + (1ull << 53)) > (1ull << 54)) ? (U)__double_as_longlong(div_pow10((int64_t)g1, (int)alpha))
                                                       : div_pow10_exact((int64_t)g1, (int)alpha);
        } else if constexpr (D == kD32) {
            v0 = (U)__float_as_uint(div_pow10((int32_t)z1, (int)alpha));
        } else {
            v0 = __half_as_ushort(__float2half_rn(
                __fdiv_rn((float)(int16_t)z1, __uint_as_float(FALCON_P10_F32[alpha - FALCON_P10_F32_LO]))));
        }
    } else {
        v0 = unzigzag(z1);
    }
    // shift by one so that lane l holds values 32l .. 32l+31 (value 1024 stays in vx)
    U carry = shfl_up_x(d[31], 1);
    if (lane == 0) carry = v0;
    const U vx = d[31];
#pragma unroll
    for (int k = 31; k > 0; --k) d[k] = d[k - 1];
    d[0] = carry;
    __syncwarp();                                 // plane words consumed

    if constexpr (kAgg) {
        // keys in the values' own width (IEEE order = unsigned order of the keys), widened to
        // FP64 keys once per chunk
        constexpr U SIGN = (U)((U)1 << (T::W - 1));
        constexpr U ABSM = (U)(SIGN - 1u);
        constexpr U INF = (U)(D == kD64 ? 0x7FF0000000000000ull : (D == kD32 ? 0x7F800000ull : 0x7C00ull));
        uint32_t nan = 0;
        U kmin = (U)~(U)0, kmax = 0;
        double sum = -0.0;                        // -0 + x == x for every x, -0 + -0 == -0
        auto take = [&](U b) {
            if ((U)(b & ABSM) > INF) { ++nan; return; }
            const U key = (b & SIGN) ? (U)~b : (U)(b | SIGN);
            kmin = key < kmin ? key : kmin;
            kmax = key > kmax ? key : kmax;
            sum = __dadd_rn(sum, value_f64(b));
        };
#pragma unroll
        for (int k = 0; k < 32; ++k)
            if (32u * (uint32_t)lane + (uint32_t)k < m) take(d[k]);
        if (m > 1024u && lane == 31) take(vx);
        nan = __reduce_add_sync(kFull, nan);
        if constexpr (D == kD64) {
            kmin = ~warp_max_u64(~kmin);
            kmax = warp_max_u64(kmax);
        } else {
            kmin = (U)__reduce_min_sync(kFull, (uint32_t)kmin);
            kmax = (U)__reduce_max_sync(kFull, (uint32_t)kmax);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum = __dadd_rn(sum, __shfl_xor_sync(kFull, sum, o));
        if (lane == 0) {
            reinterpret_cast<double *>(job.flags + tile_count(job.nchunks))[c] = sum;
            if (nan) atomicAdd(&ctl->agg[0], (unsigned long long)nan);
            if (kmax) {                           // some value was not a NaN
                auto unkey = [&](U k) { return (k & SIGN) ? (U)(k & ABSM) : (U)~k; };
                atomicMax(&ctl->agg[1], (unsigned long long)~order_key(value_f64(unkey(kmin))));
                atomicMax(&ctl->agg[2], (unsigned long long)order_key(value_f64(unkey(kmax))));
            }
        }
        __syncwarp();
        return;
    }

    // ---- c. stage (swizzled) and store --------------------------------------------------------
    constexpr int UN = T::UNITS;
#pragma unroll
    for (int u = 0; u < UN; ++u) {
        uint4 q;
        if constexpr (D == 0) {
            q = make_uint4((uint32_t)d[2 * u], (uint32_t)((uint64_t)d[2 * u] >> 32),
                           (uint32_t)d[2 * u + 1], (uint32_t)((uint64_t)d[2 * u + 1] >> 32));
        } else if constexpr (D == kD32) {
            q = make_uint4((uint32_t)d[4 * u], (uint32_t)d[4 * u + 1], (uint32_t)d[4 * u + 2], (uint32_t)d[4 * u + 3]);
        } else {
            q = make_uint4((uint32_t)d[8 * u] | ((uint32_t)d[8 * u + 1] << 16), (uint32_t)d[8 * u + 2] | ((uint32_t)d[8 * u + 3] << 16),
                           (uint32_t)d[8 * u + 4] | ((uint32_t)d[8 * u + 5] << 16), (uint32_t)d[8 * u + 6] | ((uint32_t)d[8 * u + 7] << 16));
        }
        *reinterpret_cast<uint4 *>(pbuf + (lane * UN + unit_swizzle<D>(lane, u)) * 16) = q;
    }
    if (m > 1024u && lane == 31) *reinterpret_cast<U *>(pbuf + phys_elem_byte<D>(1024)) = vx;
    __syncwarp();
    uint8_t *dst = job.out + first * T::S;
    const uint32_t nbytes = m * T::S;
    uint32_t done = 0;
    if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
        const uint32_t nunits = nbytes >> 4;
        for (uint32_t q = lane; q < nunits; q += 32)
            *reinterpret_cast<uint4 *>(dst + 16u * q) = *reinterpret_cast<const uint4 *>(pbuf + phys_unit<D>(q) * 16u);
        done = (nunits * 16u) / T::S;
    }
    for (uint32_t e = done + lane; e < m; e += 32)
        *reinterpret_cast<U *>(dst + (size_t)e * T::S) = *reinterpret_cast<const U *>(pbuf + phys_elem_byte<D>(e));
    __syncwarp();
}

}  // namespace

// Record offsets per 64-chunk tile (exclusive prefix of the u32 size array) of every job
// into the first words of job.flags.
__global__ void __launch_bounds__(1024)
offsets_kernel(const Job *__restrict__ jobs, Job single) {
    __shared__ uint64_t warp_sums[33];
    const Job &job = (jobs == nullptr) ? single : jobs[blockIdx.x];
    (void)tile_prefix(reinterpret_cast<const uint32_t *>(job.in + 32), job.nchunks, job.flags, warp_sums);
}

// Forms by dtype: kDt = 0 (every job FP64), 1 (every job FP32), 2 (either, per job).
constexpr int kDtF64 = 0, kDtF32 = 1, kDtMixed = 2, kDtF16 = 3;
// the value kind whose buffers a form needs (the either-dtype form: the largest)
template <int kDt> constexpr int layout_kind() { return kDt == kDtF32 ? kD32 : (kDt == kDtF16 ? kD16 : kD64); }

template <int kDt, bool kAgg = false>
__global__ void __launch_bounds__(32 * kMaxDecompressWarps, 1)
decompress_kernel(const Job *__restrict__ jobs, int njobs, Job single, uint64_t total_chunks, Control *ctl) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    using L = DecLayout<layout_kind<kDt>()>;
    uint8_t *wbase = smem + warp * L::kWarpBytes;
    uint8_t *pbuf = wbase + L::kBuf;
    __shared__ Job s_single;                      // the single job, read from shared memory
    if (threadIdx.x == 0) s_single = single;
    init_expand_sel();
    __syncthreads();
    const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t j = gw; j < (uint64_t)((jobs != nullptr) ? njobs : 1); j += nw) {
        const Job &jb = (jobs != nullptr) ? jobs[j] : s_single;
        if (lane == 0) jb.result[0] = jb.n;
    }
    // chunk tickets two deep: t is decoded, tn's record is fetched during t, tnn is located
    uint64_t t = ticket_of(take_ticket(ctl, kTicketDecode, lane));
    if (t >= total_chunks) return;
    uint64_t tn = ticket_of(take_ticket(ctl, kTicketDecode, lane));
    Loc lc = locate(jobs, njobs, s_single, t, lane);
    resolve(jobs, njobs, s_single, lc);
    bool okc = issue_record(job_of(jobs, njobs, s_single, t), lc, wbase, lane);
    cp_async_commit();
    Loc ln{};
    if (tn < total_chunks) ln = locate(jobs, njobs, s_single, tn, lane);
    for (;;) {
        const unsigned long long raw = tn < total_chunks ? take_ticket(ctl, kTicketDecode, lane) : 0ull;
        uint64_t tnn = total_chunks;
        bool okn = false;
        Loc lnn{};
        cp_async_wait_none();                    // the current record has landed
        __syncwarp();
        // the next record goes into the same buffer once this one has been read
        auto next = [&]() {
            if (tn < total_chunks) {
                resolve(jobs, njobs, s_single, ln);
                okn = issue_record(job_of(jobs, njobs, s_single, tn), ln, wbase, lane);
                tnn = ticket_of(raw);
                if (tnn < total_chunks) lnn = locate(jobs, njobs, s_single, tnn, lane);
            }
            cp_async_commit();
        };
        const Job &job = job_of(jobs, njobs, s_single, t);
        if constexpr (kDt == kDtF64) decode_chunk<kD64, kAgg>(job, lc, okc, wbase, pbuf, lane, next, ctl);
        else if constexpr (kDt == kDtF32) decode_chunk<kD32, kAgg>(job, lc, okc, wbase, pbuf, lane, next, ctl);
        else if constexpr (kDt == kDtF16) decode_chunk<kD16, kAgg>(job, lc, okc, wbase, pbuf, lane, next, ctl);
        else if (job.dtype == 0) decode_chunk<kD64, kAgg>(job, lc, okc, wbase, pbuf, lane, next, ctl);
        else if (job.dtype == 1) decode_chunk<kD32, kAgg>(job, lc, okc, wbase, pbuf, lane, next, ctl);
        else decode_chunk<kD16, kAgg>(job, lc, okc, wbase, pbuf, lane, next, ctl);
        if (tn >= total_chunks) break;
        t = tn;
        tn = tnn;
        lc = ln;
        okc = okn;
        ln = lnn;
    }
    cp_async_wait_none();
}

int decompress_grid(uint64_t total_chunks) {
    const int w = g_cta_warps[1];
    return persistent_grid_size(reinterpret_cast<const void *>(decompress_kernel<kDtMixed>), w,
                                w * DecLayout<kD64>::kWarpBytes,
                                g_ctas_per_sm[1], total_chunks);
}

// The aggregate's last step (one CTA): thread t adds the chunk sums of its contiguous share in
// chunk order, then a fixed tree over the threads; the NaN count and the min / max keys come
// from the control block, the status from the decode.  Every step has a fixed order, so the
// result does not depend on the schedule.
__global__ void __launch_bounds__(1024)
aggregate_finish_kernel(Job single, Control *ctl, falcon_stats *out) {
    __shared__ double part[1024];
    const uint64_t nc = single.nchunks;
    const double *sums = reinterpret_cast<const double *>(single.flags + tile_count(nc));
    const uint64_t c0 = nc * threadIdx.x / 1024u, c1 = nc * (threadIdx.x + 1u) / 1024u;
    double s = -0.0;
    for (uint64_t c = c0; c < c1; ++c) s = __dadd_rn(s, sums[c]);
    part[threadIdx.x] = s;
    __syncthreads();
    for (unsigned h = 512; h > 0; h >>= 1) {
        if (threadIdx.x < h) part[threadIdx.x] = __dadd_rn(part[threadIdx.x], part[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned long long nan = ctl->agg[0], kmin_c = ctl->agg[1], kmax = ctl->agg[2];
        auto from_key = [](uint64_t k) {
            return __longlong_as_double((long long)((k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k));
        };
        out->count = single.n;
        out->nan_count = nan;
        out->min = kmax ? from_key(~kmin_c) : __longlong_as_double(0x7FF8000000000000ll);
        out->max = kmax ? from_key(kmax) : __longlong_as_double(0x7FF8000000000000ll);
        out->sum = kmax ? part[0] : 0.0;          // no non-NaN value: the empty sum
        out->status = single.result[1];
    }
}

namespace {
template <int kDt, bool kAgg = false>
void launch_decode(const Job *d_jobs, int njobs, const Job &single, uint64_t total_chunks, Control *ctl,
                   cudaStream_t stream) {
    const int w = g_cta_warps[1], smem = w * DecLayout<layout_kind<kDt>()>::kWarpBytes;
    const int grid = persistent_grid_size(reinterpret_cast<const void *>(decompress_kernel<kDt, kAgg>), w, smem,
                                          g_ctas_per_sm[1], total_chunks);
    decompress_kernel<kDt, kAgg><<<grid, 32 * w, smem, stream>>>(d_jobs, njobs, single, total_chunks, ctl);
}
}  // namespace

cudaError_t launch_aggregate(const Job &single, Control *ctl, void *d_stats, cudaStream_t stream) {
    offsets_kernel<<<1, 1024, 0, stream>>>(nullptr, single);
    if (single.nchunks > 0) {
        if (single.dtype == 0) launch_decode<kDtF64, true>(nullptr, 1, single, single.nchunks, ctl, stream);
        else if (single.dtype == 1) launch_decode<kDtF32, true>(nullptr, 1, single, single.nchunks, ctl, stream);
        else launch_decode<kDtF16, true>(nullptr, 1, single, single.nchunks, ctl, stream);
    }
    aggregate_finish_kernel<<<1, 1024, 0, stream>>>(single, ctl, static_cast<falcon_stats *>(d_stats));
    return cudaGetLastError();
}

cudaError_t launch_decompress(const Job *d_jobs, int njobs, const Job &single, uint64_t total_chunks,
                              Control *ctl, cudaStream_t stream) {
    offsets_kernel<<<(d_jobs != nullptr) ? njobs : 1, 1024, 0, stream>>>(d_jobs, single);
    if (d_jobs != nullptr) launch_decode<kDtMixed>(d_jobs, njobs, single, total_chunks, ctl, stream);
    else if (single.dtype == 0) launch_decode<kDtF64>(d_jobs, njobs, single, total_chunks, ctl, stream);
    else if (single.dtype == 1) launch_decode<kDtF32>(d_jobs, njobs, single, total_chunks, ctl, stream);
    else launch_decode<kDtF16>(d_jobs, njobs, single, total_chunks, ctl, stream);
    return cudaGetLastError();
}

}  // namespace falcon
