// Falcon compression kernel (Sec. 3 of the paper; Alg. 3 CmpKernel) for sm_103a.
//
// One persistent launch; each warp repeatedly claims a chunk (dynamic ticket, so that the
// decoupled look-back only waits on chunks owned by running warps).  While it works on one
// chunk, the next chunk's values are already streaming into its second shared-memory buffer
// (cp.async, swizzled).  Per chunk:
//   1. read the lane's 32 values, classify (R1 specials) and take the chunk maximum,
//   2. Case 1 / Case 2 of Eq. 4: the smallest decimal place alpha_max at which every value
//      passes Alg. 2's test, in exact integer arithmetic (q_test); FP32 follows Alg. 2 value
//      by value,
//   3. G (Eq. 4), Z (Eq. 5) and the bit width w in registers,
//   4. 32x32 register transposes give one 32-bit word per bit plane (4 row bytes per lane);
//      the words go to shared memory and their non-zero bytes are counted (Sec. 3.3 lambda),
//   5. sparse/dense per row -> record size -> decoupled look-back (Sec. 3.4) -> offset,
//   6. the record is assembled in shared memory at the output's 16-byte phase, in place of
//      the plane words it consumes, and written with aligned 16-byte stores.
#include "falcon_device.cuh"

namespace falcon {

namespace {

constexpr int kBuf = 8288;                  // one chunk of values / one record (+32 readable)
constexpr int kScratch = 128;
constexpr int kWarpBytes = 2 * kBuf + kScratch;
constexpr int kPlOff = 48;                  // plane words: kPlOff + (W-1-p)*128 + 4*lane

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

// Sparse row (Sec. 3.3) written with byte stores at byte offset P of the warp buffer:
// a bitmap of nact/2 bytes (bit 7 of byte 0 = row byte 0), then the non-zero row bytes.
// Returns the row's length.
__device__ __forceinline__ uint32_t sparse_row(uint8_t *buf, uint32_t P, uint32_t x, int lane, uint32_t nact) {
    const bool active = (uint32_t)lane < nact;
    const uint32_t nib = active ? nonzero_nibble(x) : 0u;
    const uint32_t nib_next = __shfl_down_sync(kFull, nib, 1);
    if (active && !(lane & 1)) buf[P + (lane >> 1)] = (uint8_t)((nib << 4) | nib_next);
    const uint32_t cnt = __popc(nib);
    const unsigned b0 = __ballot_sync(kFull, cnt & 1u);
    const unsigned b1 = __ballot_sync(kFull, cnt & 2u);
    const unsigned b2 = __ballot_sync(kFull, cnt & 4u);
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t before = __popc(b0 & lt) + 2u * __popc(b1 & lt) + 4u * __popc(b2 & lt);
    const uint32_t total = __popc(b0) + 2u * __popc(b1) + 4u * __popc(b2);
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
template <bool F64>
__device__ __forceinline__ typename Traits<F64>::U lane_value(const uint8_t *buf, int lane, int k) {
    using U = typename Traits<F64>::U;
    constexpr int UN = Traits<F64>::UNITS;
    constexpr int PER = 16 / Traits<F64>::S;
    return *reinterpret_cast<const U *>(buf + (lane * UN + ((k / PER) ^ (lane & 7))) * 16 + (k % PER) * Traits<F64>::S);
}

// Every value of the chunk passes Alg. 2's test at a.  The values are re-read from the
// staging buffer; this runs a few times per Case-1 chunk only.
template <bool F64>
__device__ __noinline__ bool all_pass(const uint8_t *buf, int lane, uint32_t m, typename Traits<F64>::U vx, int a) {
    bool ok = q_test(vx, a);
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
        if (32u * lane + k < m) ok &= q_test(lane_value<F64>(buf, lane, k), a);
    }
    return __all_sync(kFull, ok);
}

// FP64: smallest a in [0, atop] at which every value passes, or -1 (Case 2).  For chunks of
// valid values the predicate is monotone in a (Thm 4 with Thm 3); a single failure at atop
// means some value is an exception or needs alpha > atop.
__device__ int search_alpha64(const uint8_t *buf, int lane, uint32_t m, uint64_t vx, int atop, int hint) {
    int lo, hi;
    if (hint >= 0 && hint < atop) {
        if (all_pass<true>(buf, lane, m, vx, hint)) {
            if (hint == 0 || !all_pass<true>(buf, lane, m, vx, hint - 1)) return hint;
            lo = 0;
            hi = hint - 1;
        } else {
            if (!all_pass<true>(buf, lane, m, vx, atop)) return -1;
            lo = hint + 1;
            hi = atop;
        }
    } else {
        if (!all_pass<true>(buf, lane, m, vx, atop)) return -1;
        lo = 0;
        hi = atop;
    }
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (all_pass<true>(buf, lane, m, vx, mid)) hi = mid;
        else lo = mid + 1;
    }
    return hi;
}

// FP32: alpha_max = max over values of Alg. 2's decimal place (first_pass_f32), then the R6
// check that every value round-trips at alpha_max; -1 means Case 2.
__device__ int alpha32(const uint8_t *buf, int lane, uint32_t m, uint32_t vx, int atop) {
    int amax = first_pass_f32(vx, atop);
    bool bad = amax < 0;
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
        if (32u * lane + k < m) {
            const int a = first_pass_f32(lane_value<false>(buf, lane, k), atop);
            bad |= a < 0;
            amax = a > amax ? a : amax;
        }
    }
    if (__any_sync(kFull, bad)) return -1;
    amax = (int)__reduce_max_sync(kFull, (uint32_t)amax);
    return all_pass<false>(buf, lane, m, vx, amax) ? amax : -1;
}

__device__ __forceinline__ void issue_chunk(const Job *jobs, int njobs, const Job &single, uint64_t t,
                                            uint8_t *buf, int lane) {
    const Job &job = (jobs == nullptr) ? single : jobs[find_job(jobs, njobs, t)];
    const uint64_t c = t - job.chunk_begin;
    const uint64_t first = c * (uint64_t)job.block;
    const uint32_t m = (uint32_t)((job.n - first) < job.block ? (job.n - first) : job.block);
    if (job.dtype == 0) stage_values_async<true>(job.in + first * 8u, m, buf, lane);
    else stage_values_async<false>(job.in + first * 4u, m, buf, lane);
}

// A chunk whose size is published and whose record waits for its offset.
struct Pend {
    uint64_t t;             // global ticket
    uint64_t z1;
    uint64_t dense_mask;
    uint32_t size;
    int w;
    int alpha_byte;         // header byte 0 (alpha_max or the Case-2 sentinel)
    int beta_hat;           // header byte 1
    bool valid;
};

// Steps 1-5: everything up to the record size, which is published for the look-back.
// The plane words stay in buf for finish_chunk.
template <bool F64>
__device__ void compute_chunk(const Job &job, uint64_t t, uint8_t *buf, uint8_t *scratch, int lane,
                              int &hint, Pend &pd) {
    const uint64_t c = t - job.chunk_begin;
    using T = Traits<F64>;
    using U = typename T::U;
    constexpr U ABS = F64 ? (U)0x7FFFFFFFFFFFFFFFull : (U)0x7FFFFFFFu;

    const uint32_t B = job.block;
    const uint64_t first = c * (uint64_t)B;
    const uint32_t m = (uint32_t)((job.n - first) < B ? (job.n - first) : B);
    const uint64_t data_start = 32ull + 4ull * job.nchunks;

    // ---- 1. values, specials, maximum ------------------------------------------------------
    U v[32];
    read_own<F64>(buf, lane, m, v);
    U vx = 0;                                   // value 1024 of a 1025-value chunk
    if (m > 1024u && lane == 31) vx = read_elem<F64>(buf, 1024);
    bool sp;
    U vmax;
    if constexpr (F64) {
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
            if (atop >= 0) {
                // quick rejection: Alg. 2 on the largest magnitude first (one per lane)
                U cand = 0;
                bool has = (vx & ABS) == vmax;
                if (has) cand = vx;
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const bool is_max = (v[k] & ABS) == vmax;
                    cand = is_max ? v[k] : cand;
                    has |= is_max;
                }
                bool fail = false;
                if (has) {
                    if constexpr (F64) fail = !q_test(cand, atop);
                    else fail = first_pass_f32(cand, atop) < 0;
                }
                if (!__any_sync(kFull, fail)) {
                    if constexpr (F64) alpha = search_alpha64(buf, lane, m, vx, atop, hint);
                    else alpha = alpha32(buf, lane, m, vx, atop);
                }
            }
            if (alpha >= 0) beta_hat = alpha + e_max + 1;
        }
    }
    hint = alpha;

    // ---- 3. G (Eq. 4) and Z (Eq. 5) ------------------------------------------------------------
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
    U zor = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const U hi = (k < 31) ? v[k + 1] : nxt;
        v[k] = zigzag((U)(hi - v[k]));          // v now holds Z of columns 32*lane + k
        zor |= v[k];
    }
    if (32u * lane + 32u >= m) {                 // pad columns (R11): only the last lanes
        zor = 0;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            if (32u * lane + k + 1u >= m) v[k] = 0;
            zor |= v[k];
        }
    }
    zor = warp_or_x(zor);
    const int w = zor ? (T::W - (F64 ? __clzll((long long)zor) : __clz((int)zor))) : 0;
    __syncwarp();                                // the staging buffer is reused below

    // ---- 4. bit planes -> shared memory, non-zero bytes per row ---------------------------------
    const uint32_t cols = chunk_cols(m);
    const uint32_t nact = cols / 32u;            // lanes holding row bytes
    const uint32_t row_bytes = cols / 8u;
    // lanes past the row (lane >= nact) hold only pad columns, i.e. zero plane words
    uint32_t packed[T::W / 4];
    {
        uint32_t a[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) a[j] = (uint32_t)v[j ^ 7];
        transpose32(a);
#pragma unroll
        for (int p = 0; p < 32; ++p) {
            *reinterpret_cast<uint32_t *>(buf + kPlOff + (T::W - 1 - p) * 128 + 4 * lane) = a[p];
            const uint32_t nzb = (uint32_t)__popc((((a[p] & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | a[p]) & 0x80808080u);
            if (p % 4 == 0) packed[p / 4] = nzb;
            else packed[p / 4] |= nzb << (8 * (p % 4));
        }
    }
    if constexpr (F64) {
        if (w > 32) {
            uint32_t a[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) a[j] = (uint32_t)((uint64_t)v[j ^ 7] >> 32);
            transpose32(a);
#pragma unroll
            for (int p = 0; p < 32; ++p) {
                *reinterpret_cast<uint32_t *>(buf + kPlOff + (31 - p) * 128 + 4 * lane) = a[p];
                const uint32_t nzb = (uint32_t)__popc((((a[p] & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | a[p]) & 0x80808080u);
                if (p % 4 == 0) packed[8 + p / 4] = nzb;
                else packed[8 + p / 4] |= nzb << (8 * (p % 4));
            }
        } else {
#pragma unroll
            for (int i = 8; i < 16; ++i) packed[i] = 0;
        }
    }
#pragma unroll
    for (int i = 0; i < T::W / 4; ++i) {
        const uint32_t s = __reduce_add_sync(kFull, packed[i]);
        if (lane == 0) reinterpret_cast<uint32_t *>(scratch)[i] = s;
    }
    __syncwarp();

    // ---- 5. storage choice (Sec. 3.3), record size, offset (Sec. 3.4) --------------------------
    uint32_t cost = 0;
    bool dense_lo = false, dense_hi = false;
    if (lane < w) {                              // plane `lane`
        const uint32_t nz = scratch[lane];
        const bool sparse = (row_bytes - nz) > cols / 64u;           // tie -> dense (R10)
        cost += sparse ? cols / 64u + nz : row_bytes;
        dense_lo = !sparse;
    }
    if (F64 && lane + 32 < w) {                  // plane `lane + 32`
        const uint32_t nz = scratch[lane + 32];
        const bool sparse = (row_bytes - nz) > cols / 64u;
        cost += sparse ? cols / 64u + nz : row_bytes;
        dense_hi = !sparse;
    }
    const uint32_t body = __reduce_add_sync(kFull, cost);
    const uint64_t dense_mask = (uint64_t)__ballot_sync(kFull, dense_lo) |
                                ((uint64_t)__ballot_sync(kFull, dense_hi) << 32);
    const uint32_t flag_bytes = ((uint32_t)w + 7u) / 8u;
    const uint32_t hdr = 3u + T::Z1B + flag_bytes;
    const uint32_t size = hdr + body;
    publish_size(job.flags, c, size, lane);
    pd.t = t;
    pd.z1 = (uint64_t)z1;
    pd.dense_mask = dense_mask;
    pd.size = size;
    pd.w = w;
    pd.alpha_byte = alpha >= 0 ? alpha : T::A_SENT;
    pd.beta_hat = beta_hat;
    pd.valid = true;
    (void)data_start;
}

// Steps 5-6 of a computed chunk: offset (look-back), record assembly in place of its plane
// words, and the copy to global memory.  Returns false when a bounded wait gave up.
template <bool F64>
__device__ bool finish_chunk(const Job &job, const Pend &pd, uint8_t *buf, int lane, Control *ctl) {
    using T = Traits<F64>;
    const uint64_t c = pd.t - job.chunk_begin;
    const uint32_t B = job.block;
    const uint64_t first = c * (uint64_t)B;
    const uint32_t m = (uint32_t)((job.n - first) < B ? (job.n - first) : B);
    const uint64_t data_start = 32ull + 4ull * job.nchunks;
    const uint32_t cols = chunk_cols(m);
    const uint32_t nact = cols / 32u;
    const uint32_t row_bytes = cols / 8u;
    const int w = pd.w;
    const uint32_t size = pd.size;
    const uint64_t dense_mask = pd.dense_mask;
    const uint32_t flag_bytes = ((uint32_t)w + 7u) / 8u;
    const uint32_t hdr = 3u + T::Z1B + flag_bytes;

    bool ok;
    const uint64_t excl = lookback(job.flags, job.flags + job.nchunks, c, job.nchunks, size, lane, ctl, ok);
    if (!ok) {
        if (lane == 0) set_status(job.result, kErrTimeout);
        return false;
    }
    const uint64_t rec_off = data_start + excl;
    if (c + 1 == job.nchunks && lane == 0) job.result[0] = rec_off + size;
    if (rec_off + size > job.out_cap) {          // also covers the header and size array
        if (lane == 0) set_status(job.result, kErrCapacity);
        return true;
    }
    if (lane == 0) *reinterpret_cast<uint32_t *>(job.out + 32 + 4 * c) = size;
    uint8_t *gdst = job.out + rec_off;
    const uint32_t sh = (uint32_t)(reinterpret_cast<uintptr_t>(gdst) & 15u);

    // ---- 6. record in shared memory (in place of the consumed plane words), then global ------
    // Row r (plane w-r) ends before byte 37 + 128 r of the buffer while the plane read next
    // starts at kPlOff + (64 - w + r) * 128 >= 48 + 128 r: nothing unread is overwritten.
    if ((uint32_t)lane < hdr) {
        uint32_t byte;
        const int i = lane;
        if (i == 0) byte = (uint32_t)pd.alpha_byte;
        else if (i == 1) byte = (uint32_t)pd.beta_hat;
        else if (i < 2 + T::Z1B) byte = (uint32_t)(pd.z1 >> (8 * (i - 2))) & 0xFFu;
        else if (i == 2 + T::Z1B) byte = (uint32_t)w;
        else byte = (uint32_t)(dense_mask >> (8u * (flag_bytes - 1u - (uint32_t)(i - 3 - T::Z1B)))) & 0xFFu;
        buf[sh + i] = (uint8_t)byte;
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

    uint8_t *gbase = gdst - sh;
    const uint32_t total = sh + size;
    const uint32_t units = (total + 15u) / 16u;
    for (uint32_t u = lane; u < units; u += 32) {
        const uint32_t lo = 16u * u, hi = lo + 16u;
        if (lo >= sh && hi <= total) {
            *reinterpret_cast<uint4 *>(gbase + lo) = *reinterpret_cast<const uint4 *>(buf + lo);
        } else {
            const uint32_t b0 = lo > sh ? lo : sh;
            const uint32_t b1 = hi < total ? hi : total;
            for (uint32_t b = b0; b < b1; ++b) gbase[b] = buf[b];
        }
    }
    if (c == 0 && lane == 0) {                   // the stream header, once per job
        uint4 *dst = reinterpret_cast<uint4 *>(job.out);
        dst[0] = make_uint4(0x4E434C46u, 1u | ((uint32_t)(F64 ? 0 : 1) << 8), B, 0u);
        dst[1] = make_uint4((uint32_t)job.n, (uint32_t)(job.n >> 32), (uint32_t)job.nchunks,
                            (uint32_t)(job.nchunks >> 32));
    }
    __syncwarp();
    return true;
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 3)
compress_kernel(const Job *__restrict__ jobs, int njobs, Job single, uint64_t total_chunks, Control *ctl) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint8_t *wbase = smem + warp * kWarpBytes;
    uint8_t *scratch = wbase + 2 * kBuf;
    __shared__ Job s_single;                      // the single job, read from shared memory
    if (threadIdx.x == 0) s_single = single;
    __syncthreads();

    // jobs without chunks (n = 0) still get a header and a length
    {
        const int gw = blockIdx.x * kWarpsPerCta + warp;
        const int nw = gridDim.x * kWarpsPerCta;
        const int nj = (jobs != nullptr) ? njobs : 1;
        for (int j = gw; j < nj; j += nw) {
            const Job &jb = (jobs != nullptr) ? jobs[j] : s_single;
            if (jb.nchunks == 0 && lane == 0) {
                uint4 *dst = reinterpret_cast<uint4 *>(jb.out);
                if (jb.out_cap >= 32) {
                    dst[0] = make_uint4(0x4E434C46u, 1u | (jb.dtype << 8), jb.block, 0u);
                    dst[1] = make_uint4(0u, 0u, 0u, 0u);
                    jb.result[0] = 32;
                } else {
                    set_status(jb.result, kErrCapacity);
                }
            }
        }
    }

    // Two-stage pipeline per warp: chunk t is computed and its size published before the
    // previous chunk's offset is resolved, so the look-back waits overlap useful work.
    int hint64 = -1, hint32 = -1;
    int cur = 0;
    Pend pend;
    pend.valid = false;
    while (true) {
        uint64_t t = 0;
        if (lane == 0) t = atomicAdd(&ctl->ticket, 1ull);
        t = shfl_u64(t, 0);
        if (t >= total_chunks) break;
        if (*reinterpret_cast<volatile unsigned int *>(&ctl->abort)) break;
        const Job &job = (jobs == nullptr) ? s_single : jobs[find_job(jobs, njobs, t)];
        uint8_t *buf = wbase + cur * kBuf;
        issue_chunk(jobs, njobs, s_single, t, buf, lane);
        cp_async_commit();
        cp_async_wait_none();
        __syncwarp();
        Pend next;
        if (job.dtype == 0) compute_chunk<true>(job, t, buf, scratch, lane, hint64, next);
        else compute_chunk<false>(job, t, buf, scratch, lane, hint32, next);
        if (pend.valid) {
            const Job &pj = (jobs == nullptr) ? s_single : jobs[find_job(jobs, njobs, pend.t)];
            const bool ok = (pj.dtype == 0) ? finish_chunk<true>(pj, pend, wbase + (cur ^ 1) * kBuf, lane, ctl)
                                            : finish_chunk<false>(pj, pend, wbase + (cur ^ 1) * kBuf, lane, ctl);
            if (!ok) return;
        }
        pend = next;
        cur ^= 1;
    }
    if (pend.valid) {
        const Job &pj = (jobs == nullptr) ? s_single : jobs[find_job(jobs, njobs, pend.t)];
        if (pj.dtype == 0) finish_chunk<true>(pj, pend, wbase + (cur ^ 1) * kBuf, lane, ctl);
        else finish_chunk<false>(pj, pend, wbase + (cur ^ 1) * kBuf, lane, ctl);
    }
}

constexpr int kCompressCtaSmem = kWarpsPerCta * kWarpBytes;

static int g_occ_cache[64] = {0};
static int g_sms_cache[64] = {0};

int compress_grid(uint64_t total_chunks) {
    int dev = 0;
    cudaGetDevice(&dev);
    int &occ_c = g_occ_cache[dev & 63];
    if (occ_c == 0) {
        cudaFuncSetAttribute(compress_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kCompressCtaSmem);
        int sms = 0, occ = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, compress_kernel, kThreads, kCompressCtaSmem);
        g_sms_cache[dev & 63] = sms;
        occ_c = occ > 0 ? occ : 1;
    }
    const int lim = g_ctas_per_sm[0];
    const int cached = g_sms_cache[dev & 63] * ((lim > 0 && lim < occ_c) ? lim : occ_c);
    const uint64_t need = (total_chunks + kWarpsPerCta - 1) / kWarpsPerCta;
    return (int)(need < (uint64_t)cached ? (need > 0 ? need : 1) : (uint64_t)cached);
}

cudaError_t launch_compress(const Job *d_jobs, int njobs, const Job &single, uint64_t total_chunks,
                            Control *ctl, cudaStream_t stream) {
    const int grid = compress_grid(total_chunks);
    compress_kernel<<<grid, kThreads, kCompressCtaSmem, stream>>>(d_jobs, njobs, single, total_chunks, ctl);
    return cudaGetLastError();
}

}  // namespace falcon
