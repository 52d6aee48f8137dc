// Falcon compression kernel (Sec. 3 of the paper; Alg. 3 CmpKernel) for sm_103a.
//
// One persistent launch; each warp repeatedly claims a chunk (dynamic ticket, so that
// the decoupled look-back only ever waits on chunks already owned by running warps) and
//   1. stages the chunk's values in shared memory with cp.async (swizzled),
//   2. decides Case 1 / Case 2 of Eq. 4: specials (R1) and the chunk maximum first, then
//      the smallest decimal place alpha_max at which every value passes Alg. 2's test
//      (exact integer arithmetic, see q_test), searched from the warp's previous alpha,
//   3. computes G (Eq. 4) and Z (Eq. 5), the bit width w and the bit planes (32x32
//      register transposes),
//   4. counts the zero bytes of every row (lambda) and picks sparse/dense storage
//      (Sec. 3.3), which gives the record size,
//   5. obtains its output offset by decoupled look-back (Sec. 3.4),
//   6. assembles the record in shared memory at the output's 16-byte phase and writes it
//      with aligned 16-byte stores.
#include "falcon_device.cuh"

namespace falcon {

namespace {

// Byte-stream writer over a warp's shared-memory record buffer.  Bytes before `pos` are
// final in shared memory except the partial 32-bit word at (sh + pos) & ~3, whose valid
// low bytes are kept, top-aligned, in `pend` (identical in every lane).
struct RecordWriter {
    uint8_t *buf;       // warp buffer (16-byte aligned); the record starts at buf + sh
    uint32_t sh;        // 0..15
    uint32_t pos;       // bytes of the record written so far
    uint32_t pend;

    __device__ __forceinline__ uint32_t abs_pos() const { return sh + pos; }

    __device__ __forceinline__ void reload(int lane) {
        (void)lane;
        __syncwarp();
        const uint32_t P = abs_pos();
        const uint32_t s = P & 3u;
        pend = s ? (*reinterpret_cast<const uint32_t *>(buf + (P - s)) << (32u - 8u * s)) : 0u;
    }
    __device__ __forceinline__ void flush(int lane) {
        const uint32_t P = abs_pos();
        const uint32_t s = P & 3u;
        if (lane == 0 && s) *reinterpret_cast<uint32_t *>(buf + (P - s)) = pend >> (32u - 8u * s);
        __syncwarp();
    }
    // A dense row: lane l < nact holds row bytes 4l .. 4l+3 in x (little-endian).
    __device__ __forceinline__ void dense(uint32_t x, int lane, uint32_t nact) {
        const uint32_t P = abs_pos();
        const uint32_t s = P & 3u;
        uint32_t prev = __shfl_up_sync(kFull, x, 1);
        if (lane == 0) prev = pend;
        const uint32_t word = __funnelshift_l(prev, x, 8u * s);
        if ((uint32_t)lane < nact) *reinterpret_cast<uint32_t *>(buf + (P - s) + 4u * lane) = word;
        pend = __shfl_sync(kFull, x, (int)nact - 1);
        pos += 4u * nact;
    }
    // A sparse row: bitmap of nact/2 bytes, then the non-zero bytes in row order.
    __device__ __forceinline__ void sparse(uint32_t x, int lane, uint32_t nact) {
        flush(lane);
        const uint32_t P = abs_pos();
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
        pos += nact / 2u + total;
        reload(lane);
    }
};

template <bool F64>
__device__ __forceinline__ int search_alpha(const typename Traits<F64>::U (&v)[32],
                                            typename Traits<F64>::U vx, int atop, int hint) {
    // smallest a in [0, atop] at which every value passes q_test, or -1 (Case 2).  The
    // predicate is monotone in a for chunks of valid values (Thm 4 with Thm 3), and a
    // single failure at atop means some value is an exception or needs alpha > atop.
    auto all_pass = [&](int a) -> bool {
        bool ok = q_test(vx, a);
#pragma unroll
        for (int k = 0; k < 32; ++k) ok &= q_test(v[k], a);
        return __all_sync(kFull, ok);
    };
    int lo, hi;
    if (hint >= 0 && hint < atop) {
        if (all_pass(hint)) {
            if (hint == 0 || !all_pass(hint - 1)) return hint;
            lo = 0;
            hi = hint - 1;
        } else {
            if (!all_pass(atop)) return -1;
            lo = hint + 1;
            hi = atop;
        }
    } else {
        if (!all_pass(atop)) return -1;
        lo = 0;
        hi = atop;
    }
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (all_pass(mid)) hi = mid;
        else lo = mid + 1;
    }
    return hi;
}

// FP32: alpha_max = max over values of Alg. 2's decimal place (first_pass_f32), then the
// R6 check that every value round-trips at alpha_max; -1 means Case 2.
__device__ __forceinline__ int alpha_f32(const uint32_t (&v)[32], uint32_t vx, uint32_t vmax, int atop) {
    // quick rejection on the largest magnitude(s)
    bool fail = ((vx & 0x7FFFFFFFu) == vmax) && first_pass_f32(vx, atop) < 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) fail |= ((v[k] & 0x7FFFFFFFu) == vmax) && first_pass_f32(v[k], atop) < 0;
    if (__any_sync(kFull, fail)) return -1;
    int amax = first_pass_f32(vx, atop);
    bool bad = amax < 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const int a = first_pass_f32(v[k], atop);
        bad |= a < 0;
        amax = a > amax ? a : amax;
    }
    if (__any_sync(kFull, bad)) return -1;
    amax = (int)__reduce_max_sync(kFull, (uint32_t)amax);
    bool rt = q_test(vx, amax);
#pragma unroll
    for (int k = 0; k < 32; ++k) rt &= q_test(v[k], amax);
    return __all_sync(kFull, rt) ? amax : -1;
}

template <bool F64>
__device__ void compress_chunk(const Job &job, uint64_t c, uint8_t *wsm, int lane, int &hint,
                               Control *ctl) {
    using T = Traits<F64>;
    using U = typename T::U;
    constexpr U ABS = F64 ? (U)0x7FFFFFFFFFFFFFFFull : (U)0x7FFFFFFFu;

    const uint32_t B = job.block;
    const uint64_t first = c * (uint64_t)B;
    const uint32_t m = (uint32_t)((job.n - first) < B ? (job.n - first) : B);
    const uint64_t data_start = 32ull + 4ull * job.nchunks;

    // ---- 1. stage and read the values ----------------------------------------------
    stage_values<F64>(job.in + first * T::S, m, wsm, lane);
    U v[32];
    read_own<F64>(wsm, lane, m, v);
    U vx = 0;                                   // value 1024 of a 1025-value chunk
    if (m > 1024u && lane == 31) vx = read_elem<F64>(wsm, 1024);
    __syncwarp();

    // ---- 2. Case decision (Eq. 4) -----------------------------------------------------
    bool sp = is_special(vx);
    U vmax = vx & ABS;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        sp |= is_special(v[k]);
        const U a = v[k] & ABS;
        vmax = a > vmax ? a : vmax;
    }
    sp = __any_sync(kFull, sp);
    vmax = warp_max_x(vmax);
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
                if constexpr (F64) {
                    // quick rejection: test the largest magnitude(s) first
                    bool fail = ((vx & ABS) == vmax) && !q_test(vx, atop);
#pragma unroll
                    for (int k = 0; k < 32; ++k) fail |= ((v[k] & ABS) == vmax) && !q_test(v[k], atop);
                    if (!__any_sync(kFull, fail)) alpha = search_alpha<F64>(v, vx, atop, hint);
                } else {
                    alpha = alpha_f32(v, vx, vmax, atop);
                }
                if (alpha >= 0) beta_hat = alpha + e_max + 1;
            }
        }
    }
    hint = alpha;

    // ---- 3. G (Eq. 4) and Z (Eq. 5) ----------------------------------------------------
    U g[32];
    U gx;
    if (alpha >= 0) {
#pragma unroll
        for (int k = 0; k < 32; ++k) g[k] = case1_g(v[k], alpha);
        gx = case1_g(vx, alpha);
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) g[k] = zigzag(v[k]);
        gx = zigzag(vx);
    }
    const U z1 = shfl_x(g[0], 0);
    U nxt = shfl_down_x(g[0], 1);
    if (lane == 31) nxt = gx;
    U z[32];
    U zor = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const U hi = (k < 31) ? g[k + 1] : nxt;
        U zz = zigzag((U)(hi - g[k]));
        if ((uint32_t)(32 * lane + k) + 1u >= m) zz = 0;      // pad columns (R11)
        z[k] = zz;
        zor |= zz;
    }
    zor = warp_or_x(zor);
    const int w = zor ? (T::W - (F64 ? __clzll((long long)zor) : __clz((int)zor))) : 0;

    // bit planes: plane word p, bit (k ^ 7) = bit p of z[k]; planes 0..31 in plo,
    // planes 32..63 (FP64 only) in phi
    uint32_t plo[32], phi[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        plo[j] = (uint32_t)z[j ^ 7];
        phi[j] = F64 ? (uint32_t)((uint64_t)z[j ^ 7] >> 32) : 0u;
    }
    transpose32(plo);
    if (F64 && w > 32) transpose32(phi);
#define FALCON_PLANE(p) ((p) < 32 ? plo[(p) & 31] : phi[(p) & 31])

    // ---- 4. lambda per row, storage choice, record size (Sec. 3.3) --------------------
    const uint32_t cols = chunk_cols(m);
    const uint32_t nact = cols / 32u;           // lanes holding row bytes (row = 4*nact bytes)
    const uint32_t row_bytes = cols / 8u;
    const bool active = (uint32_t)lane < nact;
    uint64_t dense_mask = 0;
    uint32_t body = 0;
#pragma unroll
    for (int p = 0; p < T::W; ++p) {
        if (p < w) {
            const int zc = active ? zero_bytes(FALCON_PLANE(p)) : 0;
            const uint32_t lam = __reduce_add_sync(kFull, (uint32_t)zc);
            const bool sparse = lam > cols / 64u;               // tie -> dense (R10)
            body += sparse ? (cols / 64u + row_bytes - lam) : row_bytes;
            if (!sparse) dense_mask |= 1ull << p;
        }
    }
    const uint32_t flag_bytes = ((uint32_t)w + 7u) / 8u;
    const uint32_t hdr = 3u + T::Z1B + flag_bytes;
    const uint32_t size = hdr + body;

    // ---- 5. output offset (decoupled look-back) ---------------------------------------
    bool ok;
    const uint64_t excl = lookback(job.flags, c, size, lane, ctl, ok);
    if (!ok) {
        if (lane == 0) set_status(job.result, kErrTimeout);
        return;
    }
    const uint64_t rec_off = data_start + excl;
    if (c + 1 == job.nchunks && lane == 0) job.result[0] = rec_off + size;
    if (rec_off + size > job.out_cap) {         // also covers the header and size array
        if (lane == 0) set_status(job.result, kErrCapacity);
        return;
    }
    if (lane == 0) *reinterpret_cast<uint32_t *>(job.out + 32 + 4 * c) = size;
    uint8_t *gdst = job.out + rec_off;
    const uint32_t sh = (uint32_t)(reinterpret_cast<uintptr_t>(gdst) & 15u);

    // ---- 6. assemble the record in shared memory -------------------------------------
    RecordWriter wr{wsm, sh, 0u, 0u};
    if ((uint32_t)lane < hdr) {
        uint32_t byte;
        const int i = lane;
        if (i == 0) byte = (uint32_t)(alpha >= 0 ? alpha : T::A_SENT);
        else if (i == 1) byte = (uint32_t)beta_hat;
        else if (i < 2 + T::Z1B) byte = (uint32_t)((uint64_t)z1 >> (8 * (i - 2))) & 0xFFu;
        else if (i == 2 + T::Z1B) byte = (uint32_t)w;
        else byte = (uint32_t)(dense_mask >> (8u * (flag_bytes - 1u - (uint32_t)(i - 3 - T::Z1B)))) & 0xFFu;
        wsm[sh + i] = (uint8_t)byte;
    }
    wr.pos = hdr;
    wr.reload(lane);
#pragma unroll
    for (int p = T::W - 1; p >= 0; --p) {
        if (p < w) {
            if ((dense_mask >> p) & 1ull) wr.dense(FALCON_PLANE(p), lane, nact);
            else wr.sparse(FALCON_PLANE(p), lane, nact);
        }
    }
    wr.flush(lane);
#undef FALCON_PLANE

    // ---- 7. copy to global: aligned 16-byte units, byte stores at the two ends -------
    uint8_t *gbase = gdst - sh;
    const uint32_t total = sh + size;
    const uint32_t units = (total + 15u) / 16u;
    for (uint32_t u = lane; u < units; u += 32) {
        const uint32_t lo = 16u * u, hi = lo + 16u;
        if (lo >= sh && hi <= total) {
            *reinterpret_cast<uint4 *>(gbase + lo) = *reinterpret_cast<const uint4 *>(wsm + lo);
        } else {
            const uint32_t b0 = lo > sh ? lo : sh;
            const uint32_t b1 = hi < total ? hi : total;
            for (uint32_t b = b0; b < b1; ++b) gbase[b] = wsm[b];
        }
    }
    // the stream header, once per job
    if (c == 0 && lane == 0) {
        uint32_t h[8];
        h[0] = 0x4E434C46u;                                    // "FLCN"
        h[1] = 1u | ((uint32_t)(F64 ? 0 : 1) << 8);
        h[2] = B;
        h[3] = 0;
        h[4] = (uint32_t)job.n;
        h[5] = (uint32_t)(job.n >> 32);
        h[6] = (uint32_t)job.nchunks;
        h[7] = (uint32_t)(job.nchunks >> 32);
        uint4 *dst = reinterpret_cast<uint4 *>(job.out);
        dst[0] = make_uint4(h[0], h[1], h[2], h[3]);
        dst[1] = make_uint4(h[4], h[5], h[6], h[7]);
    }
    __syncwarp();
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 4)
compress_kernel(const Job *__restrict__ jobs, int njobs, Job single, uint64_t total_chunks,
                Control *ctl) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint8_t *wsm = smem + warp * kWarpSmem;

    // jobs without chunks (n = 0) still get a header and a length
    {
        const int gw = blockIdx.x * kWarpsPerCta + warp;
        const int nw = gridDim.x * kWarpsPerCta;
        const int nj = (jobs != nullptr) ? njobs : 1;
        for (int j = gw; j < nj; j += nw) {
            const Job &jb = (jobs != nullptr) ? jobs[j] : single;
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

    int hint64 = -1, hint32 = -1;
    while (true) {
        uint64_t t = 0;
        if (lane == 0) t = atomicAdd(&ctl->ticket, 1ull);
        t = shfl_u64(t, 0);
        if (t >= total_chunks) break;
        if (*reinterpret_cast<volatile unsigned int *>(&ctl->abort)) break;
        const Job &job = (jobs == nullptr) ? single : jobs[find_job(jobs, njobs, t)];
        const uint64_t c = t - job.chunk_begin;
        if (job.dtype == 0) compress_chunk<true>(job, c, wsm, lane, hint64, ctl);
        else compress_chunk<false>(job, c, wsm, lane, hint32, ctl);
    }
}

static int g_grid_cache[64] = {0};

int compress_grid(uint64_t total_chunks) {
    int dev = 0;
    cudaGetDevice(&dev);
    int &cached = g_grid_cache[dev & 63];
    if (cached == 0) {
        int sms = 0, occ = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, compress_kernel, kThreads, kCtaSmem);
        cached = sms * (occ > 0 ? occ : 1);
    }
    const uint64_t need = (total_chunks + kWarpsPerCta - 1) / kWarpsPerCta;
    return (int)(need < (uint64_t)cached ? (need > 0 ? need : 1) : (uint64_t)cached);
}

cudaError_t launch_compress(const Job *d_jobs, int njobs, const Job &single, uint64_t total_chunks,
                            Control *ctl, cudaStream_t stream) {
    const int grid = compress_grid(total_chunks);
    compress_kernel<<<grid, kThreads, kCtaSmem, stream>>>(d_jobs, njobs, single, total_chunks, ctl);
    return cudaGetLastError();
}

}  // namespace falcon
