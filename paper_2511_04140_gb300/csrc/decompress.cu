// Falcon decompression kernel (Sec. 4 of the paper) for sm_103a.
//
// Persistent launch, one warp per chunk (dynamic ticket).  A warp prepares chunk t+1 (reads
// its size, decoupled look-back for its offset, starts the cp.async of its record) before it
// decodes chunk t, so record loads overlap decoding.  Decoding a chunk:
//   1. parse the header and flags; every row is expanded into one 32-bit word per lane
//      (dense: an unaligned 4-byte read; sparse: bitmap nibble + popcount rank) and stored
//      in the warp's plane buffer,
//   2. 32x32 register transposes give Z back; unzigzag + warp scan give G (inverse Eq. 5);
//      Case 1 divides by 10^alpha (correctly rounded), Case 2 undoes the zigzag of the
//      IEEE bits (inverse Eq. 4),
//   3. values are staged (swizzled) and written with coalesced 16-byte stores.
// Every read of a record is bounds-checked against its size; a malformed record sets
// FALCON_ERR_CORRUPT and writes nothing.
#include "falcon_device.cuh"

namespace falcon {

namespace {

constexpr int kBuf = 8256;
constexpr int kWarpBytes = 3 * kBuf;        // two record buffers + plane / value buffer

// unaligned little-endian 32-bit read at byte i of a 16-byte aligned shared buffer
__device__ __forceinline__ uint32_t ld_u32_unaligned(const uint8_t *b, uint32_t i) {
    const uint32_t s = i & 3u;
    const uint32_t *w = reinterpret_cast<const uint32_t *>(b + (i - s));
    return __funnelshift_r(w[0], w[1], 8u * s);
}

__device__ __forceinline__ double div_pow10(int64_t g, int a) {
    return __ddiv_rn(__ll2double_rn(g), __longlong_as_double((long long)FALCON_P10_F64[a - FALCON_P10_F64_LO]));
}
__device__ __forceinline__ float div_pow10(int32_t g, int a) {
    return __fdiv_rn(__int2float_rn(g), __uint_as_float(FALCON_P10_F32[a - FALCON_P10_F32_LO]));
}

// A chunk whose record is on its way into shared memory.
struct Pending {
    uint64_t t;          // global ticket
    uint64_t rec_off;    // record offset in the stream
    uint32_t size;       // record bytes
    uint32_t sh;         // 16-byte phase of the record in global (and shared) memory
    bool bad;            // size/offset inconsistent with the stream
    bool ok;             // look-back completed
};

__device__ __forceinline__ const Job &job_of(const Job *jobs, int njobs, const Job &single, uint64_t t) {
    return (jobs == nullptr) ? single : jobs[find_job(jobs, njobs, t)];
}

// Size, offset and record load of ticket t (no wait).
__device__ void prepare(const Job &job, uint64_t t, uint8_t *rbuf, int lane, Control *ctl, Pending &pd) {
    const uint64_t c = t - job.chunk_begin;
    const uint32_t B = job.block;
    const uint64_t first = c * (uint64_t)B;
    const uint32_t m = (uint32_t)((job.n - first) < B ? (job.n - first) : B);
    const uint32_t cols = chunk_cols(m);
    const uint32_t W = job.dtype == 0 ? 64u : 32u;
    const uint32_t z1b = W / 8u;
    const uint32_t max_rec = 3u + z1b + W / 8u + W * (cols / 8u);
    const uint64_t data_start = 32ull + 4ull * job.nchunks;

    uint32_t size = 0;
    if (lane == 0) size = *reinterpret_cast<const uint32_t *>(job.in + 32 + 4 * c);
    size = __shfl_sync(kFull, size, 0);
    pd.t = t;
    pd.size = size;
    const uint64_t excl = lookback(job.flags, job.flags + job.nchunks, c, job.nchunks, size, lane, ctl, pd.ok);
    if (!pd.ok) return;
    pd.rec_off = data_start + excl;
    pd.bad = (size < 3u + z1b) || (size > max_rec) || (pd.rec_off + size > job.in_bytes) ||
             (pd.rec_off + size < pd.rec_off);
    const uint8_t *gsrc = job.in + pd.rec_off;
    pd.sh = (uint32_t)(reinterpret_cast<uintptr_t>(gsrc) & 15u);
    if (pd.bad) return;
    const uint8_t *gbase = gsrc - pd.sh;                       // >= job.in (16-byte aligned)
    const uint8_t *gend = job.in + job.in_bytes;
    const uint32_t units = (pd.sh + size + 15u) / 16u;
    const uint32_t base = smem_addr(rbuf);
    for (uint32_t u = lane; u < units; u += 32) {
        const uint8_t *src = gbase + 16u * u;
        if (src + 16 <= gend) cp_async16(base + 16u * u, src);
        else
            for (uint32_t b = 0; b < 16u && src + b < gend; ++b) rbuf[16u * u + b] = src[b];
    }
}

template <bool F64>
__device__ void decode_chunk(const Job &job, const Pending &pd, const uint8_t *rbuf, uint8_t *pbuf, int lane) {
    using T = Traits<F64>;
    using U = typename T::U;

    const uint64_t c = pd.t - job.chunk_begin;
    const uint32_t B = job.block;
    const uint64_t first = c * (uint64_t)B;
    const uint32_t m = (uint32_t)((job.n - first) < B ? (job.n - first) : B);
    const uint32_t cols = chunk_cols(m);
    const uint32_t nact = cols / 32u;
    const uint32_t row_bytes = cols / 8u;
    const uint32_t size = pd.size;
    const uint32_t sh = pd.sh;
    const uint8_t *rec = rbuf + sh;

    // ---- 1. header, flags, rows -> plane words ---------------------------------------------
    bool bad = pd.bad;
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
#pragma unroll 1
    for (int p = (int)w - 1; p >= 0 && !bad; --p) {
        uint32_t x = 0;
        if ((dense_mask >> p) & 1ull) {
            if (pos + row_bytes > size) { bad = true; break; }
            if (active) x = ld_u32_unaligned(rbuf, sh + pos + 4u * lane);
            pos += row_bytes;
        } else {
            if (pos + bm_bytes > size) { bad = true; break; }
            uint32_t nib = 0;
            if (active) {
                const uint32_t byte = rec[pos + (lane >> 1)];
                nib = (lane & 1) ? (byte & 0xFu) : (byte >> 4);
            }
            const uint32_t cnt = __popc(nib);
            const unsigned b0 = __ballot_sync(kFull, cnt & 1u);
            const unsigned b1 = __ballot_sync(kFull, cnt & 2u);
            const unsigned b2 = __ballot_sync(kFull, cnt & 4u);
            const unsigned lt = (1u << lane) - 1u;
            const uint32_t before = __popc(b0 & lt) + 2u * __popc(b1 & lt) + 4u * __popc(b2 & lt);
            const uint32_t nnz = __popc(b0) + 2u * __popc(b1) + 4u * __popc(b2);
            if (pos + bm_bytes + nnz > size) { bad = true; break; }
            uint32_t q = pos + bm_bytes + before;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if ((nib >> (3 - i)) & 1u) x |= (uint32_t)rec[q++] << (8 * i);
            pos += bm_bytes + nnz;
        }
        *reinterpret_cast<uint32_t *>(pbuf + p * 128 + 4 * lane) = x;
    }
    if (pos != size) bad = true;
    if (bad) {
        if (lane == 0) set_status(job.result, kErrCorrupt);
        return;
    }
    __syncwarp();

    // ---- 2. Z -> G -> values -------------------------------------------------------------------
    U d[32];
    {
        uint32_t a[32];
#pragma unroll
        for (int p = 0; p < 32; ++p) a[p] = ((uint32_t)p < w) ? *reinterpret_cast<const uint32_t *>(pbuf + p * 128 + 4 * lane) : 0u;
        transpose32(a);
#pragma unroll
        for (int k = 0; k < 32; ++k) d[k] = (U)a[k ^ 7];
    }
    if constexpr (F64) {
        if (w > 32) {
            uint32_t a[32];
#pragma unroll
            for (int p = 0; p < 32; ++p)
                a[p] = ((uint32_t)(p + 32) < w) ? *reinterpret_cast<const uint32_t *>(pbuf + (p + 32) * 128 + 4 * lane) : 0u;
            transpose32(a);
#pragma unroll
            for (int k = 0; k < 32; ++k) d[k] |= (U)a[k ^ 7] << 32;
        }
    }
    U run = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) { run += unzigzag(d[k]); d[k] = run; }
    U lane_off;
    if constexpr (F64) lane_off = warp_exclusive_u64(run, lane);
    else lane_off = (U)warp_exclusive_u64((uint64_t)run, lane);
    const U gbase = z1 + lane_off;               // G of value 32*lane + k + 1 = gbase + d[k]
    const bool case1 = alpha <= (uint32_t)T::A_MAX && beta_hat <= (uint32_t)T::B_MAX;
    if (case1) {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const U gk = gbase + d[k];
            if constexpr (F64) d[k] = (U)__double_as_longlong(div_pow10((int64_t)gk, (int)alpha));
            else d[k] = (U)__float_as_uint(div_pow10((int32_t)gk, (int)alpha));
        }
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) d[k] = unzigzag((U)(gbase + d[k]));
    }
    U v0;
    if (case1) {
        if constexpr (F64) v0 = (U)__double_as_longlong(div_pow10((int64_t)z1, (int)alpha));
        else v0 = (U)__float_as_uint(div_pow10((int32_t)z1, (int)alpha));
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

    // ---- 3. stage (swizzled) and store -----------------------------------------------------------
    constexpr int UN = T::UNITS;
#pragma unroll
    for (int u = 0; u < UN; ++u) {
        uint4 q;
        if constexpr (F64) {
            q = make_uint4((uint32_t)d[2 * u], (uint32_t)((uint64_t)d[2 * u] >> 32),
                           (uint32_t)d[2 * u + 1], (uint32_t)((uint64_t)d[2 * u + 1] >> 32));
        } else {
            q = make_uint4((uint32_t)d[4 * u], (uint32_t)d[4 * u + 1], (uint32_t)d[4 * u + 2], (uint32_t)d[4 * u + 3]);
        }
        *reinterpret_cast<uint4 *>(pbuf + (lane * UN + (u ^ (lane & 7))) * 16) = q;
    }
    if (m > 1024u && lane == 31) *reinterpret_cast<U *>(pbuf + phys_elem_byte<F64>(1024)) = vx;
    __syncwarp();
    uint8_t *dst = job.out + first * T::S;
    const uint32_t nbytes = m * T::S;
    uint32_t done = 0;
    if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
        const uint32_t nunits = nbytes >> 4;
        for (uint32_t q = lane; q < nunits; q += 32)
            *reinterpret_cast<uint4 *>(dst + 16u * q) = *reinterpret_cast<const uint4 *>(pbuf + phys_unit<F64>(q) * 16u);
        done = (nunits * 16u) / T::S;
    }
    for (uint32_t e = done + lane; e < m; e += 32)
        *reinterpret_cast<U *>(dst + (size_t)e * T::S) = *reinterpret_cast<const U *>(pbuf + phys_elem_byte<F64>(e));
    __syncwarp();
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 2)
decompress_kernel(const Job *__restrict__ jobs, int njobs, Job single, uint64_t total_chunks, Control *ctl) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint8_t *wbase = smem + warp * kWarpBytes;
    uint8_t *pbuf = wbase + 2 * kBuf;
    {
        const int gw = blockIdx.x * kWarpsPerCta + warp;
        const int nw = gridDim.x * kWarpsPerCta;
        const int nj = (jobs != nullptr) ? njobs : 1;
        for (int j = gw; j < nj; j += nw) {
            const Job &jb = (jobs != nullptr) ? jobs[j] : single;
            if (lane == 0) jb.result[0] = jb.n;
        }
    }
    int cur = 0;
    Pending pd{}, pn{};
    uint64_t t = 0;
    if (lane == 0) t = atomicAdd(&ctl->ticket, 1ull);
    t = shfl_u64(t, 0);
    if (t < total_chunks) prepare(job_of(jobs, njobs, single, t), t, wbase, lane, ctl, pd);
    cp_async_commit();
    while (t < total_chunks) {
        uint64_t tn = 0;
        if (lane == 0) tn = atomicAdd(&ctl->ticket, 1ull);
        tn = shfl_u64(tn, 0);
        pn.ok = true;
        if (tn < total_chunks) prepare(job_of(jobs, njobs, single, tn), tn, wbase + (cur ^ 1) * kBuf, lane, ctl, pn);
        cp_async_commit();
        cp_async_wait_prior();                   // the current record has landed
        __syncwarp();
        const Job &job = job_of(jobs, njobs, single, t);
        if (!pd.ok) {
            if (lane == 0) set_status(job.result, kErrTimeout);
            break;
        }
        if (job.dtype == 0) decode_chunk<true>(job, pd, wbase + cur * kBuf, pbuf, lane);
        else decode_chunk<false>(job, pd, wbase + cur * kBuf, pbuf, lane);
        if (!pn.ok && tn < total_chunks) {
            if (lane == 0) set_status(job_of(jobs, njobs, single, tn).result, kErrTimeout);
            break;
        }
        t = tn;
        pd = pn;
        cur ^= 1;
    }
    cp_async_wait_none();
}

constexpr int kDecompressCtaSmem = kWarpsPerCta * kWarpBytes;

static int g_grid_cache[64] = {0};

int decompress_grid(uint64_t total_chunks) {
    int dev = 0;
    cudaGetDevice(&dev);
    int &cached = g_grid_cache[dev & 63];
    if (cached == 0) {
        cudaFuncSetAttribute(decompress_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDecompressCtaSmem);
        int sms = 0, occ = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, decompress_kernel, kThreads, kDecompressCtaSmem);
        cached = sms * (occ > 0 ? occ : 1);
    }
    const uint64_t need = (total_chunks + kWarpsPerCta - 1) / kWarpsPerCta;
    return (int)(need < (uint64_t)cached ? (need > 0 ? need : 1) : (uint64_t)cached);
}

cudaError_t launch_decompress(const Job *d_jobs, int njobs, const Job &single, uint64_t total_chunks,
                              Control *ctl, cudaStream_t stream) {
    const int grid = decompress_grid(total_chunks);
    decompress_kernel<<<grid, kThreads, kDecompressCtaSmem, stream>>>(d_jobs, njobs, single, total_chunks, ctl);
    return cudaGetLastError();
}

}  // namespace falcon
