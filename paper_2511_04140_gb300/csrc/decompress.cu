// Falcon decompression kernel (Sec. 4 of the paper) for sm_103a.
//
// Persistent launch, one warp per chunk (dynamic ticket).  Per chunk:
//   1. exclusive prefix of the u32 size array by decoupled look-back -> record offset,
//   2. the record is staged in shared memory with cp.async (16-byte window),
//   3. header and flags are parsed; every row is expanded into per-lane plane words
//      (dense: an unaligned 4-byte read; sparse: bitmap nibble + popcount rank),
//   4. 32x32 register transposes give Z back, unzigzag + warp scan give G (inverse
//      Eq. 5), and Case 1 divides by 10^alpha (correctly rounded) while Case 2 undoes the
//      zigzag of the IEEE bits (inverse Eq. 4),
//   5. values are staged (swizzled) and written with coalesced 16-byte stores.
// Every read of the record is bounds-checked against its size; a malformed record sets
// FALCON_ERR_CORRUPT and writes nothing.
#include "falcon_device.cuh"

namespace falcon {

namespace {

__device__ __forceinline__ uint32_t ld_u8(const uint8_t *b, uint32_t i) { return b[i]; }

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

template <bool F64>
__device__ void decompress_chunk(const Job &job, uint64_t c, uint8_t *wsm, int lane, Control *ctl) {
    using T = Traits<F64>;
    using U = typename T::U;

    const uint32_t B = job.block;
    const uint64_t first = c * (uint64_t)B;
    const uint32_t m = (uint32_t)((job.n - first) < B ? (job.n - first) : B);
    const uint64_t data_start = 32ull + 4ull * job.nchunks;
    const uint32_t cols = chunk_cols(m);
    const uint32_t nact = cols / 32u;
    const uint32_t row_bytes = cols / 8u;
    const uint32_t max_rec = 3u + T::Z1B + T::W / 8u + T::W * row_bytes;

    // ---- 1. record offset ----------------------------------------------------------------
    uint32_t size = 0;
    if (lane == 0) size = *reinterpret_cast<const uint32_t *>(job.in + 32 + 4 * c);
    size = __shfl_sync(kFull, size, 0);
    bool ok;
    const uint64_t excl = lookback(job.flags, c, size, lane, ctl, ok);
    if (!ok) {
        if (lane == 0) set_status(job.result, kErrTimeout);
        return;
    }
    const uint64_t rec_off = data_start + excl;
    bool bad = (size < 3u + T::Z1B) || (size > max_rec) || (rec_off + size > job.in_bytes) ||
               (rec_off + size < rec_off);

    // ---- 2. stage the record --------------------------------------------------------------
    const uint8_t *gsrc = job.in + rec_off;
    const uint32_t sh = (uint32_t)(reinterpret_cast<uintptr_t>(gsrc) & 15u);
    if (!bad) {
        const uint8_t *gbase = gsrc - sh;                       // >= job.in (16-byte aligned)
        const uint8_t *gend = job.in + job.in_bytes;
        const uint32_t total = sh + size;
        const uint32_t units = (total + 15u) / 16u;
        const uint32_t base = smem_addr(wsm);
        for (uint32_t u = lane; u < units; u += 32) {
            const uint8_t *src = gbase + 16u * u;
            if (src + 16 <= gend) {
                cp_async16(base + 16u * u, src);
            } else {
                for (uint32_t b = 0; b < 16u && src + b < gend; ++b) wsm[16u * u + b] = src[b];
            }
        }
        cp_async_wait_all();
    }
    __syncwarp();

    // ---- 3. parse the header and the rows ------------------------------------------------
    const uint8_t *rec = wsm + sh;
    uint32_t alpha = 0, beta_hat = 0, w = 0;
    U z1 = 0;
    uint64_t dense_mask = 0;
    uint32_t pos = 0;
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
    uint32_t plo[32], phi[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) { plo[j] = 0; phi[j] = 0; }
    const bool active = (uint32_t)lane < nact;
#pragma unroll
    for (int p = T::W - 1; p >= 0; --p) {
        if (!bad && (uint32_t)p < w) {
            uint32_t x = 0;
            if ((dense_mask >> p) & 1ull) {
                if (pos + row_bytes > size) bad = true;
                else if (active) x = ld_u32_unaligned(wsm, sh + pos + 4u * lane);
                pos += row_bytes;
            } else {
                const uint32_t bm_bytes = nact / 2u;
                if (pos + bm_bytes > size) {
                    bad = true;
                } else {
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
                    if (pos + bm_bytes + nnz > size) {
                        bad = true;
                    } else {
                        uint32_t q = pos + bm_bytes + before;
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if ((nib >> (3 - i)) & 1u) x |= ld_u8(rec, q++) << (8 * i);
                    }
                    pos += bm_bytes + nnz;
                }
            }
            if (p < 32) plo[p & 31] = x;
            else phi[p & 31] = x;
        }
    }
    if (pos != size) bad = true;
    if (bad) {
        if (lane == 0) set_status(job.result, kErrCorrupt);
        return;
    }
    __syncwarp();                                   // the record buffer is reused below

    // ---- 4. Z -> G -> values ----------------------------------------------------------------
    transpose32(plo);
    if (F64 && w > 32) transpose32(phi);
    U val[32];                                      // value index 32*lane + k + 1
    {
        U d[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const int j = k ^ 7;
            const U zk = F64 ? (U)(((uint64_t)phi[j] << 32) | plo[j]) : (U)plo[j];
            d[k] = unzigzag(zk);
        }
        U run = 0;
#pragma unroll
        for (int k = 0; k < 32; ++k) { run += d[k]; d[k] = run; }
        U lane_off;
        if constexpr (F64) lane_off = warp_exclusive_u64(run, lane);
        else lane_off = (U)warp_exclusive_u64((uint64_t)run, lane);
        const U gbase = z1 + lane_off;
        const bool case1 = alpha <= (uint32_t)T::A_MAX && beta_hat <= (uint32_t)T::B_MAX;
        if (case1) {
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const U gk = gbase + d[k];
                if constexpr (F64) val[k] = (U)__double_as_longlong(div_pow10((int64_t)gk, (int)alpha));
                else val[k] = (U)__float_as_uint(div_pow10((int32_t)gk, (int)alpha));
            }
        } else {
#pragma unroll
            for (int k = 0; k < 32; ++k) val[k] = unzigzag((U)(gbase + d[k]));
        }
        // value 0 from z_1
        U v0;
        if (case1) {
            if constexpr (F64) v0 = (U)__double_as_longlong(div_pow10((int64_t)z1, (int)alpha));
            else v0 = (U)__float_as_uint(div_pow10((int32_t)z1, (int)alpha));
        } else {
            v0 = unzigzag(z1);
        }
        // shift by one so that lane l holds values 32l .. 32l+31 (value 1024 stays in vx)
        U carry = shfl_up_x(val[31], 1);
        if (lane == 0) carry = v0;
        const U vx = val[31];
#pragma unroll
        for (int k = 31; k > 0; --k) val[k] = val[k - 1];
        val[0] = carry;

        // ---- 5. stage (swizzled) and store --------------------------------------------------
        constexpr int UN = T::UNITS;
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            uint4 q;
            if constexpr (F64) {
                q = make_uint4((uint32_t)val[2 * u], (uint32_t)((uint64_t)val[2 * u] >> 32),
                               (uint32_t)val[2 * u + 1], (uint32_t)((uint64_t)val[2 * u + 1] >> 32));
            } else {
                q = make_uint4((uint32_t)val[4 * u], (uint32_t)val[4 * u + 1], (uint32_t)val[4 * u + 2],
                               (uint32_t)val[4 * u + 3]);
            }
            *reinterpret_cast<uint4 *>(wsm + (lane * UN + (u ^ (lane & 7))) * 16) = q;
        }
        if (m > 1024u && lane == 31) *reinterpret_cast<U *>(wsm + phys_elem_byte<F64>(1024)) = vx;
    }
    __syncwarp();
    uint8_t *dst = job.out + first * T::S;
    const uint32_t nbytes = m * T::S;
    uint32_t done = 0;
    if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
        const uint32_t nunits = nbytes >> 4;
        for (uint32_t q = lane; q < nunits; q += 32)
            *reinterpret_cast<uint4 *>(dst + 16u * q) = *reinterpret_cast<const uint4 *>(wsm + phys_unit<F64>(q) * 16u);
        done = (nunits * 16u) / T::S;
    }
    for (uint32_t e = done + lane; e < m; e += 32)
        *reinterpret_cast<U *>(dst + (size_t)e * T::S) = *reinterpret_cast<const U *>(wsm + phys_elem_byte<F64>(e));
    __syncwarp();
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 4)
decompress_kernel(const Job *__restrict__ jobs, int njobs, Job single, uint64_t total_chunks,
                  Control *ctl) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint8_t *wsm = smem + warp * kWarpSmem;
    if (jobs != nullptr) {
        const int gw = blockIdx.x * kWarpsPerCta + warp;
        const int nw = gridDim.x * kWarpsPerCta;
        for (int j = gw; j < njobs; j += nw)
            if (lane == 0) jobs[j].result[0] = jobs[j].n;
    } else if (blockIdx.x == 0 && threadIdx.x == 0) {
        single.result[0] = single.n;
    }
    while (true) {
        uint64_t t = 0;
        if (lane == 0) t = atomicAdd(&ctl->ticket, 1ull);
        t = shfl_u64(t, 0);
        if (t >= total_chunks) break;
        if (*reinterpret_cast<volatile unsigned int *>(&ctl->abort)) break;
        const Job &job = (jobs == nullptr) ? single : jobs[find_job(jobs, njobs, t)];
        const uint64_t c = t - job.chunk_begin;
        if (job.dtype == 0) decompress_chunk<true>(job, c, wsm, lane, ctl);
        else decompress_chunk<false>(job, c, wsm, lane, ctl);
    }
}

static int g_grid_cache[64] = {0};

int decompress_grid(uint64_t total_chunks) {
    int dev = 0;
    cudaGetDevice(&dev);
    int &cached = g_grid_cache[dev & 63];
    if (cached == 0) {
        int sms = 0, occ = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, decompress_kernel, kThreads, kCtaSmem);
        cached = sms * (occ > 0 ? occ : 1);
    }
    const uint64_t need = (total_chunks + kWarpsPerCta - 1) / kWarpsPerCta;
    return (int)(need < (uint64_t)cached ? (need > 0 ? need : 1) : (uint64_t)cached);
}

cudaError_t launch_decompress(const Job *d_jobs, int njobs, const Job &single, uint64_t total_chunks,
                              Control *ctl, cudaStream_t stream) {
    const int grid = decompress_grid(total_chunks);
    decompress_kernel<<<grid, kThreads, kCtaSmem, stream>>>(d_jobs, njobs, single, total_chunks, ctl);
    return cudaGetLastError();
}

}  // namespace falcon
