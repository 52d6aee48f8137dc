// falcon_compress_noalloc: compression whose workspace scratch is a fixed device array of
// this file instead of caller- or library-allocated memory.  Host code plus one static
// device symbol; the work itself is falcon_compress_async's.
#include <mutex>

#include "falcon.h"
#include "falcon_internal.h"

namespace {

// control block + the per-chunk workspace words, in the layout falcon_workspace_bytes
// describes, for FALCON_NOALLOC_MAX_CHUNKS chunks
constexpr size_t kWords = falcon::workspace_words(FALCON_NOALLOC_MAX_CHUNKS);
constexpr size_t kScratchBytes = falcon::kControlBytes + (8 * kWords + 255) / 256 * 256;
static_assert(kScratchBytes == 1057280, "scratch size as documented in falcon.h");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per device.
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FALCON_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return FALCON_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return FALCON_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return FALCON_OK;
}

}  // namespace

// Forgets the looked-up addresses (falcon_release): after a context reset the array lives at
// a new address, which the next call looks up again.
void falcon_noalloc_release() {
    std::lock_guard<std::mutex> lk(g_mu);
    for (void *&p : g_addr) p = nullptr;
}

extern "C" int falcon_compress_noalloc(const void *d_in, uint64_t n, int dtype, uint32_t block_size, void *d_out,
                                       size_t out_capacity, uint64_t *d_result, void *stream) {
    // the argument errors first, as falcon_compress_async reports them, then the size limit
    int st = falcon::compress_args(d_in, n, dtype, block_size, d_out, out_capacity);
    if (st) return st;
    if (!d_result || (uintptr_t)d_result % 8 != 0) return FALCON_ERR_INVALID;
    const uint64_t chunks = n / block_size + (n % block_size != 0);
    if (chunks > FALCON_NOALLOC_MAX_CHUNKS) return FALCON_ERR_UNSUPPORTED;
    void *scratch = nullptr;
    if ((st = scratch_address(&scratch))) return st;
    // zeroes, on `stream`, the control block, the per-chunk words this call uses and
    // d_result, then enqueues the three compression launches
    return falcon_compress_async(d_in, n, dtype, block_size, d_out, out_capacity, scratch, kScratchBytes, d_result,
                                 stream);
}
