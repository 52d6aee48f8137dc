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
static_assert(kScratchBytes == 1057024, "scratch size as documented in falcon.h");

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

extern "C" int falcon_compress_noalloc(const void *d_in, uint64_t n, int dtype, uint32_t block_size, void *d_out,
                                       size_t out_capacity, uint64_t *d_result, void *stream) {
    if (block_size >= 2) {
        const uint64_t chunks = n / block_size + (n % block_size != 0);
        if (chunks > FALCON_NOALLOC_MAX_CHUNKS) return FALCON_ERR_UNSUPPORTED;
    }
    void *scratch = nullptr;
    const int st = scratch_address(&scratch);
    if (st) return st;
    // zeroes the control block, the look-back words in use and d_result on `stream`, then
    // launches the kernel
    return falcon_compress_async(d_in, n, dtype, block_size, d_out, out_capacity, scratch, kScratchBytes, d_result,
                                 stream);
}
