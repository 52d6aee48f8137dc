// C-ABI entry points of libfalcon (declared in include/falcon.h): argument checks,
// workspace management and kernel launches.  No compute happens here.
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "falcon.h"
#include "falcon_internal.h"

using namespace falcon;

void falcon_pipeline_release();
void falcon_noalloc_release();

namespace falcon {
int g_ctas_per_sm[2] = {0, 0};
int g_cta_warps[2] = {kWarpsPerCta, kWarpsPerCta};
}

namespace {

constexpr size_t kResultOffset = 64;     // plain API: 2 x u64 result inside the control block

uint64_t num_chunks(uint64_t n, uint32_t block) { return (n + block - 1) / block; }
size_t elem_bytes(int dtype) { return dtype_bytes(dtype); }

int check_block(uint32_t block) {
    if (block < 2 || block > kMaxBlock) return FALCON_ERR_INVALID;
    return FALCON_OK;
}

size_t record_bound(uint64_t m, int dtype) {
    const size_t W = 8 * dtype_bytes(dtype);
    const size_t cols = m <= 1 ? 0 : ((m - 1 + 63) / 64) * 64;
    return 2 + W / 8 + 1 + W / 8 + W * (cols / 8);
}

// Library-owned workspaces for the synchronous entry points, one per (device, stream).
struct Workspace {
    void *ptr = nullptr;
    size_t bytes = 0;
};
std::mutex g_mu;
std::unordered_map<uint64_t, Workspace> g_ws;

int get_workspace(cudaStream_t stream, size_t bytes, void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FALCON_ERR_CUDA;
    const uint64_t key = ((uint64_t)dev << 56) ^ (uint64_t)(uintptr_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace &w = g_ws[key];
    if (w.bytes < bytes) {
        if (w.ptr) {
            cudaStreamSynchronize(stream);
            cudaFree(w.ptr);
            w.ptr = nullptr;
            w.bytes = 0;
        }
        size_t sz = bytes < (1u << 20) ? (1u << 20) : bytes + bytes / 4;
        if (cudaMalloc(&w.ptr, sz) != cudaSuccess) return FALCON_ERR_CUDA;
        w.bytes = sz;
    }
    *out = w.ptr;
    return FALCON_OK;
}

struct Header {
    uint64_t n, nchunks;
    uint32_t block;
    int dtype;
};

int parse_header(const uint8_t *h, size_t len, Header *out) {
    if (len < FALCON_HEADER_BYTES) return FALCON_ERR_CORRUPT;
    if (std::memcmp(h, "FLCN", 4) != 0 || h[4] != 1 || h[6] != 0 || h[7] != 0) return FALCON_ERR_CORRUPT;
    Header r;
    r.dtype = h[5];
    std::memcpy(&r.block, h + 8, 4);
    std::memcpy(&r.n, h + 16, 8);
    std::memcpy(&r.nchunks, h + 24, 8);
    if (!dtype_valid(r.dtype)) return FALCON_ERR_CORRUPT;
    if (r.block < 2 || r.block > kMaxBlock) return FALCON_ERR_CORRUPT;
    if (r.nchunks != num_chunks(r.n, r.block)) return FALCON_ERR_CORRUPT;
    *out = r;
    return FALCON_OK;
}

}  // namespace

// Argument checks shared by every compression entry point (falcon_internal.h).
int falcon::compress_args(const void *d_in, uint64_t n, int dtype, uint32_t block, void *d_out,
                          size_t out_capacity) {
    if (!dtype_valid(dtype)) return FALCON_ERR_INVALID;
    int st = check_block(block);
    if (st) return st;
    if (!d_out || (n > 0 && !d_in)) return FALCON_ERR_INVALID;
    if ((uintptr_t)d_in % elem_bytes(dtype) != 0 || (uintptr_t)d_out % 16 != 0) return FALCON_ERR_INVALID;
    if (out_capacity < FALCON_HEADER_BYTES + 4 * num_chunks(n, block)) return FALCON_ERR_CAPACITY;
    return FALCON_OK;
}

namespace {

Job make_compress_job(const void *d_in, uint64_t n, int dtype, uint32_t block, void *d_out,
                      size_t out_capacity, void *flags, uint64_t *result) {
    Job j{};
    j.in = static_cast<const uint8_t *>(d_in);
    j.out = static_cast<uint8_t *>(d_out);
    j.in_bytes = n * elem_bytes(dtype);
    j.out_cap = out_capacity;
    j.n = n;
    j.nchunks = num_chunks(n, block);
    j.chunk_begin = 0;
    j.flags = static_cast<unsigned long long *>(flags);
    j.result = reinterpret_cast<unsigned long long *>(result);
    j.block = block;
    j.dtype = (uint32_t)dtype;
    return j;
}

int decompress_args(const void *d_in, size_t in_bytes, const Header &h, void *d_out,
                    size_t out_capacity_bytes) {
    int st = check_block(h.block);
    if (st) return st == FALCON_ERR_INVALID ? FALCON_ERR_CORRUPT : st;
    if (!d_in || (h.n > 0 && !d_out)) return FALCON_ERR_INVALID;
    if ((uintptr_t)d_in % 16 != 0 || (uintptr_t)d_out % elem_bytes(h.dtype) != 0) return FALCON_ERR_INVALID;
    if (h.nchunks > (in_bytes - FALCON_HEADER_BYTES) / 4) return FALCON_ERR_CORRUPT;
    if (h.n > out_capacity_bytes / elem_bytes(h.dtype)) return FALCON_ERR_CAPACITY;
    return FALCON_OK;
}

Job make_decompress_job(const void *d_in, size_t in_bytes, const Header &h, void *d_out,
                        size_t out_capacity_bytes, void *flags, uint64_t *result) {
    Job j{};
    j.in = static_cast<const uint8_t *>(d_in);
    j.out = static_cast<uint8_t *>(d_out);
    j.in_bytes = in_bytes;
    j.out_cap = out_capacity_bytes;
    j.n = h.n;
    j.nchunks = h.nchunks;
    j.chunk_begin = 0;
    j.flags = static_cast<unsigned long long *>(flags);
    j.result = reinterpret_cast<unsigned long long *>(result);
    j.block = h.block;
    j.dtype = (uint32_t)h.dtype;
    return j;
}

int finish_sync(cudaStream_t stream, const void *d_result, uint64_t *value) {
    uint64_t h[2] = {0, 0};
    if (cudaMemcpyAsync(h, d_result, sizeof h, cudaMemcpyDeviceToHost, stream) != cudaSuccess) return FALCON_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return FALCON_ERR_CUDA;
    if (h[1] != 0) return (int)h[1];
    *value = h[0];
    return FALCON_OK;
}

}  // namespace

extern "C" {

int falcon_abi_version(void) { return FALCON_ABI_VERSION; }

const char *falcon_status_string(int status) {
    switch (status) {
        case FALCON_OK: return "ok";
        case FALCON_ERR_INVALID: return "invalid argument";
        case FALCON_ERR_CAPACITY: return "output capacity too small";
        case FALCON_ERR_CORRUPT: return "corrupt stream";
        case FALCON_ERR_CUDA: return "CUDA error";
        case FALCON_ERR_TIMEOUT: return "device wait timed out";
        case FALCON_ERR_UNSUPPORTED: return "unsupported parameter";
        default: return "unknown status";
    }
}

size_t falcon_bound(uint64_t n, int dtype, uint32_t block_size) {
    if (!dtype_valid(dtype) || block_size < 2 || block_size > kMaxBlock) return 0;
    const uint64_t nc = num_chunks(n, block_size);
    size_t total = FALCON_HEADER_BYTES + 4 * (size_t)nc;
    if (nc == 0) return total;
    total += (size_t)(nc - 1) * record_bound(block_size, dtype);
    total += record_bound(n - (nc - 1) * (uint64_t)block_size, dtype);
    return total;
}

int falcon_stream_info(const void *h_header, size_t len, uint64_t *n, int *dtype, uint32_t *block_size,
                       uint64_t *nchunks) {
    if (!h_header) return FALCON_ERR_INVALID;
    Header h;
    const int st = parse_header(static_cast<const uint8_t *>(h_header), len, &h);
    if (st) return st;
    if (n) *n = h.n;
    if (dtype) *dtype = h.dtype;
    if (block_size) *block_size = h.block;
    if (nchunks) *nchunks = h.nchunks;
    return FALCON_OK;
}

size_t falcon_workspace_bytes(uint64_t nchunks) {
    const size_t words = (size_t)workspace_words(nchunks);
    return kControlBytes + ((8 * words + 255) / 256) * 256;
}

int falcon_compress(const void *d_in, uint64_t n, int dtype, uint32_t block_size, void *d_out,
                    size_t out_capacity, size_t *out_bytes, void *stream) {
    int st = compress_args(d_in, n, dtype, block_size, d_out, out_capacity);
    if (st) return st;
    if (!out_bytes) return FALCON_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t nc = num_chunks(n, block_size);
    const size_t ws_bytes = falcon_workspace_bytes(nc);
    void *ws = nullptr;
    if ((st = get_workspace(s, ws_bytes, &ws))) return st;
    if (cudaMemsetAsync(ws, 0, ws_bytes, s) != cudaSuccess) return FALCON_ERR_CUDA;
    uint8_t *w8 = static_cast<uint8_t *>(ws);
    uint64_t *result = reinterpret_cast<uint64_t *>(w8 + kResultOffset);
    const Job j = make_compress_job(d_in, n, dtype, block_size, d_out, out_capacity, w8 + kControlBytes, result);
    if (launch_compress(nullptr, 1, j, nc, reinterpret_cast<Control *>(ws), s) != cudaSuccess) return FALCON_ERR_CUDA;
    uint64_t v = 0;
    st = finish_sync(s, result, &v);
    if (st) return st;
    *out_bytes = (size_t)v;
    return FALCON_OK;
}

int falcon_compress_async(const void *d_in, uint64_t n, int dtype, uint32_t block_size, void *d_out,
                          size_t out_capacity, void *d_workspace, size_t workspace_bytes,
                          uint64_t *d_result, void *stream) {
    return falcon_compress_variant_async(d_in, n, dtype, block_size, FALCON_VARIANT_FALCON, d_out, out_capacity,
                                         d_workspace, workspace_bytes, d_result, stream);
}

size_t falcon_variant_bound(uint64_t n, int dtype, uint32_t block_size, int variant) {
    if (variant < FALCON_VARIANT_FALCON || variant > FALCON_VARIANT_ELF) return 0;
    size_t total = falcon_bound(n, dtype, block_size);
    if (total == 0 || variant != FALCON_VARIANT_SPARSE) return total;
    const uint64_t nc = num_chunks(n, block_size);
    if (nc == 0) return total;
    const size_t W = 8 * dtype_bytes(dtype);
    auto cols = [](uint64_t m) -> size_t { return m <= 1 ? 0 : ((m - 1 + 63) / 64) * 64; };
    total += (size_t)(nc - 1) * W * (cols(block_size) / 64);
    total += W * (cols(n - (nc - 1) * (uint64_t)block_size) / 64);
    return total;
}

int falcon_compress_variant_async(const void *d_in, uint64_t n, int dtype, uint32_t block_size, int variant,
                                  void *d_out, size_t out_capacity, void *d_workspace, size_t workspace_bytes,
                                  uint64_t *d_result, void *stream) {
    if (variant < FALCON_VARIANT_FALCON || variant > FALCON_VARIANT_ELF) return FALCON_ERR_INVALID;
    int st = compress_args(d_in, n, dtype, block_size, d_out, out_capacity);
    if (st) return st;
    const uint64_t nc = num_chunks(n, block_size);
    const size_t need = falcon_workspace_bytes(nc);
    if (!d_workspace || !d_result || workspace_bytes < need || (uintptr_t)d_workspace % 256 != 0 ||
        (uintptr_t)d_result % 8 != 0)
        return FALCON_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_workspace, 0, need, s) != cudaSuccess) return FALCON_ERR_CUDA;
    if (cudaMemsetAsync(d_result, 0, 16, s) != cudaSuccess) return FALCON_ERR_CUDA;
    uint8_t *w8 = static_cast<uint8_t *>(d_workspace);
    Job j = make_compress_job(d_in, n, dtype, block_size, d_out, out_capacity, w8 + kControlBytes, d_result);
    j.variant = (uint32_t)variant;
    if (launch_compress(nullptr, 1, j, nc, reinterpret_cast<Control *>(d_workspace), s) != cudaSuccess)
        return FALCON_ERR_CUDA;
    return FALCON_OK;
}

int falcon_decompress(const void *d_in, size_t in_bytes, void *d_out, size_t out_capacity_bytes,
                      uint64_t *n_out, void *stream) {
    if (!d_in || !n_out) return FALCON_ERR_INVALID;
    if ((uintptr_t)d_in % 16 != 0) return FALCON_ERR_INVALID;
    if (in_bytes < FALCON_HEADER_BYTES) return FALCON_ERR_CORRUPT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t hdr[FALCON_HEADER_BYTES];
    if (cudaMemcpyAsync(hdr, d_in, sizeof hdr, cudaMemcpyDeviceToHost, s) != cudaSuccess) return FALCON_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FALCON_ERR_CUDA;
    Header h;
    int st = parse_header(hdr, sizeof hdr, &h);
    if (st) return st;
    if ((st = decompress_args(d_in, in_bytes, h, d_out, out_capacity_bytes))) return st;
    const size_t ws_bytes = falcon_workspace_bytes(h.nchunks);
    void *ws = nullptr;
    if ((st = get_workspace(s, ws_bytes, &ws))) return st;
    if (cudaMemsetAsync(ws, 0, ws_bytes, s) != cudaSuccess) return FALCON_ERR_CUDA;
    uint8_t *w8 = static_cast<uint8_t *>(ws);
    uint64_t *result = reinterpret_cast<uint64_t *>(w8 + kResultOffset);
    const Job j = make_decompress_job(d_in, in_bytes, h, d_out, out_capacity_bytes, w8 + kControlBytes, result);
    if (launch_decompress(nullptr, 1, j, h.nchunks, reinterpret_cast<Control *>(ws), s) != cudaSuccess)
        return FALCON_ERR_CUDA;
    uint64_t v = 0;
    st = finish_sync(s, result, &v);
    if (st) return st;
    *n_out = v;
    return FALCON_OK;
}

int falcon_decompress_async(const void *d_in, size_t in_bytes, const void *h_header, void *d_out,
                            size_t out_capacity_bytes, void *d_workspace, size_t workspace_bytes,
                            uint64_t *d_result, void *stream) {
    if (!d_in || !h_header) return FALCON_ERR_INVALID;
    if (in_bytes < FALCON_HEADER_BYTES) return FALCON_ERR_CORRUPT;
    Header h;
    int st = parse_header(static_cast<const uint8_t *>(h_header), FALCON_HEADER_BYTES, &h);
    if (st) return st;
    if ((st = decompress_args(d_in, in_bytes, h, d_out, out_capacity_bytes))) return st;
    const size_t need = falcon_workspace_bytes(h.nchunks);
    if (!d_workspace || !d_result || workspace_bytes < need || (uintptr_t)d_workspace % 256 != 0 ||
        (uintptr_t)d_result % 8 != 0)
        return FALCON_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_workspace, 0, need, s) != cudaSuccess) return FALCON_ERR_CUDA;
    if (cudaMemsetAsync(d_result, 0, 16, s) != cudaSuccess) return FALCON_ERR_CUDA;
    uint8_t *w8 = static_cast<uint8_t *>(d_workspace);
    const Job j = make_decompress_job(d_in, in_bytes, h, d_out, out_capacity_bytes, w8 + kControlBytes, d_result);
    if (launch_decompress(nullptr, 1, j, h.nchunks, reinterpret_cast<Control *>(d_workspace), s) != cudaSuccess)
        return FALCON_ERR_CUDA;
    return FALCON_OK;
}

int falcon_aggregate_async(const void *d_in, size_t in_bytes, const void *h_header, void *d_workspace,
                           size_t workspace_bytes, falcon_stats *d_stats, void *stream) {
    if (!d_in || !h_header) return FALCON_ERR_INVALID;
    if (in_bytes < FALCON_HEADER_BYTES) return FALCON_ERR_CORRUPT;
    Header h;
    int st = parse_header(static_cast<const uint8_t *>(h_header), FALCON_HEADER_BYTES, &h);
    if (st) return st;
    if ((uintptr_t)d_in % 16 != 0) return FALCON_ERR_INVALID;
    if (h.nchunks > (in_bytes - FALCON_HEADER_BYTES) / 4) return FALCON_ERR_CORRUPT;
    const size_t need = falcon_workspace_bytes(h.nchunks);
    if (!d_workspace || !d_stats || workspace_bytes < need || (uintptr_t)d_workspace % 256 != 0 ||
        (uintptr_t)d_stats % 8 != 0)
        return FALCON_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_workspace, 0, need, s) != cudaSuccess) return FALCON_ERR_CUDA;
    uint8_t *w8 = static_cast<uint8_t *>(d_workspace);
    // no values are stored: the job has no output; its status word sits in the control region
    uint64_t *result = reinterpret_cast<uint64_t *>(w8 + kResultOffset);
    const Job j = make_decompress_job(d_in, in_bytes, h, nullptr, 0, w8 + kControlBytes, result);
    if (launch_aggregate(j, reinterpret_cast<Control *>(d_workspace), d_stats, s) != cudaSuccess)
        return FALCON_ERR_CUDA;
    return FALCON_OK;
}

int falcon_aggregate(const void *d_in, size_t in_bytes, falcon_stats *h_stats, void *stream) {
    if (!d_in || !h_stats) return FALCON_ERR_INVALID;
    if ((uintptr_t)d_in % 16 != 0) return FALCON_ERR_INVALID;
    if (in_bytes < FALCON_HEADER_BYTES) return FALCON_ERR_CORRUPT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t hdr[FALCON_HEADER_BYTES];
    if (cudaMemcpyAsync(hdr, d_in, sizeof hdr, cudaMemcpyDeviceToHost, s) != cudaSuccess) return FALCON_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FALCON_ERR_CUDA;
    Header h;
    int st = parse_header(hdr, sizeof hdr, &h);
    if (st) return st;
    // the workspace, then one falcon_stats after it, in the cached buffer
    const size_t ws_bytes = falcon_workspace_bytes(h.nchunks);
    void *ws = nullptr;
    if ((st = get_workspace(s, ws_bytes + 256, &ws))) return st;
    falcon_stats *d_stats = reinterpret_cast<falcon_stats *>(static_cast<uint8_t *>(ws) + ws_bytes);
    if ((st = falcon_aggregate_async(d_in, in_bytes, hdr, ws, ws_bytes, d_stats, stream))) return st;
    if (cudaMemcpyAsync(h_stats, d_stats, sizeof(falcon_stats), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FALCON_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FALCON_ERR_CUDA;
    return (int)h_stats->status;
}

int falcon_release(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : g_ws) {
        if (kv.second.ptr) {
            cudaSetDevice((int)(kv.first >> 56));
            cudaFree(kv.second.ptr);
        }
    }
    g_ws.clear();
    cudaSetDevice(cur);
    falcon_pipeline_release();
    falcon_noalloc_release();
    return FALCON_OK;
}

}  // extern "C"

/* ------------------------------------------------------------------------- batched form */

namespace {
struct BatchPlan {
    int direction;
    int count;
    uint64_t total_chunks;
    size_t reset_bytes;       // control block + workspace words, zeroed before each launch
    uint64_t *d_results;
};
std::mutex g_plan_mu;
std::unordered_map<uintptr_t, BatchPlan> g_plans;

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Host-side job table for a batch (no device pointers dereferenced); returns a status.
int build_jobs(int direction, const falcon_series *series, int count, std::vector<Job> &jobs,
               uint64_t &total_chunks, size_t &words) {
    jobs.resize((size_t)count);
    total_chunks = 0;
    words = 0;
    for (int i = 0; i < count; ++i) {
        const falcon_series &sr = series[i];
        Job j{};
        if (direction == FALCON_COMPRESS) {
            const int st = compress_args(sr.d_in, sr.n, sr.dtype, sr.block_size, sr.d_out, sr.out_capacity);
            if (st) return st;
            j = make_compress_job(sr.d_in, sr.n, sr.dtype, sr.block_size, sr.d_out, sr.out_capacity, nullptr, nullptr);
        } else if (direction == FALCON_DECOMPRESS) {
            if (!sr.h_header || !sr.d_in) return FALCON_ERR_INVALID;
            if ((uintptr_t)sr.d_in % 16 != 0) return FALCON_ERR_INVALID;
            if (sr.in_bytes < FALCON_HEADER_BYTES) return FALCON_ERR_CORRUPT;
            Header h;
            int st = parse_header(static_cast<const uint8_t *>(sr.h_header), FALCON_HEADER_BYTES, &h);
            if (st) return st;
            if ((st = decompress_args(sr.d_in, sr.in_bytes, h, sr.d_out, sr.out_capacity))) return st;
            j = make_decompress_job(sr.d_in, sr.in_bytes, h, sr.d_out, sr.out_capacity, nullptr, nullptr);
        } else {
            return FALCON_ERR_INVALID;
        }
        j.chunk_begin = total_chunks;
        total_chunks += j.nchunks;
        // per-chunk workspace words, 8-byte each
        j.flags = reinterpret_cast<unsigned long long *>((uintptr_t)words);   // offset, fixed up later
        words += (size_t)workspace_words(j.nchunks);
        jobs[(size_t)i] = j;
    }
    return FALCON_OK;
}
}  // namespace

extern "C" {

size_t falcon_batch_workspace_bytes(int direction, const falcon_series *h_series, int count) {
    if (count < 0 || (count > 0 && !h_series)) return 0;
    std::vector<Job> jobs;
    uint64_t total = 0;
    size_t words = 0;
    if (build_jobs(direction, h_series, count, jobs, total, words) != FALCON_OK) return 0;
    return kControlBytes + align256(sizeof(Job) * (size_t)count) + align256(8 * words);
}

int falcon_batch_plan(int direction, const falcon_series *h_series, int count, void *d_workspace,
                      size_t workspace_bytes, uint64_t *d_results, void *stream) {
    if (count < 0 || (count > 0 && (!h_series || !d_results)) || !d_workspace) return FALCON_ERR_INVALID;
    if ((uintptr_t)d_workspace % 256 != 0 || (uintptr_t)d_results % 8 != 0) return FALCON_ERR_INVALID;
    std::vector<Job> jobs;
    uint64_t total = 0;
    size_t words = 0;
    int st = build_jobs(direction, h_series, count, jobs, total, words);
    if (st) return st;
    const size_t table = align256(sizeof(Job) * (size_t)count);
    const size_t need = kControlBytes + table + align256(8 * words);
    if (workspace_bytes < need) return FALCON_ERR_INVALID;
    uint8_t *w8 = static_cast<uint8_t *>(d_workspace);
    unsigned long long *flags = reinterpret_cast<unsigned long long *>(w8 + kControlBytes + table);
    for (int i = 0; i < count; ++i) {
        jobs[(size_t)i].flags = flags + (uintptr_t)jobs[(size_t)i].flags;
        jobs[(size_t)i].result = reinterpret_cast<unsigned long long *>(d_results + 2 * (size_t)i);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (count > 0 &&
        cudaMemcpyAsync(w8 + kControlBytes, jobs.data(), sizeof(Job) * (size_t)count, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return FALCON_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FALCON_ERR_CUDA;   // the host table is freed below
    BatchPlan plan{direction, count, total, kControlBytes + table + 8 * words, d_results};
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans[(uintptr_t)d_workspace] = plan;
    return FALCON_OK;
}

int falcon_batch_launch(void *d_workspace, void *stream) {
    BatchPlan plan;
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        auto it = g_plans.find((uintptr_t)d_workspace);
        if (it == g_plans.end()) return FALCON_ERR_INVALID;
        plan = it->second;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *w8 = static_cast<uint8_t *>(d_workspace);
    // the control block and the workspace words; the job table in between is kept
    const size_t table = align256(sizeof(Job) * (size_t)plan.count);
    if (cudaMemsetAsync(w8, 0, kControlBytes, s) != cudaSuccess) return FALCON_ERR_CUDA;
    if (plan.reset_bytes > kControlBytes + table &&
        cudaMemsetAsync(w8 + kControlBytes + table, 0, plan.reset_bytes - kControlBytes - table, s) != cudaSuccess)
        return FALCON_ERR_CUDA;
    if (plan.count > 0 && cudaMemsetAsync(plan.d_results, 0, 16 * (size_t)plan.count, s) != cudaSuccess)
        return FALCON_ERR_CUDA;
    if (plan.count == 0) return FALCON_OK;
    const Job *d_jobs = reinterpret_cast<const Job *>(w8 + kControlBytes);
    Control *ctl = reinterpret_cast<Control *>(w8);
    Job dummy{};
    const cudaError_t e = (plan.direction == FALCON_COMPRESS)
                              ? launch_compress(d_jobs, plan.count, dummy, plan.total_chunks, ctl, s)
                              : launch_decompress(d_jobs, plan.count, dummy, plan.total_chunks, ctl, s);
    return e == cudaSuccess ? FALCON_OK : FALCON_ERR_CUDA;
}

int falcon_batch_forget(void *d_workspace) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans.erase((uintptr_t)d_workspace);
    return FALCON_OK;
}

int falcon_set_cta_warps(int compress_warps, int decompress_warps) {
    if (compress_warps < 1 || compress_warps > kMaxCompressWarps || decompress_warps < 1 ||
        decompress_warps > kMaxDecompressWarps)
        return FALCON_ERR_INVALID;
    g_cta_warps[0] = compress_warps;
    g_cta_warps[1] = decompress_warps;
    return FALCON_OK;
}

int falcon_set_launch_config(int compress_ctas_per_sm, int decompress_ctas_per_sm) {
    if (compress_ctas_per_sm < 0 || decompress_ctas_per_sm < 0) return FALCON_ERR_INVALID;
    g_ctas_per_sm[0] = compress_ctas_per_sm;
    g_ctas_per_sm[1] = decompress_ctas_per_sm;
    return FALCON_OK;
}

}  // extern "C"
