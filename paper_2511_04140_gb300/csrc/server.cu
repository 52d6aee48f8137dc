// Continuous-batching request server (falcon_server_* in include/falcon.h): host code only.
//
// One worker thread per server repeats:
//   1. take the newly submitted requests into the FIFO queue;
//   2. admit from the head of the queue while the request's device block (input, output,
//      per-chunk workspace words) fits the device arena and its output fits the host arena,
//      at most max_batch requests (and max_batch_bytes of input, so that batches pipeline)
//      and one batch slot per direction;
//   3. per direction with admitted requests, enqueue
//        up stream:      H2D inputs                                           -> event U
//        compute stream: wait U; job-table H2D; control/result reset; batched
//                        persistent kernel; per-request result D2H             -> event K
//        down stream:    (decompress only) wait K; output D2H into the host arena -> event O
//   4. poll the batches in flight: once K has fired for a compress batch, read each stream
//      length and enqueue the output D2H -> event O; once O has fired, release the device
//      blocks, shrink compress outputs to their length and publish the completions.
// Nothing on this path allocates device or pinned memory per request: both arenas are
// allocated once, and a first-fit allocator with neighbour coalescing hands out blocks.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "falcon.h"
#include "falcon_internal.h"

using namespace falcon;

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kGranule = 256;
size_t granules(size_t bytes) { return ((bytes ? bytes : 1) + kGranule - 1) / kGranule * kGranule; }

// First-fit allocator over [0, capacity) in 256-byte granules; freed blocks merge with free
// neighbours.  Not thread-safe (callers lock).
class Arena {
  public:
    void init(size_t capacity) {
        free_.clear();
        capacity_ = capacity / kGranule * kGranule;
        if (capacity_) free_[0] = capacity_;
        used_ = peak_ = 0;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = granules(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, tail = it->first + bytes;
            free_.erase(it);
            if (rest) free_[tail] = rest;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = granules(bytes);
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                off = prev->first;
                bytes += prev->second;
                free_.erase(prev);
            }
        }
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            free_.erase(next);
        }
        free_[off] = bytes;
    }
    size_t capacity() const { return capacity_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

  private:
    std::map<size_t, size_t> free_;   // offset -> bytes
    size_t capacity_ = 0, used_ = 0, peak_ = 0;
};

struct Request {
    uint64_t tag = 0;
    int op = 0;
    const uint8_t *h_in = nullptr;
    uint64_t in_bytes = 0, n = 0, nchunks = 0, out_cap = 0;
    int dtype = 0;
    uint32_t block = 0;
    size_t words = 0;                  // per-chunk workspace words
    size_t dev_bytes = 0, dev_off = 0;
    size_t host_bytes = 0, host_off = 0;
    Clock::time_point t_submit;
    uint64_t value = 0;                // stream bytes / values reported by the kernel
    int status = FALCON_OK;

    size_t in_span() const { return granules(in_bytes); }
    size_t out_span() const { return granules(out_cap); }
};

// Per-batch device area [Control | 2 x u64 results x max_batch | job table] and its pinned
// host mirrors, reused once the batch that held it has completed.
struct Slot {
    uint8_t *d_area = nullptr;
    Job *h_jobs = nullptr;
    unsigned long long *h_results = nullptr;
    cudaEvent_t up = nullptr, kernel = nullptr, out = nullptr;
    bool busy = false;
};

struct Batch {
    Slot *slot = nullptr;
    int op = 0;
    int stage = 0;                     // 0: kernel pending; 1: output copies pending
    std::vector<Request> reqs;
};

size_t elem(int dtype) { return dtype_bytes(dtype); }

}  // namespace

struct falcon_server {
    int device = 0;
    int max_batch = 0;
    size_t max_batch_bytes = 0;        // 0: no limit
    uint8_t *d_base = nullptr;
    Arena dev;                         // worker thread only
    uint8_t *h_base = nullptr;
    Arena host;                        // guarded by host_mu
    std::mutex host_mu;
    std::unordered_map<uintptr_t, size_t> live;   // output pointer -> bytes held (host_mu)
    cudaStream_t up = nullptr, down[2] = {nullptr, nullptr};
    std::vector<cudaStream_t> compute;
    size_t next_compute = 0;
    std::vector<Slot> slots;

    std::mutex mu;                     // submission queue and shutdown
    std::condition_variable cv;
    std::deque<Request> submitted;
    bool stop = false;
    std::atomic<bool> broken{false};   // a CUDA call failed: every later request fails

    std::mutex done_mu;                // completion queue
    std::condition_variable done_cv;
    std::deque<falcon_completion> done;

    std::mutex stats_mu;
    falcon_server_stats st{};
    uint64_t in_flight = 0;            // worker thread only

    std::thread worker;

    size_t results_bytes() const { return granules(16 * (size_t)max_batch); }
    Job *d_jobs(Slot &s) const { return reinterpret_cast<Job *>(s.d_area + kControlBytes + results_bytes()); }
    unsigned long long *d_results(Slot &s) const {
        return reinterpret_cast<unsigned long long *>(s.d_area + kControlBytes);
    }

    Slot *take_slot() {
        for (Slot &s : slots)
            if (!s.busy) {
                s.busy = true;
                return &s;
            }
        return nullptr;
    }

    void publish(std::vector<falcon_completion> &out) {
        if (out.empty()) return;
        {
            std::lock_guard<std::mutex> lk(done_mu);
            for (auto &c : out) done.push_back(c);
        }
        done_cv.notify_all();
    }

    falcon_completion failed(const Request &r, int status) {
        falcon_completion c{};
        c.tag = r.tag;
        c.status = status;
        c.op = r.op;
        c.values = r.n;
        c.latency_s = std::chrono::duration<double>(Clock::now() - r.t_submit).count();
        return c;
    }

    // Admits from the head of `pending` and enqueues one batch per direction.
    bool launch_admitted(std::deque<Request> &pending, std::vector<Batch> &inflight) {
        if (pending.empty()) return false;
        Batch b[2];
        b[0].op = FALCON_COMPRESS;
        b[1].op = FALCON_DECOMPRESS;
        size_t in_bytes[2] = {0, 0};
        {
            std::lock_guard<std::mutex> hl(host_mu);
            while (!pending.empty()) {
                Request &r = pending.front();
                Batch &g = b[r.op];
                if (g.reqs.size() >= (size_t)max_batch) break;
                if (max_batch_bytes && !g.reqs.empty() && in_bytes[r.op] + r.in_bytes > max_batch_bytes) break;
                if (!g.slot && !(g.slot = take_slot())) break;
                if (!dev.alloc(r.dev_bytes, &r.dev_off)) break;
                if (!host.alloc(r.host_bytes, &r.host_off)) {
                    dev.release(r.dev_off, r.dev_bytes);
                    break;
                }
                in_bytes[r.op] += r.in_bytes;
                g.reqs.push_back(r);
                pending.pop_front();
            }
            std::lock_guard<std::mutex> sl(stats_mu);
            st.device_in_use = dev.used();
            st.device_peak = dev.peak();
            st.host_in_use = host.used();
            st.host_peak = host.peak();
        }
        bool any = false;
        for (Batch &g : b) {
            if (g.reqs.empty()) {
                if (g.slot) g.slot->busy = false;
                continue;
            }
            any = true;
            in_flight += g.reqs.size();
            {
                std::lock_guard<std::mutex> sl(stats_mu);
                st.batches += 1;
                st.multi_request_batches += g.reqs.size() > 1;
                st.max_batch = std::max<uint64_t>(st.max_batch, g.reqs.size());
                st.max_in_flight = std::max<uint64_t>(st.max_in_flight, in_flight);
            }
            if (enqueue(g) != FALCON_OK) broken = true;
            inflight.push_back(std::move(g));
        }
        return any;
    }

    int enqueue(Batch &g) {
        Slot &s = *g.slot;
        const int count = (int)g.reqs.size();
        unsigned long long *res = d_results(s);
        uint64_t total = 0;
        for (int i = 0; i < count; ++i) {
            Request &r = g.reqs[(size_t)i];
            uint8_t *d_in = d_base + r.dev_off;
            uint8_t *d_out = d_in + r.in_span();
            auto *words = reinterpret_cast<unsigned long long *>(d_out + r.out_span());
            Job j{};
            j.in = d_in;
            j.out = d_out;
            j.in_bytes = r.in_bytes;
            j.out_cap = r.out_cap;
            j.n = r.n;
            j.nchunks = r.nchunks;
            j.chunk_begin = total;
            j.flags = words;
            j.result = res + 2 * i;
            j.block = r.block;
            j.dtype = (uint32_t)r.dtype;
            total += r.nchunks;
            s.h_jobs[i] = j;
            if (r.in_bytes && cudaMemcpyAsync(d_in, r.h_in, r.in_bytes, cudaMemcpyHostToDevice, up) != cudaSuccess)
                return FALCON_ERR_CUDA;
        }
        if (cudaEventRecord(s.up, up) != cudaSuccess) return FALCON_ERR_CUDA;
        cudaStream_t cs = compute[next_compute++ % compute.size()];
        if (cudaStreamWaitEvent(cs, s.up, 0) != cudaSuccess) return FALCON_ERR_CUDA;
        if (cudaMemcpyAsync(d_jobs(s), s.h_jobs, sizeof(Job) * (size_t)count, cudaMemcpyHostToDevice, cs) != cudaSuccess)
            return FALCON_ERR_CUDA;
        if (cudaMemsetAsync(s.d_area, 0, kControlBytes + 16 * (size_t)count, cs) != cudaSuccess) return FALCON_ERR_CUDA;
        if (g.op == FALCON_COMPRESS)            // the analysis adds record sizes to per-tile and per-group sums
            for (const Request &r : g.reqs) {
                if (r.nchunks == 0) continue;
                auto *words = reinterpret_cast<unsigned long long *>(d_base + r.dev_off + r.in_span() + r.out_span());
                if (cudaMemsetAsync(words + 2 * r.nchunks, 0, 8 * (tile_count(r.nchunks) + group_count(r.nchunks)),
                                    cs) != cudaSuccess)
                    return FALCON_ERR_CUDA;
            }
        Job dummy{};
        auto *ctl = reinterpret_cast<Control *>(s.d_area);
        const cudaError_t e = g.op == FALCON_COMPRESS ? launch_compress(d_jobs(s), count, dummy, total, ctl, cs)
                                                       : launch_decompress(d_jobs(s), count, dummy, total, ctl, cs);
        if (e != cudaSuccess) return FALCON_ERR_CUDA;
        if (cudaMemcpyAsync(s.h_results, res, 16 * (size_t)count, cudaMemcpyDeviceToHost, cs) != cudaSuccess)
            return FALCON_ERR_CUDA;
        if (cudaEventRecord(s.kernel, cs) != cudaSuccess) return FALCON_ERR_CUDA;
        if (g.op == FALCON_DECOMPRESS) {
            if (cudaStreamWaitEvent(down[1], s.kernel, 0) != cudaSuccess) return FALCON_ERR_CUDA;
            for (Request &r : g.reqs)
                if (r.out_cap && cudaMemcpyAsync(h_base + r.host_off, d_base + r.dev_off + r.in_span(), r.out_cap,
                                                 cudaMemcpyDeviceToHost, down[1]) != cudaSuccess)
                    return FALCON_ERR_CUDA;
            if (cudaEventRecord(s.out, down[1]) != cudaSuccess) return FALCON_ERR_CUDA;
        }
        g.stage = 0;
        return FALCON_OK;
    }

    // Advances the batches in flight; returns whether anything moved.
    bool poll(std::vector<Batch> &inflight) {
        bool moved = false;
        for (size_t i = 0; i < inflight.size();) {
            Batch &g = inflight[i];
            Slot &s = *g.slot;
            if (g.stage == 0) {
                const cudaError_t q = cudaEventQuery(s.kernel);
                if (q == cudaErrorNotReady) {
                    ++i;
                    continue;
                }
                if (q != cudaSuccess) {
                    broken = true;
                    return moved;
                }
                for (size_t k = 0; k < g.reqs.size(); ++k) {
                    Request &r = g.reqs[k];
                    r.value = s.h_results[2 * k];
                    r.status = (int)s.h_results[2 * k + 1];
                    if (r.status == FALCON_OK && g.op == FALCON_COMPRESS && r.value > r.out_cap)
                        r.status = FALCON_ERR_CAPACITY;
                    if (r.status == FALCON_OK && g.op == FALCON_DECOMPRESS && r.value != r.n)
                        r.status = FALCON_ERR_CORRUPT;
                }
                if (g.op == FALCON_COMPRESS) {
                    for (Request &r : g.reqs)
                        if (r.status == FALCON_OK &&
                            cudaMemcpyAsync(h_base + r.host_off, d_base + r.dev_off + r.in_span(), r.value,
                                            cudaMemcpyDeviceToHost, down[0]) != cudaSuccess) {
                            broken = true;
                            return moved;
                        }
                    if (cudaEventRecord(s.out, down[0]) != cudaSuccess) {
                        broken = true;
                        return moved;
                    }
                }
                g.stage = 1;
                moved = true;
            }
            const cudaError_t q = cudaEventQuery(s.out);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            if (q != cudaSuccess) {
                broken = true;
                return moved;
            }
            complete(g);
            inflight.erase(inflight.begin() + (std::ptrdiff_t)i);
            moved = true;
        }
        return moved;
    }

    void complete(Batch &g) {
        std::vector<falcon_completion> out;
        out.reserve(g.reqs.size());
        uint64_t ok = 0, bad = 0;
        {
            std::lock_guard<std::mutex> hl(host_mu);
            for (Request &r : g.reqs) {
                dev.release(r.dev_off, r.dev_bytes);
                falcon_completion c = failed(r, r.status);
                if (r.status == FALCON_OK) {
                    const uint64_t bytes = g.op == FALCON_COMPRESS ? r.value : r.n * elem(r.dtype);
                    const size_t keep = granules(bytes);
                    if (keep < r.host_bytes) host.release(r.host_off + keep, r.host_bytes - keep);
                    c.h_out = h_base + r.host_off;
                    c.out_bytes = bytes;
                    live[(uintptr_t)c.h_out] = keep;
                    ++ok;
                } else {
                    host.release(r.host_off, r.host_bytes);
                    ++bad;
                }
                out.push_back(c);
            }
            std::lock_guard<std::mutex> sl(stats_mu);
            st.completed += ok + bad;
            st.failed += bad;
            st.device_in_use = dev.used();
            st.host_in_use = host.used();
        }
        in_flight -= g.reqs.size();
        g.slot->busy = false;
        publish(out);
    }

    void fail_all(std::deque<Request> &pending, std::vector<Batch> &inflight, int status) {
        std::vector<falcon_completion> out;
        for (Request &r : pending) out.push_back(failed(r, status));
        for (Batch &g : inflight)
            for (Request &r : g.reqs) out.push_back(failed(r, status));
        {
            std::lock_guard<std::mutex> sl(stats_mu);
            st.completed += out.size();
            st.failed += out.size();
        }
        pending.clear();
        inflight.clear();          // device and host blocks of a broken server are not reused
        publish(out);
    }

    void run() {
        cudaSetDevice(device);
        std::deque<Request> pending;
        std::vector<Batch> inflight;
        for (;;) {
            bool stopping;
            {
                std::unique_lock<std::mutex> lk(mu);
                if (pending.empty() && inflight.empty() && submitted.empty()) {
                    if (stop) return;
                    cv.wait(lk, [&] { return stop || !submitted.empty(); });
                    if (submitted.empty()) return;
                }
                while (!submitted.empty()) {
                    pending.push_back(submitted.front());
                    submitted.pop_front();
                }
                stopping = stop;
                if (broken) {
                    lk.unlock();
                    fail_all(pending, inflight, FALCON_ERR_CUDA);
                    continue;
                }
            }
            bool moved = launch_admitted(pending, inflight);
            moved |= poll(inflight);
            if (moved) continue;
            if (!inflight.empty()) {
                std::this_thread::yield();
            } else if (!pending.empty()) {
                // queue head waits for host-arena room that only the client can free
                if (stopping) {
                    std::deque<Request> rest;
                    rest.swap(pending);
                    std::vector<Batch> none;
                    fail_all(rest, none, FALCON_ERR_CAPACITY);
                    continue;
                }
                std::unique_lock<std::mutex> lk(mu);
                cv.wait_for(lk, std::chrono::microseconds(200));
            }
        }
    }
};

extern "C" {

int falcon_server_create(int device, size_t device_budget_bytes, size_t host_budget_bytes, int compute_streams,
                         int max_batch, size_t max_batch_bytes, falcon_server **out) {
    if (!out || compute_streams < 1 || compute_streams > 64 || max_batch < 1 || max_batch > 65536 ||
        device_budget_bytes < kGranule || host_budget_bytes < kGranule)
        return FALCON_ERR_INVALID;
    *out = nullptr;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return FALCON_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return FALCON_ERR_INVALID;
    auto *s = new falcon_server();
    s->device = device;
    s->max_batch = max_batch;
    s->max_batch_bytes = max_batch_bytes;
    int st = FALCON_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && st == FALCON_OK) st = FALCON_ERR_CUDA;
        return st == FALCON_OK;
    };
    const size_t dcap = device_budget_bytes / kGranule * kGranule, hcap = host_budget_bytes / kGranule * kGranule;
    if (ok(cudaMalloc(&s->d_base, dcap)) && ok(cudaHostAlloc(&s->h_base, hcap, cudaHostAllocDefault)) &&
        ok(cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking)) &&
        ok(cudaStreamCreateWithFlags(&s->down[0], cudaStreamNonBlocking)) &&
        ok(cudaStreamCreateWithFlags(&s->down[1], cudaStreamNonBlocking))) {
        s->compute.resize((size_t)compute_streams, nullptr);
        for (auto &c : s->compute)
            if (!ok(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking))) break;
    }
    if (st == FALCON_OK) {
        s->slots.resize((size_t)(2 * compute_streams + 4));
        const size_t area = kControlBytes + s->results_bytes() + sizeof(Job) * (size_t)max_batch;
        for (Slot &sl : s->slots) {
            if (!ok(cudaMalloc(&sl.d_area, area)) ||
                !ok(cudaHostAlloc(&sl.h_jobs, sizeof(Job) * (size_t)max_batch, cudaHostAllocDefault)) ||
                !ok(cudaHostAlloc(&sl.h_results, 16 * (size_t)max_batch, cudaHostAllocDefault)) ||
                !ok(cudaEventCreateWithFlags(&sl.up, cudaEventDisableTiming)) ||
                !ok(cudaEventCreateWithFlags(&sl.kernel, cudaEventDisableTiming)) ||
                !ok(cudaEventCreateWithFlags(&sl.out, cudaEventDisableTiming)))
                break;
        }
    }
    s->dev.init(dcap);
    s->host.init(hcap);
    s->st.device_capacity = s->dev.capacity();
    s->st.host_capacity = s->host.capacity();
    if (st == FALCON_OK) {
        s->worker = std::thread([s] { s->run(); });
        *out = s;
    } else {
        falcon_server_destroy(s);
    }
    cudaSetDevice(prev);
    return st;
}

int falcon_server_submit(falcon_server *s, int op, const void *h_in, uint64_t count, int dtype, uint32_t block_size,
                         uint64_t tag) {
    if (!s) return FALCON_ERR_INVALID;
    Request r;
    r.tag = tag;
    r.op = op;
    r.h_in = static_cast<const uint8_t *>(h_in);
    if (op == FALCON_COMPRESS) {
        if (!dtype_valid(dtype)) return FALCON_ERR_INVALID;
        if (block_size < 2 || block_size > kMaxBlock) return FALCON_ERR_INVALID;
        if (count > 0 && !h_in) return FALCON_ERR_INVALID;
        if (count > (1ull << 58)) return FALCON_ERR_CAPACITY;
        r.n = count;
        r.dtype = dtype;
        r.block = block_size;
        r.in_bytes = count * elem(dtype);
        r.nchunks = (count + block_size - 1) / block_size;
        r.out_cap = falcon_bound(count, dtype, block_size);
    } else if (op == FALCON_DECOMPRESS) {
        if (!h_in) return FALCON_ERR_INVALID;
        if (count < FALCON_HEADER_BYTES) return FALCON_ERR_CORRUPT;
        uint64_t n = 0, nc = 0;
        int dt = 0;
        uint32_t blk = 0;
        const int st = falcon_stream_info(h_in, count, &n, &dt, &blk, &nc);
        if (st) return st;
        if (nc > (count - FALCON_HEADER_BYTES) / 4) return FALCON_ERR_CORRUPT;
        if (n > (1ull << 58)) return FALCON_ERR_CAPACITY;
        r.n = n;
        r.dtype = dt;
        r.block = blk;
        r.in_bytes = count;
        r.nchunks = nc;
        r.out_cap = n * elem(dt);
    } else {
        return FALCON_ERR_INVALID;
    }
    r.words = (size_t)workspace_words(r.nchunks);
    r.dev_bytes = r.in_span() + r.out_span() + granules(8 * r.words);
    r.host_bytes = r.out_span();
    if (r.dev_bytes > s->st.device_capacity || r.host_bytes > s->st.host_capacity) return FALCON_ERR_CAPACITY;
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return FALCON_ERR_INVALID;
        if (s->broken) return FALCON_ERR_CUDA;
        s->submitted.push_back(r);
    }
    {
        std::lock_guard<std::mutex> sl(s->stats_mu);
        s->st.submitted += 1;
    }
    s->cv.notify_one();
    return FALCON_OK;
}

int falcon_server_poll(falcon_server *s, falcon_completion *out, int max_completions, int timeout_us, int *count) {
    if (!s || !count || max_completions < 0 || (max_completions > 0 && !out)) return FALCON_ERR_INVALID;
    std::unique_lock<std::mutex> lk(s->done_mu);
    if (s->done.empty() && timeout_us > 0)
        s->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !s->done.empty(); });
    int k = 0;
    while (k < max_completions && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *count = k;
    return FALCON_OK;
}

int falcon_server_free_output(falcon_server *s, const void *h_out) {
    if (!s || !h_out) return FALCON_ERR_INVALID;
    {
        std::lock_guard<std::mutex> hl(s->host_mu);
        auto it = s->live.find((uintptr_t)h_out);
        if (it == s->live.end()) return FALCON_ERR_INVALID;
        s->host.release((size_t)(static_cast<const uint8_t *>(h_out) - s->h_base), it->second);
        s->live.erase(it);
        std::lock_guard<std::mutex> sl(s->stats_mu);
        s->st.host_in_use = s->host.used();
    }
    s->cv.notify_one();
    return FALCON_OK;
}

int falcon_server_get_stats(falcon_server *s, falcon_server_stats *stats) {
    if (!s || !stats) return FALCON_ERR_INVALID;
    std::lock_guard<std::mutex> sl(s->stats_mu);
    *stats = s->st;
    return FALCON_OK;
}

int falcon_server_destroy(falcon_server *s) {
    if (!s) return FALCON_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (cudaStream_t c : s->compute)
        if (c) cudaStreamSynchronize(c);
    for (cudaStream_t c : {s->up, s->down[0], s->down[1]})
        if (c) cudaStreamSynchronize(c);
    for (Slot &sl : s->slots) {
        if (sl.up) cudaEventDestroy(sl.up);
        if (sl.kernel) cudaEventDestroy(sl.kernel);
        if (sl.out) cudaEventDestroy(sl.out);
        if (sl.d_area) cudaFree(sl.d_area);
        if (sl.h_jobs) cudaFreeHost(sl.h_jobs);
        if (sl.h_results) cudaFreeHost(sl.h_results);
    }
    for (cudaStream_t c : s->compute)
        if (c) cudaStreamDestroy(c);
    for (cudaStream_t c : {s->up, s->down[0], s->down[1]})
        if (c) cudaStreamDestroy(c);
    if (s->d_base) cudaFree(s->d_base);
    if (s->h_base) cudaFreeHost(s->h_base);
    cudaSetDevice(prev);
    delete s;
    return FALCON_OK;
}

}  // extern "C"
