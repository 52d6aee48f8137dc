// Host <-> device streaming pipeline (Sec. 3.1, Alg. 1 of the paper): host code only.
//
// Compression runs one of the three schedulers of Sec. 3.1 (Fig. 5), on nstreams CUDA
// stream slots; each frame is a complete stream and the output is the frames in order:
//   event-driven (Alg. 1, the paper's choice): every slot cycles through
//     Idle   -> H2D(frame) ; compress (async) ; D2H(16-byte result) ; event      -> MPend
//     MPend  -> (when this frame is the next one to be placed and its event fired)
//               offset fixed ; D2H(payload -> h_out + offset) ; event            -> PPend
//     PPend  -> (event fired)                                                    -> Idle
//     Frames go to whichever slot is idle, in frame order; offsets are fixed in that order.
//   sync-based: the host waits for each frame's size (M-D2H) before it launches the next
//     frame; only the payload copy (P-D2H) of a frame overlaps the next frame's upload and
//     kernel.
//   pre-allocation: every frame's output goes to a fixed slot of the worst-case size; the
//     whole slot is copied back (bytes past the stream included), then the host merges the
//     frames into h_out in order.
// Decompression knows every frame's output position from its header (pre-allocation), so
// each slot runs H2D -> decompress -> D2H without ordering between slots.
#include <cstring>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "falcon.h"
#include "falcon_internal.h"

namespace {

enum SlotState { kIdle, kMPend, kPPend };

struct Slot {
    cudaStream_t stream = nullptr;
    uint8_t *d_in = nullptr;
    uint8_t *d_out = nullptr;
    uint8_t *d_ws = nullptr;
    uint64_t *d_res = nullptr;
    uint64_t *h_res = nullptr;        // pinned
    uint8_t *h_stage = nullptr;       // pinned, pre-allocation scheduler only
    size_t stage_bytes = 0;
    cudaEvent_t ev = nullptr;
    cudaEvent_t up = nullptr;         // the frame's upload is done
    SlotState state = kIdle;
    uint64_t frame = 0;
};

struct SlotSet {
    std::vector<Slot> slots;
    // one stream for every frame's kernels, in launch order: compression is an order of
    // magnitude faster than the host link, and frames whose kernels ran side by side on
    // several streams could finish out of order, holding up the in-order placement
    cudaStream_t compute = nullptr;
    ~SlotSet() {
        if (compute) {
            cudaStreamSynchronize(compute);
            cudaStreamDestroy(compute);
        }
        for (Slot &s : slots) {
            if (s.stream) cudaStreamSynchronize(s.stream);
            if (s.ev) cudaEventDestroy(s.ev);
            if (s.up) cudaEventDestroy(s.up);
            if (s.stream) cudaStreamDestroy(s.stream);
            cudaFree(s.d_in);
            cudaFree(s.d_out);
            cudaFree(s.d_ws);
            cudaFree(s.d_res);
            if (s.h_res) cudaFreeHost(s.h_res);
            if (s.h_stage) cudaFreeHost(s.h_stage);
        }
    }
    int init(int n, size_t in_bytes, size_t out_bytes, size_t ws_bytes) {
        if (cudaStreamCreateWithFlags(&compute, cudaStreamNonBlocking) != cudaSuccess) return FALCON_ERR_CUDA;
        slots.resize((size_t)n);
        for (Slot &s : slots) {
            if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) return FALCON_ERR_CUDA;
            if (cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess) return FALCON_ERR_CUDA;
            if (cudaEventCreateWithFlags(&s.up, cudaEventDisableTiming) != cudaSuccess) return FALCON_ERR_CUDA;
            if (cudaMalloc(&s.d_in, in_bytes ? in_bytes : 16) != cudaSuccess) return FALCON_ERR_CUDA;
            if (cudaMalloc(&s.d_out, out_bytes ? out_bytes : 16) != cudaSuccess) return FALCON_ERR_CUDA;
            if (cudaMalloc(&s.d_ws, ws_bytes) != cudaSuccess) return FALCON_ERR_CUDA;
            if (cudaMalloc(&s.d_res, 16) != cudaSuccess) return FALCON_ERR_CUDA;
            if (cudaHostAlloc(&s.h_res, 16, cudaHostAllocDefault) != cudaSuccess) return FALCON_ERR_CUDA;
        }
        return FALCON_OK;
    }
};

// Slot sets are kept between calls (per device): allocating a frame's buffers on every
// call would cost more than streaming a few frames.  One call uses a set at a time.
struct CachedSet {
    std::mutex mu;
    std::unique_ptr<SlotSet> set;
    int n = 0;
    size_t in_bytes = 0, out_bytes = 0, ws_bytes = 0;
};
CachedSet g_cache[64];

int acquire_slots(int n, size_t in_bytes, size_t out_bytes, size_t ws_bytes, std::unique_lock<std::mutex> &hold,
                  SlotSet *&out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FALCON_ERR_CUDA;
    CachedSet &c = g_cache[dev & 63];
    hold = std::unique_lock<std::mutex>(c.mu);
    if (!c.set || c.n < n || c.in_bytes < in_bytes || c.out_bytes < out_bytes || c.ws_bytes < ws_bytes) {
        c.set.reset();
        c.set.reset(new SlotSet());
        c.n = n > c.n ? n : c.n;
        c.in_bytes = in_bytes > c.in_bytes ? in_bytes : c.in_bytes;
        c.out_bytes = out_bytes > c.out_bytes ? out_bytes : c.out_bytes;
        c.ws_bytes = ws_bytes > c.ws_bytes ? ws_bytes : c.ws_bytes;
        const int st = c.set->init(c.n, c.in_bytes, c.out_bytes, c.ws_bytes);
        if (st) {
            c.set.reset();
            c.n = 0;
            c.in_bytes = c.out_bytes = c.ws_bytes = 0;
            return st;
        }
    }
    for (Slot &sl : c.set->slots) sl.state = kIdle;
    out = c.set.get();
    return FALCON_OK;
}

}  // namespace

// Frees the cached pipeline buffers of every device (called by falcon_release).
void falcon_pipeline_release() {
    int cur = 0;
    cudaGetDevice(&cur);
    for (int d = 0; d < 64; ++d) {
        std::lock_guard<std::mutex> lk(g_cache[d].mu);
        if (g_cache[d].set) {
            cudaSetDevice(d);
            g_cache[d].set.reset();
            g_cache[d].n = 0;
            g_cache[d].in_bytes = g_cache[d].out_bytes = g_cache[d].ws_bytes = 0;
        }
    }
    cudaSetDevice(cur);
}

extern "C" {

int falcon_pipeline_compress(const void *h_in, uint64_t n, int dtype, uint32_t block_size, uint64_t frame_values,
                             int nstreams, void *h_out, size_t out_capacity, uint64_t *h_frame_bytes,
                             size_t *out_bytes) {
    return falcon_pipeline_compress_with(h_in, n, dtype, block_size, frame_values, nstreams,
                                         FALCON_SCHED_EVENT_DRIVEN, h_out, out_capacity, h_frame_bytes, out_bytes);
}

int falcon_pipeline_compress_with(const void *h_in, uint64_t n, int dtype, uint32_t block_size,
                                  uint64_t frame_values, int nstreams, int scheduler, void *h_out,
                                  size_t out_capacity, uint64_t *h_frame_bytes, size_t *out_bytes) {
    if (!falcon::dtype_valid(dtype) || !h_out || !out_bytes || !h_frame_bytes) return FALCON_ERR_INVALID;
    if (n > 0 && !h_in) return FALCON_ERR_INVALID;
    if (frame_values == 0 || nstreams < 1 || nstreams > 256) return FALCON_ERR_INVALID;
    if (scheduler < FALCON_SCHED_EVENT_DRIVEN || scheduler > FALCON_SCHED_PRE_ALLOCATION) return FALCON_ERR_INVALID;
    if (falcon_bound(frame_values, dtype, block_size) == 0) return FALCON_ERR_INVALID;
    const size_t s = falcon::dtype_bytes(dtype);
    const uint64_t nframes = (n + frame_values - 1) / frame_values;
    const uint64_t fchunks = (frame_values + block_size - 1) / block_size;
    const size_t fbound = falcon_bound(frame_values, dtype, block_size);
    const size_t ws_bytes = falcon_workspace_bytes(fchunks);
    std::unique_lock<std::mutex> hold;
    SlotSet *setp = nullptr;
    const int want = (int)(nframes < (uint64_t)nstreams ? (nframes ? nframes : 1) : (uint64_t)nstreams);
    int st = acquire_slots(want, frame_values * s, fbound, ws_bytes, hold, setp);
    if (st) return st;
    SlotSet &set = *setp;
    const uint64_t ns = (uint64_t)want;
    const uint8_t *in8 = static_cast<const uint8_t *>(h_in);
    uint8_t *out8 = static_cast<uint8_t *>(h_out);
    const bool prealloc = scheduler == FALCON_SCHED_PRE_ALLOCATION;
    if (prealloc) {
        for (uint64_t i = 0; i < ns; ++i) {
            Slot &sl = set.slots[i];
            if (sl.stage_bytes < fbound) {
                if (sl.h_stage) cudaFreeHost(sl.h_stage);
                sl.h_stage = nullptr;
                sl.stage_bytes = 0;
                if (cudaHostAlloc(&sl.h_stage, fbound, cudaHostAllocDefault) != cudaSuccess) return FALCON_ERR_CUDA;
                sl.stage_bytes = fbound;
            }
        }
    }
    // launch: upload, kernels and the result words (pre-allocation: the whole output slot)
    auto launch = [&](Slot &sl, uint64_t f) -> int {
        const uint64_t first = f * frame_values;
        const uint64_t m = (n - first) < frame_values ? (n - first) : frame_values;
        // upload on the slot's stream; kernels and the result words on the shared compute
        // stream, in launch order; the whole output slot (pre-allocation) on the slot's stream
        if (cudaMemcpyAsync(sl.d_in, in8 + first * s, m * s, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
            return FALCON_ERR_CUDA;
        if (cudaEventRecord(sl.up, sl.stream) != cudaSuccess) return FALCON_ERR_CUDA;
        if (cudaStreamWaitEvent(set.compute, sl.up, 0) != cudaSuccess) return FALCON_ERR_CUDA;
        const int r = falcon_compress_async(sl.d_in, m, dtype, block_size, sl.d_out, fbound, sl.d_ws, ws_bytes,
                                            sl.d_res, set.compute);
        if (r) return r;
        if (cudaMemcpyAsync(sl.h_res, sl.d_res, 16, cudaMemcpyDeviceToHost, set.compute) != cudaSuccess)
            return FALCON_ERR_CUDA;
        if (prealloc) {
            if (cudaEventRecord(sl.up, set.compute) != cudaSuccess) return FALCON_ERR_CUDA;
            if (cudaStreamWaitEvent(sl.stream, sl.up, 0) != cudaSuccess) return FALCON_ERR_CUDA;
            if (cudaMemcpyAsync(sl.h_stage, sl.d_out, fbound, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
                return FALCON_ERR_CUDA;
            if (cudaEventRecord(sl.ev, sl.stream) != cudaSuccess) return FALCON_ERR_CUDA;
        } else if (cudaEventRecord(sl.ev, set.compute) != cudaSuccess) {
            return FALCON_ERR_CUDA;
        }
        sl.frame = f;
        sl.state = kMPend;
        return FALCON_OK;
    };
    size_t offset = 0;
    int status = FALCON_OK;
    // places frame sl.frame (its size is back): records it and fixes its offset
    auto place = [&](Slot &sl) -> size_t {
        const uint64_t cs = sl.h_res[0];
        if (sl.h_res[1] != 0 && status == FALCON_OK) status = (int)sl.h_res[1];
        if (status == FALCON_OK && offset + cs > out_capacity) status = FALCON_ERR_CAPACITY;
        h_frame_bytes[sl.frame] = cs;
        return cs;
    };
    if (scheduler == FALCON_SCHED_SYNC_BASED) {
        for (uint64_t f = 0; f < nframes && status == FALCON_OK; ++f) {
            Slot &sl = set.slots[f % ns];
            if (cudaStreamSynchronize(sl.stream) != cudaSuccess) return FALCON_ERR_CUDA;   // its last payload copy
            if ((st = launch(sl, f))) return st;
            if (cudaEventSynchronize(sl.ev) != cudaSuccess) return FALCON_ERR_CUDA;         // M-D2H: the size
            const size_t cs = place(sl);
            if (status == FALCON_OK &&
                cudaMemcpyAsync(out8 + offset, sl.d_out, cs, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
                return FALCON_ERR_CUDA;
            offset += cs;
        }
    } else {
        uint64_t next = 0, placed = 0, done = 0;   // frames launched / placed / finished
        while (done < next || (next < nframes && status == FALCON_OK)) {
            bool progress = false;
            for (uint64_t i = 0; i < ns; ++i) {
                Slot &sl = set.slots[i];
                if (sl.state == kIdle) {
                    if (next < nframes && status == FALCON_OK && next - placed < ns) {
                        if ((st = launch(sl, next))) return st;
                        ++next;
                        progress = true;
                    }
                } else if (sl.state == kMPend) {
                    if (sl.frame != placed) continue;                 // offsets are fixed in launch order
                    const cudaError_t q = cudaEventQuery(sl.ev);
                    if (q == cudaErrorNotReady) continue;
                    if (q != cudaSuccess) return FALCON_ERR_CUDA;
                    const size_t cs = place(sl);
                    if (prealloc) {
                        // the merge step: the frame's bytes from its fixed slot into place
                        if (status == FALCON_OK) std::memcpy(out8 + offset, sl.h_stage, cs);
                        sl.state = kIdle;
                        ++done;
                    } else {
                        if (status == FALCON_OK &&
                            cudaMemcpyAsync(out8 + offset, sl.d_out, cs, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
                            return FALCON_ERR_CUDA;
                        if (cudaEventRecord(sl.ev, sl.stream) != cudaSuccess) return FALCON_ERR_CUDA;
                        sl.state = kPPend;
                    }
                    offset += cs;
                    ++placed;
                    progress = true;
                } else {
                    const cudaError_t q = cudaEventQuery(sl.ev);
                    if (q == cudaErrorNotReady) continue;
                    if (q != cudaSuccess) return FALCON_ERR_CUDA;
                    sl.state = kIdle;
                    ++done;
                    progress = true;
                }
            }
            if (!progress) std::this_thread::yield();
        }
    }
    if (cudaStreamSynchronize(set.compute) != cudaSuccess) return FALCON_ERR_CUDA;
    for (uint64_t i = 0; i < ns; ++i)
        if (cudaStreamSynchronize(set.slots[i].stream) != cudaSuccess) return FALCON_ERR_CUDA;
    if (status != FALCON_OK) return status;
    *out_bytes = offset;
    return FALCON_OK;
}

int falcon_pipeline_decompress(const void *h_in, const uint64_t *h_frame_bytes, uint64_t nframes, int nstreams,
                               void *h_out, size_t out_capacity_bytes, uint64_t *n_out) {
    if (!h_frame_bytes || !n_out || (nframes > 0 && (!h_in || !h_out))) return FALCON_ERR_INVALID;
    if (nstreams < 1 || nstreams > 256) return FALCON_ERR_INVALID;
    const uint8_t *in8 = static_cast<const uint8_t *>(h_in);
    uint8_t *out8 = static_cast<uint8_t *>(h_out);
    // frame positions from the headers (host memory)
    std::vector<uint64_t> in_off(nframes), out_off(nframes), nvals(nframes);
    uint64_t ioff = 0, ooff = 0, total = 0;
    size_t max_in = 16, max_vals = 1, max_chunks = 0;
    for (uint64_t f = 0; f < nframes; ++f) {
        if (h_frame_bytes[f] < FALCON_HEADER_BYTES) return FALCON_ERR_CORRUPT;
        uint64_t nv = 0, nc = 0;
        int dt = 0;
        uint32_t blk = 0;
        const int st = falcon_stream_info(in8 + ioff, h_frame_bytes[f], &nv, &dt, &blk, &nc);
        if (st) return st;
        const size_t s = falcon::dtype_bytes(dt);
        in_off[f] = ioff;
        out_off[f] = ooff;
        nvals[f] = nv;
        ioff += h_frame_bytes[f];
        ooff += nv * s;
        total += nv;
        if (h_frame_bytes[f] > max_in) max_in = h_frame_bytes[f];
        if (nv * s > max_vals) max_vals = nv * s;
        if (nc > max_chunks) max_chunks = nc;
    }
    if (ooff > out_capacity_bytes) return FALCON_ERR_CAPACITY;
    std::unique_lock<std::mutex> hold;
    SlotSet *setp = nullptr;
    const int want = (int)(nframes < (uint64_t)nstreams ? (nframes ? nframes : 1) : (uint64_t)nstreams);
    int st = acquire_slots(want, (max_in + 15) / 16 * 16, max_vals, falcon_workspace_bytes(max_chunks), hold, setp);
    if (st) return st;
    SlotSet &set = *setp;
    const uint64_t ns = (uint64_t)want;
    uint64_t next = 0, done = 0;
    int status = FALCON_OK;
    while (done < nframes) {
        for (uint64_t i = 0; i < ns; ++i) {
            Slot &sl = set.slots[i];
            if (sl.state == kIdle) {
                if (next < nframes && status == FALCON_OK) {
                    const uint64_t f = next++;
                    if (cudaMemcpyAsync(sl.d_in, in8 + in_off[f], h_frame_bytes[f], cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
                        return FALCON_ERR_CUDA;
                    st = falcon_decompress_async(sl.d_in, h_frame_bytes[f], in8 + in_off[f], sl.d_out, max_vals, sl.d_ws,
                                                 falcon_workspace_bytes(max_chunks), sl.d_res, sl.stream);
                    if (st) return st;
                    const size_t s = falcon::dtype_bytes(in8[in_off[f] + 5]);
                    if (cudaMemcpyAsync(out8 + out_off[f], sl.d_out, nvals[f] * s, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
                        return FALCON_ERR_CUDA;
                    if (cudaMemcpyAsync(sl.h_res, sl.d_res, 16, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
                        return FALCON_ERR_CUDA;
                    if (cudaEventRecord(sl.ev, sl.stream) != cudaSuccess) return FALCON_ERR_CUDA;
                    sl.frame = f;
                    sl.state = kPPend;
                }
            } else {
                const cudaError_t q = cudaEventQuery(sl.ev);
                if (q == cudaErrorNotReady) continue;
                if (q != cudaSuccess) return FALCON_ERR_CUDA;
                if (sl.h_res[1] != 0 && status == FALCON_OK) status = (int)sl.h_res[1];
                sl.state = kIdle;
                ++done;
            }
        }
        if (status != FALCON_OK && done == next) break;
    }
    for (uint64_t i = 0; i < ns; ++i)
        if (cudaStreamSynchronize(set.slots[i].stream) != cudaSuccess) return FALCON_ERR_CUDA;
    if (status != FALCON_OK) return status;
    *n_out = total;
    return FALCON_OK;
}

}  // extern "C"
