/*
 * falcon.h -- C ABI of libfalcon, a GB300 (sm_103a) implementation of the Falcon codec:
 * lossless, per-chunk compression of FP64 / FP32 / FP16 series (Falcon: GPU-Based
 * Floating-point Adaptive Lossless Compression, arXiv 2511.04140).
 *
 * What one call computes (per chunk of block_size consecutive values):
 *   - the float-to-integer transform of Sec. 3.2 (Alg. 2 decimal place detection, Eq. 4:
 *     Case 1 g_i = round(v_i * 10^alpha_max) when alpha_max <= 22 and beta_hat_max <= 15,
 *     verified to round-trip bit for bit; otherwise Case 2 g_i = Zigzag(BinLong(v_i)));
 *   - delta + zigzag coding (Eq. 5);
 *   - the adaptive sparse/dense bit-plane encoding of Sec. 3.3 (Fig. 8);
 *   - the compressed-size synchronisation and chunk writing of Sec. 3.4 (Alg. 3): the record
 *     sizes and their sums per 64- and 4096-chunk group, then every record written at its
 *     offset (two kernel launches on the caller's stream, none waiting on another warp);
 * and decompression (Sec. 4) is its exact inverse.  FP32 follows the same steps with
 * alpha <= 10, beta <= 7 and 32-bit integers; FP16 (binary16, FALCON_F16; Sec. 2.1 extends
 * the method to other precisions, this library fixes its constants) with alpha <= 4,
 * beta <= 3, eps <= |x| 2^-10, 16-bit integers and fl16 round trips.
 *
 * Stream format (self-describing, little-endian):
 *   bytes 0..31   "FLCN", version u8 (=1), dtype u8 (falcon_dtype), u16 0, block_size u32, u32 0,
 *                 n u64, num_chunks u64
 *   then          u32 size[num_chunks]  (compressed bytes of each chunk record)
 *   then          the chunk records back to back:
 *                 [alpha_max u8][beta_hat_max u8][z_1: 8 B (FP32: 4 B, FP16: 2 B)][w u8]
 *                 [flags: ceil(w/8) B, the last w bits = rows 1..w, 1 = dense]
 *                 [row 1 = bit plane w-1] ... [row w = bit plane 0]
 *   A sparse row is a bitmap of cols/64 bytes (bit 7 of byte 0 = row byte 0) followed by
 *   the row's non-zero bytes; a dense row is its cols/8 bytes; cols = round_up(m-1, 64)
 *   for a chunk of m values.  Case-2 records carry alpha_max = 23, beta_hat_max = 16
 *   (FP32: 11 and 8; FP16: 5 and 4).
 *
 * Conventions for every entry point:
 *   - Return value: a falcon_status.  Nothing is thrown across the ABI.  On error the
 *     contents of output buffers are undefined.
 *   - "d_" pointers are device pointers (cudaMalloc / torch CUDA storage) on the current
 *     device; "h_" pointers are host pointers.  The caller owns every buffer it passes.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Value buffers must be aligned to the element size; stream buffers to 16 bytes.
 *   - Block sizes: 2 <= block_size <= 1025 (FALCON_MAX_BLOCK).  Sec. 3.3 chooses chunks of
 *     n = 64k + 1 values so that every row of the transposed bit-plane matrix is byte-aligned
 *     and uses n = 1025 (k = 16); the format of this library takes k <= 16 (and any other
 *     n up to 1025, with the zero-pad columns of a partial row).  Larger block sizes are
 *     invalid everywhere: FALCON_ERR_INVALID from the compression entry points, 0 from
 *     falcon_bound, FALCON_ERR_CORRUPT for a stream header that names one.
 */
#ifndef FALCON_H_
#define FALCON_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FALCON_ABI_VERSION 1
#define FALCON_HEADER_BYTES 32
#define FALCON_MAX_BLOCK 1025

typedef enum { FALCON_F64 = 0, FALCON_F32 = 1, FALCON_F16 = 2 } falcon_dtype;

typedef enum {
    FALCON_OK = 0,
    FALCON_ERR_INVALID = 1,     /* bad argument (null pointer, dtype, alignment, ...) */
    FALCON_ERR_CAPACITY = 2,    /* output buffer too small */
    FALCON_ERR_CORRUPT = 3,     /* malformed or truncated compressed stream */
    FALCON_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    FALCON_ERR_TIMEOUT = 5,     /* reserved: no kernel of this version waits on another warp */
    FALCON_ERR_UNSUPPORTED = 6  /* a request beyond a documented limit (FALCON_NOALLOC_MAX_CHUNKS) */
} falcon_status;

/* Library version (FALCON_ABI_VERSION). */
int falcon_abi_version(void);

/* Human-readable name of a status code (static string). */
const char *falcon_status_string(int status);

/* Worst-case stream size in bytes for n values of `dtype` in chunks of block_size:
 * 32 + 4*ceil(n/B) + sum over chunks of (2 + z1 + 1 + W/8 + W*cols/8), W = 64 (FP64) or 32,
 * z1 = W/8 bytes.  The paper fixes only the chunk record (Sec. 3.3, Fig. 8: every row dense
 * at w = W is its largest form) and "size array, then chunk data" (Sec. 3.4); the 32-byte
 * header and the u32 size entries are this library's stream format.  Pure host function;
 * returns 0 for invalid arguments (dtype, or block_size outside 2..1025). */
size_t falcon_bound(uint64_t n, int dtype, uint32_t block_size);

/* Parses the 32-byte header of a stream held in HOST memory (len >= 32).  The header is this
 * library's own (the paper's batch output is the size array and the chunk data, Sec. 3.4,
 * with no header): "FLCN", version 1, dtype, block_size, n and the number of chunks.
 * Outputs may be NULL.  FALCON_ERR_INVALID for a NULL h_header; FALCON_ERR_CORRUPT if the
 * header is malformed (magic, version, dtype, block_size outside 2..1025, or a chunk count
 * other than ceil(n / block_size)). */
int falcon_stream_info(const void *h_header, size_t len, uint64_t *n, int *dtype,
                       uint32_t *block_size, uint64_t *num_chunks);

/* Compresses n values at d_in (FP64 or FP32, device) into d_out (device, out_capacity
 * bytes) and stores the stream length in *out_bytes (host).  Enqueued on `stream`; the
 * call synchronises that stream once to read the length and status back.  Uses a
 * per-(device, stream) workspace cached by the library (freed by falcon_release).
 * Sec. 3 (Alg. 3) of the paper. */
int falcon_compress(const void *d_in, uint64_t n, int dtype, uint32_t block_size,
                    void *d_out, size_t out_capacity, size_t *out_bytes, void *stream);

/* Decompresses the stream at d_in (device, in_bytes) into d_out (device,
 * out_capacity_bytes) and stores the value count in *n_out (host).  Reads the 32-byte
 * header back to the host first, then enqueues the kernel and synchronises `stream` once
 * for the status.  Sec. 4 of the paper. */
int falcon_decompress(const void *d_in, size_t in_bytes, void *d_out, size_t out_capacity_bytes,
                      uint64_t *n_out, void *stream);

/* Device workspace (bytes) needed by the asynchronous entry points for a stream of
 * num_chunks chunks.  Must be 256-byte aligned device memory. */
size_t falcon_workspace_bytes(uint64_t num_chunks);

/* Asynchronous compression: enqueues a workspace reset and the kernels on `stream` and
 * returns without synchronising, so it can be captured in a CUDA graph.
 * d_result (device, 2 x uint64): [0] = stream length in bytes, [1] = falcon_status of the
 * device-side work (the host return value only covers argument checks and launch).
 * d_workspace: falcon_workspace_bytes(ceil(n / block_size)) bytes of device memory owned
 * by the caller; calls that share a workspace must be ordered on one stream. */
int falcon_compress_async(const void *d_in, uint64_t n, int dtype, uint32_t block_size,
                          void *d_out, size_t out_capacity, void *d_workspace,
                          size_t workspace_bytes, uint64_t *d_result, void *stream);

/* Asynchronous decompression.  h_header is a HOST copy of the stream's first 32 bytes
 * (the caller produced the stream or read it back); it sizes the launch.  d_result:
 * [0] = number of values, [1] = falcon_status.  Workspace and capture rules as above. */
int falcon_decompress_async(const void *d_in, size_t in_bytes, const void *h_header,
                            void *d_out, size_t out_capacity_bytes, void *d_workspace,
                            size_t workspace_bytes, uint64_t *d_result, void *stream);

/* ---------------------------------------------------------------------------------------
 * Analytics on compressed data (Sec. 7 names it as future work and fixes nothing; this
 * library's reading): an aggregate of a stream's values computed from its records on the
 * GPU, the records decoded in registers and never written out as values.
 *   count      number of values (n of the header);
 *   nan_count  number of NaN values;
 *   min, max   smallest / largest non-NaN value in IEEE 754 totalOrder (-0 < +0), widened
 *              exactly to FP64; NaN when every value is a NaN or the stream is empty;
 *   sum        sum of the non-NaN values in FP64: each 32-value group in index order, then
 *              fixed trees over groups, chunks and the stream, so the result is reproducible;
 *              within depth * 2^-53 * sum(|x|) of the exact sum (depth: the additions on
 *              any path, 38 + ceil(chunks / 1024) + 10); +0 when there is no non-NaN value;
 *   status     falcon_status of the device-side work (FALCON_ERR_CORRUPT for a malformed
 *              record).
 */
typedef struct {
    uint64_t count;
    uint64_t nan_count;
    double min;
    double max;
    double sum;
    uint64_t status;
} falcon_stats;

/* Asynchronous aggregate of the stream at d_in (device, in_bytes; h_header a host copy of
 * its first 32 bytes) into d_stats (device, one falcon_stats).  d_workspace:
 * falcon_workspace_bytes(number of chunks) bytes of 256-byte aligned device memory owned by
 * the caller.  Enqueues four launches on `stream` and returns without synchronising
 * (capturable).  Errors as falcon_decompress_async. */
int falcon_aggregate_async(const void *d_in, size_t in_bytes, const void *h_header, void *d_workspace,
                           size_t workspace_bytes, falcon_stats *d_stats, void *stream);

/* Synchronous form: reads the header back, uses the library's cached workspace, copies the
 * result to *h_stats (host) and returns its status. */
int falcon_aggregate(const void *d_in, size_t in_bytes, falcon_stats *h_stats, void *stream);

/* ---------------------------------------------------------------------------------------
 * Codec variants: Falcon and the three ablations of Sec. 5.4.2 (Fig. 12b).  Each changes one
 * step and keeps the record layout, so falcon_decompress reads every variant's streams:
 *   FALCON_VARIANT_FALCON  the method itself (what falcon_compress writes);
 *   FALCON_VARIANT_SPARSE  Fal._Sparse: every row of the transposed bit-plane matrix stored
 *                          sparse (bitmap + non-zero bytes), whatever its zero-byte count;
 *   FALCON_VARIANT_DENSE   Fal._Dense: every row stored dense;
 *   FALCON_VARIANT_ELF     Fal._Elf: a value's decimal place is the trial-and-error one of
 *                          Sec. 1 (the first i with v (x) 10^i integral, within Alg. 2's bounds
 *                          alpha <= 22 and beta <= 15; FP32 10 and 7), in place of Alg. 2; the
 *                          chunk's Case decision and round-trip check are Falcon's.
 * ------------------------------------------------------------------------------------- */
typedef enum {
    FALCON_VARIANT_FALCON = 0,
    FALCON_VARIANT_SPARSE = 1,
    FALCON_VARIANT_DENSE = 2,
    FALCON_VARIANT_ELF = 3
} falcon_variant;

/* Worst-case stream size of a variant: falcon_bound, except FALCON_VARIANT_SPARSE, whose rows
 * may each carry their cols/64-byte bitmap on top of cols/8 non-zero bytes.  0 for invalid
 * arguments. */
size_t falcon_variant_bound(uint64_t n, int dtype, uint32_t block_size, int variant);

/* falcon_compress_async for a codec variant (same arguments, workspace, d_result and errors;
 * FALCON_ERR_INVALID for an unknown variant).  Size d_out with falcon_variant_bound. */
int falcon_compress_variant_async(const void *d_in, uint64_t n, int dtype, uint32_t block_size,
                                  int variant, void *d_out, size_t out_capacity, void *d_workspace,
                                  size_t workspace_bytes, uint64_t *d_result, void *stream);

/* Allocation-free compression.  The paper has no counterpart: it is a deployment variant of
 * falcon_compress_async whose scratch (control block and per-chunk words) is a file-scope
 * static device array of the library, sized for FALCON_NOALLOC_MAX_CHUNKS chunks
 * (1,057,280 bytes per device; 67,108,864 values at block_size 1024), instead of a workspace.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 *   - The first call on a device looks the array's address up (cudaGetSymbolAddress, with
 *     that device current) and keeps it; make that first call before any stream capture.
 *   - Zeroes, on `stream`, the scratch words it uses and d_result before the kernels.
 *   - Every call on a device uses the same array: calls that overlap in time (two streams,
 *     or two host threads without ordering) race and corrupt each other's output; order
 *     them on one stream.
 *   - The looked-up address belongs to the device's current context: after a context reset
 *     (cudaDeviceReset) call falcon_release() before the next call, which then looks the
 *     address up again.
 *   - Arguments are checked first, with the errors of falcon_compress_async; then more than
 *     FALCON_NOALLOC_MAX_CHUNKS chunks gives FALCON_ERR_UNSUPPORTED, with nothing enqueued.
 * d_result is as for falcon_compress_async. */
#define FALCON_NOALLOC_MAX_CHUNKS 65536
int falcon_compress_noalloc(const void *d_in, uint64_t n, int dtype, uint32_t block_size,
                            void *d_out, size_t out_capacity, uint64_t *d_result, void *stream);

/* Frees the workspaces cached by falcon_compress / falcon_decompress and the host pipeline
 * on every device, and forgets the scratch addresses of falcon_compress_noalloc. */
int falcon_release(void);

/* ---------------------------------------------------------------------------------------
 * Batched form: many independent series (mixed lengths, dtypes and block sizes) compressed
 * or decompressed by the same launches as one series, each covering all (series, chunk) work
 * items at once (compression: analysis, offsets, emit; decompression: offsets, decode).  Each
 * series still produces / consumes
 * its own self-describing stream.  The paper processes one batch per kernel call (Alg. 1,
 * Alg. 3); this entry point is how the library serves many series at once.
 * ------------------------------------------------------------------------------------- */
typedef enum { FALCON_COMPRESS = 0, FALCON_DECOMPRESS = 1 } falcon_direction;

typedef struct {
    const void *d_in;       /* compress: n values (device); decompress: a stream (device) */
    void *d_out;            /* compress: stream buffer; decompress: value buffer (device) */
    uint64_t n;             /* compress: number of values (decompress: taken from h_header) */
    uint64_t in_bytes;      /* decompress: stream length in bytes (compress: ignored) */
    uint64_t out_capacity;  /* bytes available at d_out */
    int32_t dtype;          /* compress: FALCON_F64, FALCON_F32 or FALCON_F16 (decompress: ignored) */
    uint32_t block_size;    /* compress: values per chunk (decompress: ignored) */
    const void *h_header;   /* decompress: HOST copy of the stream's first 32 bytes; compress: NULL */
} falcon_series;

/* Device workspace (bytes) a batch plan of `count` series needs (job table + per-chunk
 * words).  Returns 0 if a series is invalid. */
size_t falcon_batch_workspace_bytes(int direction, const falcon_series *h_series, int count);

/* Validates the series, lays out the job table and per-chunk words in d_workspace (256-byte
 * aligned device memory of workspace_bytes) and uploads the table with a copy enqueued on
 * `stream`.  d_results (device, 2 * count uint64): after each launch [2i] = stream bytes
 * (compress) or values (decompress) of series i and [2i+1] = its falcon_status.
 * The plan stays valid until falcon_batch_forget(d_workspace) or a new plan on the same
 * workspace; buffers named in it must stay allocated while it is launched. */
int falcon_batch_plan(int direction, const falcon_series *h_series, int count, void *d_workspace,
                      size_t workspace_bytes, uint64_t *d_results, void *stream);

/* Enqueues one execution of the plan held by d_workspace on `stream` (workspace and result
 * reset, then the persistent kernel): no host synchronisation, capturable in a CUDA graph. */
int falcon_batch_launch(void *d_workspace, void *stream);

/* Drops the host-side record of the plan held by d_workspace. */
int falcon_batch_forget(void *d_workspace);

/* ---------------------------------------------------------------------------------------
 * Host <-> device streaming (Sec. 3.1, Alg. 1).  Values in HOST memory are cut into frames of
 * frame_values values; each frame goes H2D -> compress -> D2H on one of nstreams CUDA
 * streams.  As in the paper's event-driven scheduler, a frame's place in the output is
 * fixed in launch order as soon as its compressed size has come back (the "M-D2H"), so the
 * payload copy ("P-D2H") of frame f overlaps the upload and compression of later frames and
 * the output needs no merging pass.  Frames are taken by whichever stream is idle.  Every frame is a complete stream; the frames are
 * concatenated in h_out.  Host buffers should be page-locked (cudaHostAlloc) for the copies
 * to overlap; pageable memory works but serialises them.  The device buffers
 * (nstreams x (frame input + frame bound + workspace)) are allocated on first use, kept per
 * device for later calls (grown when a call needs more) and freed by falcon_release().
 * Calls on the same device run one at a time.
 * ------------------------------------------------------------------------------------- */

/* Compresses n values at h_in.  h_frame_bytes (host, ceil(n / frame_values) entries)
 * receives each frame's stream length; *out_bytes the total.  FALCON_ERR_CAPACITY if the
 * frames do not fit in out_capacity bytes. */
int falcon_pipeline_compress(const void *h_in, uint64_t n, int dtype, uint32_t block_size,
                             uint64_t frame_values, int nstreams, void *h_out, size_t out_capacity,
                             uint64_t *h_frame_bytes, size_t *out_bytes);

/* The three compression schedulers of Sec. 3.1 (Fig. 5), for the ablation of Sec. 5.4.1
 * (Fig. 12a); all write the same bytes:
 *   FALCON_SCHED_EVENT_DRIVEN   Alg. 1 (falcon_pipeline_compress): each frame's size comes back
 *                               first (M-D2H), frames are placed in launch order as their
 *                               sizes arrive and their payload copies (P-D2H) overlap later
 *                               frames; any idle stream takes the next frame;
 *   FALCON_SCHED_SYNC_BASED     the host waits for a frame's size before it launches the next
 *                               frame: only the payload copy overlaps the next frame's work;
 *   FALCON_SCHED_PRE_ALLOCATION every frame is copied back whole from a fixed output slot of
 *                               the worst-case size (falcon_bound of a frame) into page-locked
 *                               staging memory kept by the library, then merged into h_out in
 *                               frame order by the host. */
typedef enum {
    FALCON_SCHED_EVENT_DRIVEN = 0,
    FALCON_SCHED_SYNC_BASED = 1,
    FALCON_SCHED_PRE_ALLOCATION = 2
} falcon_scheduler;

/* falcon_pipeline_compress with a chosen scheduler (same arguments and results;
 * FALCON_ERR_INVALID for an unknown scheduler). */
int falcon_pipeline_compress_with(const void *h_in, uint64_t n, int dtype, uint32_t block_size,
                                  uint64_t frame_values, int nstreams, int scheduler, void *h_out,
                                  size_t out_capacity, uint64_t *h_frame_bytes, size_t *out_bytes);

/* Decompresses nframes concatenated streams (lengths in h_frame_bytes) from h_in into h_out.
 * Output positions follow from the frame headers, so frames are processed fully in
 * parallel (the pre-allocation scheduler of Sec. 4).  *n_out receives the value count. */
int falcon_pipeline_decompress(const void *h_in, const uint64_t *h_frame_bytes, uint64_t nframes,
                               int nstreams, void *h_out, size_t out_capacity_bytes, uint64_t *n_out);

/* ---------------------------------------------------------------------------------------
 * Request server: continuous batching of independent compress / decompress requests whose
 * inputs are in host memory.  The paper has no server (it compresses one stream per call);
 * this is how the library serves a stream of requests of mixed size and direction.
 *
 * A server owns, for its lifetime, on one device:
 *   - a device arena of device_budget_bytes.  Every request in flight holds one block of it
 *     (its input, its output and its per-chunk workspace words).  Requests are admitted in
 *     submission order, each only when its block fits, so the server's device memory never
 *     exceeds the budget (the memory-budget admission);
 *   - a page-locked host arena of host_budget_bytes that receives the outputs;
 *   - a worker thread and CUDA streams (one per copy direction, compute_streams for kernels).
 * Each pass of the worker admits what fits (at most max_batch requests per direction) and
 * turns the admitted requests into ONE batched launch per direction (the persistent kernels
 * of the batched form above).  Uploads, the launch and the read-back of the per-request
 * results are enqueued with device-side event dependencies.  A decompression's output copy
 * is enqueued with them (its size is in the header); a compression's output is copied once
 * its stream length has come back.  Requests that arrive while a batch runs join the next
 * batch.  Input buffers should be page-locked for the uploads to overlap.
 * ------------------------------------------------------------------------------------- */
typedef struct falcon_server falcon_server;

typedef struct {
    uint64_t tag;          /* the caller's tag from falcon_server_submit */
    int32_t status;        /* falcon_status of the request */
    int32_t op;            /* FALCON_COMPRESS or FALCON_DECOMPRESS */
    const void *h_out;     /* status OK: the output in the server's page-locked host arena
                              (compress: the stream; decompress: the values), valid until
                              falcon_server_free_output(h_out) or falcon_server_destroy.
                              NULL on error. */
    uint64_t out_bytes;    /* bytes at h_out */
    uint64_t values;       /* values in the series (either direction) */
    double latency_s;      /* submit -> completion, seconds (host steady clock) */
} falcon_completion;

typedef struct {
    uint64_t submitted, completed, failed;          /* requests */
    uint64_t batches, multi_request_batches;        /* batched launches (> 1 request) */
    uint64_t max_batch, max_in_flight;              /* requests per launch / admitted at once */
    uint64_t device_capacity, device_in_use, device_peak;   /* device arena bytes */
    uint64_t host_capacity, host_in_use, host_peak;         /* host arena bytes */
} falcon_server_stats;

/* Creates a server on CUDA device `device`: allocates both arenas (cudaMalloc and
 * cudaHostAlloc of the budgets) and starts the worker.  compute_streams >= 1;
 * 1 <= max_batch <= 65536.  A batch also closes once its inputs reach max_batch_bytes (0: no
 * byte limit; a larger single request still forms a batch), so that the uploads of one batch
 * overlap the kernels and downloads of the previous ones.  *out receives the handle. */
int falcon_server_create(int device, size_t device_budget_bytes, size_t host_budget_bytes,
                         int compute_streams, int max_batch, size_t max_batch_bytes, falcon_server **out);

/* Queues one request; thread-safe.
 *   op = FALCON_COMPRESS:   h_in = count values of dtype, chunks of block_size values;
 *   op = FALCON_DECOMPRESS: h_in = a stream of count bytes (dtype and block_size ignored).
 * h_in must stay valid and unchanged until the request's completion has been polled.
 * Returns FALCON_OK (exactly one completion with `tag` follows) or, with nothing queued:
 * FALCON_ERR_INVALID (arguments, or the server is shutting down), FALCON_ERR_CORRUPT (the
 * stream header is malformed), FALCON_ERR_CAPACITY (the
 * request's device block or output can never fit the arenas), FALCON_ERR_CUDA (a CUDA call
 * of the server failed earlier; the server accepts no more work). */
int falcon_server_submit(falcon_server *server, int op, const void *h_in, uint64_t count,
                         int dtype, uint32_t block_size, uint64_t tag);

/* Moves up to max_completions finished requests into out[] (any order) and their number into
 * *count, waiting up to timeout_us microseconds for the first one.  Thread-safe.  A request
 * whose kernel found an error (e.g. a corrupt chunk-size array) completes with that status;
 * requests still queued when the server is destroyed complete with FALCON_ERR_CAPACITY if
 * the host arena never had room for them. */
int falcon_server_poll(falcon_server *server, falcon_completion *out, int max_completions,
                       int timeout_us, int *count);

/* Returns an output (completion.h_out) to the host arena.  Outputs that are never returned
 * keep their space, and admission waits for host-arena room. */
int falcon_server_free_output(falcon_server *server, const void *h_out);

/* Counters and arena occupancy (a snapshot). */
int falcon_server_get_stats(falcon_server *server, falcon_server_stats *stats);

/* Stops accepting requests, finishes every admitted and queued request, stops the worker
 * and frees the arenas, streams and the handle.  Outputs not yet freed become invalid;
 * completions not yet polled are dropped. */
int falcon_server_destroy(falcon_server *server);

/* Persistent-grid size: at most ctas_per_sm resident CTAs per SM for each direction
 * (0 = as many as fit).  Does not change any output byte; used by the autotuner. */
int falcon_set_launch_config(int compress_ctas_per_sm, int decompress_ctas_per_sm);

/* Threads per CTA of the persistent kernels, in warps (each warp works on its own chunks):
 * 1..16 for compression, 1..12 for decompression (default 4 and 4).  Does not change any
 * output byte; used by the autotuner.  FALCON_ERR_INVALID outside those ranges. */
int falcon_set_cta_warps(int compress_warps, int decompress_warps);

#ifdef __cplusplus
}
#endif

#endif /* FALCON_H_ */
