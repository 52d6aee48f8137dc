// Host/device shared declarations of libfalcon (not part of the public ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace falcon {

// Warps per CTA of the persistent kernels: a launch parameter (falcon_set_cta_warps) that
// changes no output byte; every warp works on its own chunks.  The launch bounds keep the
// register budget of the default shape (4 warps, 4 CTAs per SM for compression; 3 CTAs per SM
// of 4 warps for decompression) at every allowed shape.
constexpr int kWarpsPerCta = 4;                 // default
constexpr int kThreads = 32 * kWarpsPerCta;
constexpr int kMaxCompressWarps = 16;           // 512 threads: 128 registers per thread
constexpr int kMaxDecompressWarps = 12;         // 384 threads: 170 registers per thread
constexpr uint32_t kMaxBlock = 1025;

// Status codes (identical numbering to falcon_status in include/falcon.h).
enum : uint32_t { kOk = 0, kErrInvalid = 1, kErrCapacity = 2, kErrCorrupt = 3, kErrCuda = 4,
                  kErrTimeout = 5, kErrUnsupported = 6 };

// One series to compress or decompress.
//   compress:   in = values (n * S bytes), out = stream (out_cap bytes)
//   decompress: in = stream (in_bytes),    out = values (out_cap bytes)
struct Job {
    const uint8_t *in;
    uint8_t *out;
    uint64_t in_bytes;
    uint64_t out_cap;
    uint64_t n;
    uint64_t nchunks;
    uint64_t chunk_begin;          // first global work ticket of this job
    unsigned long long *flags;     // the job's workspace words (workspace_words(nchunks))
    unsigned long long *result;    // [0] stream bytes (compress) / values (decompress), [1] status
    uint32_t block;
    uint32_t dtype;                // 0 = FP64, 1 = FP32
    uint32_t variant;              // compression: kVariant* (decompression: unused)
};

// Codec variants: Falcon, and the three ablations of Sec. 5.4.2 (every row sparse, every
// row dense, Elf's trial-and-error decimal place).  All write the same record layout.
enum : uint32_t { kVariantFalcon = 0, kVariantSparse = 1, kVariantDense = 2, kVariantElf = 3 };

// Per-launch control block at the start of the workspace (zeroed before each set of launches):
// the chunk tickets of the persistent kernels.  A warp takes its next chunk with one atomic
// add on its kernel's counter (analysis, emit, decode), so warps that met cheaper chunks take
// more of them and a launch ends with its average warp, not its unluckiest one.
// agg[] holds the aggregate launch's running values (analytics on compressed data): the NaN
// count, the largest complement of a min key, the largest max key (zero: none yet).
enum { kTicketAnalyse = 0, kTicketEmit = 1, kTicketDecode = 2 };
struct Control {
    unsigned long long ticket[4];
    unsigned long long agg[4];
};
static_assert(sizeof(Control) == 64, "control block is 64 bytes");

constexpr size_t kControlBytes = 256;   // control block region (keeps flags 256-aligned)

// Workspace words of a job: compression keeps two per chunk (the analysis results and the
// dense-row mask), then one per 64-chunk tile and one per 4096-chunk group (the sums of their
// record sizes, which the analysis adds up); decompression keeps the record offset of each tile
// in the first words.
// value kinds of the stream format: 0 FP64, 1 FP32, 2 FP16 (binary16)
inline bool dtype_valid(int dtype) { return dtype >= 0 && dtype <= 2; }
inline size_t dtype_bytes(int dtype) { return dtype == 0 ? 8 : (dtype == 1 ? 4 : 2); }

constexpr uint64_t kTile = 64;
constexpr uint64_t kGroup = 4096;
__host__ __device__ constexpr uint64_t tile_count(uint64_t nchunks) { return (nchunks + kTile - 1) / kTile; }
__host__ __device__ constexpr uint64_t group_count(uint64_t nchunks) { return (nchunks + kGroup - 1) / kGroup; }
__host__ __device__ constexpr uint64_t workspace_words(uint64_t nchunks) {
    return 2 * nchunks + tile_count(nchunks) + group_count(nchunks);
}

cudaError_t launch_compress(const Job *d_jobs, int njobs, const Job &single,
                            uint64_t total_chunks, Control *ctl, cudaStream_t stream);
cudaError_t launch_decompress(const Job *d_jobs, int njobs, const Job &single,
                              uint64_t total_chunks, Control *ctl, cudaStream_t stream);
// analytics on compressed data: the decode without the stores, then the aggregate into
// d_stats (falcon_stats); the chunk sums go into job.flags after the tile offsets
cudaError_t launch_aggregate(const Job &single, Control *ctl, void *d_stats, cudaStream_t stream);

// Status of the arguments of a compression call (dtype, block size, pointers, alignment,
// room for the header and size array), checked before anything is enqueued.
int compress_args(const void *d_in, uint64_t n, int dtype, uint32_t block, void *d_out, size_t out_capacity);

// Resident CTAs per SM used by the persistent grids (0 = occupancy limit); [0] compress,
// [1] decompress.  Set through falcon_set_launch_config.
extern int g_ctas_per_sm[2];

// Warps per CTA used by the persistent grids; [0] compress, [1] decompress.
extern int g_cta_warps[2];

// Persistent grid of a kernel with `warps` warps per CTA and smem_bytes dynamic shared memory:
// as many CTAs as fit (at most lim per SM when lim > 0), fewer when there is less work.
int persistent_grid_size(const void *kernel, int warps, int smem_bytes, int lim, uint64_t total_chunks);

// Grid size used for a launch over total_chunks work items (persistent, occupancy-bound).
int compress_grid(uint64_t total_chunks);
int decompress_grid(uint64_t total_chunks);

}  // namespace falcon
