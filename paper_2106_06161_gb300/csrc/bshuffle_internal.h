// Internal declarations shared by the C-ABI translation unit and the kernel
// translation units of libbshuffle.  Not part of the public interface.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bsh {

constexpr uint32_t kMaxRounds = 64;

// Device-resident header of a workspace.  One launch at a time uses it
// (stream order).  The last CTA of every launch resets `ticket` and `done`
// and advances `tag`, so no per-call memset is needed and a launch replayed
// from a CUDA graph sees a clean header.
struct WsHeader {
    uint32_t ticket;      // next tile ticket of the running launch
    uint32_t done;        // CTAs of the running launch that have finished
    uint32_t tag;         // tile-status tag of the running launch, 1 .. 2^31-1
    int32_t error;        // first device-side error code, 0 = none
    uint64_t error_info;  // detail of that error (tile index or slot)
    uint32_t batch_ticket;  // ticket of the persistent batched kernel
    uint32_t batch_done;    // finished CTAs of the persistent batched kernel
    // Built with BSHUFFLE_LOOKBACK_CLOCKS=1 only: SM clock cycles that tiles
    // waited on the look-back, and cycles the CTAs ran (plain and pipelined
    // single passes); 0 otherwise.
    unsigned long long lookback_cycles;
    unsigned long long cta_cycles;
};

// Shape of one shuffle: n kept slots out of a 2^k domain whose indices are
// split into a left half of L = floor(k/2) bits and a right half of
// R = ceil(k/2) bits (Sec. 3.2).
struct Geometry {
    uint32_t n;        // number of kept slots, n <= 2^32 - 1
    uint32_t k;        // domain exponent, 4 <= k <= 32
    uint32_t L, R;     // half widths
    uint32_t lmask;    // 2^L - 1
    uint32_t rmask;    // 2^R - 1
    uint64_t domain;   // 2^k
    uint32_t odd_mul;  // 2^(31 - L): multiplying by it moves bit L to bit 31
    uint32_t lift_mul; // 2^L: multiplying by it moves bit 0 to bit L
};

// Everything one fused tile launch needs, passed by value (param space).
struct TileArgs {
    const void *in;
    void *out;
    Geometry g;
    uint32_t rounds;
    uint32_t num_tiles;
    uint32_t elem_bytes;        // element width for the row kernels
    uint32_t range_first;       // range launches: first domain index of the range
    uint64_t range_end;         // range launches: one past the last domain index
    uint64_t range_cap;         // range launches: elements the output holds
    int64_t skip_publish_tile;  // test hook, -1 = off
    uint64_t timeout_ns;        // look-back wait limit
    WsHeader *ws;
    uint64_t *status;           // one word per tile
    uint32_t lcg_a, lcg_c;      // LCG bijection (odd a), both reduced mod 2^k
    uint32_t keys[kMaxRounds];
};

// What a fused launch writes.
enum class Mode : int {
    Gather = 0,   // out[j] = in[f(i_j)]            (bshuffle_permute)
    Scatter = 1,  // out[f(i_j)] = in[j]            (bshuffle_inverse)
    Index32 = 2,  // out[j] = (uint32) f(i_j)       (bshuffle_indices)
    Index64 = 3,  // out[j] = (uint64) f(i_j)
};

// Shape of a persistent pipelined kernel: compute warps, domain indices per
// compute thread, resident CTAs per SM its register budget targets, and
// whether the default round count runs fully unrolled (1) or in a loop (0).
struct PipeConfig {
    int warps;
    int items;
    int ctas_per_sm;
    int unroll;
};

// Configurations of the element kernel: CTA size, items per thread, and
// rounds unrolled at compile time (0 = read at run time).  Configuration 0
// is the default and is instantiated for every mode and width; the others
// serve bshuffle_permute with 4, 8 or 16-byte elements.
struct ElemConfig {
    int block;
    int items;
    int rounds;
};
constexpr int kNumElemConfigs = 7;
extern const ElemConfig kElemConfigs[kNumElemConfigs];

// The configuration selected for a width (0 for untunable widths), the one a
// call with this mode and round count uses, and selection (-1 if invalid).
int selected_elem_config(uint32_t elem_bytes);
int elem_config_for(uint32_t elem_bytes, Mode mode, uint32_t rounds);
int select_elem_config(uint32_t elem_bytes, int config);

// Domain indices per tile of an element-kernel configuration and of the
// row kernels.
uint32_t elem_tile_size(int config);
uint32_t rows_tile_size(uint32_t row_bytes);

// Enqueue one fused launch of num_tiles CTAs in configuration `config`.
cudaError_t launch_elem(const TileArgs &a, Mode mode, uint32_t elem_bytes, int config, cudaStream_t stream);
cudaError_t launch_gather_tuned(const TileArgs &a, uint32_t elem_bytes, int config, cudaStream_t stream);
// The fused gather with the LCG bijection (default configuration).
cudaError_t launch_gather_lcg(const TileArgs &a, uint32_t elem_bytes, cudaStream_t stream);
// Algorithm 1 restricted to the domain range [range_first, range_end): the
// gather of the range's kept indices into out[0 .. count) (num_tiles tiles of
// elem_tile_size(0) indices from range_first), and the count alone (added to
// *count, which the caller zeroes).  elem_bytes 1, 2, 4, 8 or 16.
cudaError_t launch_permute_range(const TileArgs &a, uint32_t elem_bytes, cudaStream_t stream);
cudaError_t launch_count_range(const Geometry &g, const uint32_t *keys, uint32_t rounds, uint64_t first,
                               uint64_t end, unsigned long long *count, cudaStream_t stream);
cudaError_t launch_rows(const TileArgs &a, Mode mode, cudaStream_t stream);
// Power-of-two lengths (g.n == g.domain >= 16): Algorithm 1 without its scan,
// which is the identity when nothing is dropped.  Every mode; elem_bytes 1,
// 2, 4, 8, 16 or rows of a multiple of 16 bytes.
cudaError_t launch_direct(const TileArgs &a, Mode mode, uint32_t elem_bytes, cudaStream_t stream);
// The gather of the domain range [range_first, range_end) of a power-of-two
// length (n <= 2^31) into out[0 .. range_end - range_first), bounded by
// range_cap; no workspace, no scan.  elem_bytes 1, 2, 4, 8 or 16.
cudaError_t launch_direct_range(const TileArgs &a, uint32_t elem_bytes, cudaStream_t stream);
// Writes `value` into *count on `stream` (the count of a range of a
// power-of-two length: its length).
cudaError_t launch_store_count(unsigned long long *count, uint64_t value, cudaStream_t stream);

// ------------------------------------------------------------------ batched

// Device-side descriptor, layout identical to the public bshuffle_desc.
struct BatchDesc {
    const void *in;
    void *out;
    uint64_t n;
    uint64_t seed;
};

// Per-instance plan written by the planning kernel.
struct BatchPlan {
    uint64_t first_tile;  // global index of the instance's first tile
    uint32_t k;           // domain exponent (0 for an empty instance)
    uint32_t tiles;       // tiles of the instance
};

struct BatchArgs {
    const BatchDesc *descs;
    BatchPlan *plan;        // count entries
    uint64_t *tile_prefix;  // count + 1 entries: exclusive scan of tile counts, then the total
    uint32_t count;
    uint32_t rounds;
    uint32_t elem_bytes;
    uint32_t grid;          // CTAs of the persistent kernel
    uint32_t tile;          // domain indices per tile of the persistent kernel's shape
    uint32_t pad0;
    uint64_t timeout_ns;
    int64_t skip_publish_tile;
    WsHeader *ws;
    uint64_t *status;       // look-back ring of batch_ring_words() words
    uint64_t *total_tiles;  // written by the planning kernel
};

// Shapes of the pipelined persistent kernel (4-, 8- and 16-byte elements):
// compute warps, items per compute thread, resident CTAs per SM targeted,
// default rounds unrolled; the shape selected per width.
constexpr int kNumBatchConfigs = 6;
extern const PipeConfig kBatchConfigs[kNumBatchConfigs];
int select_batch_config(uint32_t elem_bytes, int config);
int selected_batch_config(uint32_t elem_bytes);
uint64_t batch_ring_words();
// Enqueue the planning kernel and the persistent kernel (elem_bytes 1..16).
cudaError_t launch_batched(const BatchArgs &a, cudaStream_t stream);

// ------------------------------------------------------------------ staged path

// The staged shuffle: same output as the fused single pass, two streaming
// passes (see kernels_staged.cu).  For n == 2^k a bucket is a window of
// output slots; for other n (the ranked form) a bucket is a window of domain
// indices, and the second pass ranks its kept indices with a bitmap.
struct StagedArgs {
    const void *in;
    void *out;
    Geometry g;             // g.n <= g.domain
    uint32_t rounds;
    uint32_t dst_shift;     // log2 of a bucket's span (output slots, or domain indices when ranked)
    uint32_t num_dst;       // buckets, <= 4096
    uint32_t sub_shift;     // ranked: log2 of the domain indices one pass-2 CTA ranks (<= dst_shift)
    void *dval;             // values, bucket-major, 2^dst_shift entries reserved per bucket
    uint32_t *dpos;         // offsets within the bucket's span
    uint32_t *dst_cursor;   // num_dst, zero at launch
    uint32_t *bucket_base;  // ranked: num_dst first slots, written by pass 2a
    WsHeader *ws;           // error word
    uint32_t keys[kMaxRounds];
};

uint32_t staged_tile_size();
// log2 of the destination bucket (output window) in elements for a staged
// shuffle of n = 2^k elements of elem_bytes.
uint32_t staged_window_shift(uint64_t n, uint32_t elem_bytes);
// The ranked form (n < 2^k): log2 of a bucket's span of domain indices and of
// the span one pass-2 CTA ranks, for n elements of elem_bytes on a 2^k domain.
void staged_rank_shifts(uint64_t n, uint32_t k, uint32_t elem_bytes, uint32_t *bucket_shift, uint32_t *sub_shift);
// Enqueue the two passes (elem_bytes 4, 8 or 16) of the shuffle, or of the
// inverse shuffle when `inverse`; the caller zeroes the cursors first.
// marks, when not null, are 3 events recorded before P1, between the passes
// and after P2.
cudaError_t launch_staged(const StagedArgs &a, uint32_t elem_bytes, bool inverse, cudaStream_t stream,
                          cudaEvent_t *marks = nullptr);

// ------------------------------------------------------------------ fusion ablation

// Algorithm 1 with less fusion (Sec. 6): Bijective0 (variant 0: transform,
// compaction and gather as separate kernels) and Bijective1 (variant 1: fused
// with a two-pass scan).  Same output as bshuffle_permute.
struct AblationArgs {
    const void *in;
    void *out;
    Geometry g;
    uint32_t rounds;
    uint32_t num_tiles;       // tiles of ablation_tile_size() domain indices
    uint32_t *w;              // variant 0: the 2^k images
    uint32_t *j;              // variant 0: the n kept images in order
    uint32_t *tile_count;     // variant 1: kept per tile
    uint32_t *tile_prefix;    // variant 1: exclusive scan of tile_count
    uint64_t timeout_ns;
    WsHeader *ws;
    uint64_t *status;         // variant 0's compaction look-back
    uint32_t keys[kMaxRounds];
};

uint32_t ablation_tile_size();
cudaError_t launch_ablation(const AblationArgs &a, uint32_t elem_bytes, int variant, cudaStream_t stream);

// ------------------------------------------------------------------ statistics (Sec. 5)

uint32_t kendall_max_n();
cudaError_t launch_kendall_pairs(const uint32_t *perms, uint32_t n, uint64_t pairs, uint64_t *out,
                                 cudaStream_t stream);
cudaError_t launch_invert_rows(const uint32_t *idx, uint32_t n, uint64_t rows, uint32_t *sigma, cudaStream_t stream);

// ------------------------------------------------------------------ Monte Carlo

// Fused permutation statistic: T[b] = mean(y[:n1]) - mean(y[n1:]) of x
// shuffled with seed base_seed + b, for b < count.
struct McArgs {
    const float *x;
    double *T;
    Geometry g;  // g.n = length of x
    uint32_t n1;
    uint32_t count;
    uint32_t rounds;
    uint32_t pad0;
    uint64_t base_seed;
};

cudaError_t launch_mc(const McArgs &a, cudaStream_t stream);

// Pipelined single pass: which calls it serves, its shapes (compute warps,
// items per compute thread, resident CTAs per SM targeted, default rounds
// unrolled), the shape selected per width (gathers of 4, 8 and 16 bytes; 0
// for every other call), its tile size, and launch.
constexpr int kNumPipeConfigs = 6;
extern const PipeConfig kPipeConfigs[kNumPipeConfigs];
int pipe_config_for(uint32_t elem_bytes, Mode mode);
int select_pipe_config(uint32_t elem_bytes, int config);
int selected_pipe_config(uint32_t elem_bytes);
bool pipe_supports(Mode mode, uint32_t elem_bytes);
uint32_t pipe_tile_size(uint32_t elem_bytes, int config);
cudaError_t launch_pipe(const TileArgs &a, Mode mode, uint32_t elem_bytes, int config, cudaStream_t stream);
cudaError_t launch_pipe_tuned(const TileArgs &a, uint32_t elem_bytes, int config, cudaStream_t stream);

struct ShapleyArgs {
    const uint32_t *w;  // player weights
    uint64_t *counts;   // pivot counts per player, zeroed by the caller
    Geometry g;         // g.n = number of players
    uint64_t quota;
    uint64_t seed0;
    uint64_t samples;
    uint32_t rounds;
    uint32_t pad0;
};

cudaError_t launch_shapley_voting(const ShapleyArgs &a, cudaStream_t stream);

// Measurement kernel: out[i] = in[h(i)], n = 2^k, elem_bytes 4, 8 or 16.
cudaError_t launch_random_gather(const void *in, void *out, uint32_t k, uint32_t elem_bytes, cudaStream_t stream);
cudaError_t launch_window_scatter(const void *in, void *out, uint32_t k, uint32_t m, uint32_t elem_bytes,
                                  cudaStream_t s);

}  // namespace bsh
