/*
 * bshuffle.h -- C ABI of the GB300 bijective-shuffle library (libbshuffle.so).
 *
 * The method is the "bijective shuffle" of Mitchell, Stokes, Frank and Holmes,
 * "Bandwidth-Optimal Random Shuffling for GPUs" (arXiv 2106.06161):
 *   - a keyed pseudo-random bijection f on the power-of-two domain [0, 2^k)
 *     (VariablePhilox, Sec. 3.2, Listing 1), and
 *   - Algorithm 1 (Sec. 4): evaluate b = f(i) for every i in [0, 2^k), keep the
 *     images b < n, place the j-th kept image at output slot j (exclusive scan
 *     of the keep flags) and gather Y[j] = X[b].
 * Proposition 1 (Sec. 4) shows that deleting the images >= n from a uniform
 * permutation of [0, 2^k) leaves a uniform permutation of [0, n).
 *
 * Every step runs on the GPU.  The paper's design is one fused kernel per
 * call: the bijection in registers, the compaction as an in-tile scan chained
 * across tiles by decoupled look-back (single pass, Sec. 4 last paragraph and
 * the "Bijective2" variant of Sec. 6), the gather of each kept element once,
 * and a coalesced store into its compacted slot.  By default the library
 * picks among variants with the same output (see bshuffle_set_strategy):
 * inputs much larger than L2 run a staged variant whose HBM accesses are all
 * sequential; other power-of-two lengths run one launch without the scan
 * (with nothing dropped, slot j holds X[f(j)]); other lengths run the single
 * pass, pipelined on large domains (a dedicated warp per CTA does the
 * look-back while the other warps evaluate the next tile).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Domain.     k = max(ceil(log2 n), 4).  Sec. 4 pads to "the nearest power of
 *             two"; the floor of 2^4 is a reading: with k <= 3 the left half
 *             of the cipher has one bit, the cipher is affine over GF(2) and
 *             reaches at most 2^k of the n! permutations.
 * Rounds.     0 <= rounds <= BSHUFFLE_MAX_ROUNDS.  Sec. 5 recommends 24
 *             (BSHUFFLE_DEFAULT_ROUNDS); 0 rounds is the identity bijection.
 * Keys.       key[r] = low 32 bits of the r-th output of SplitMix64 seeded with
 *             `seed` (Steele, Lea, Flood 2014).  The paper leaves the key
 *             schedule open (one key per round in Listing 1; Sec. 7).
 * Sizes.      0 <= n <= BSHUFFLE_MAX_N.  n = 0 is a successful no-op.
 * Elements.   elem_bytes is 1, 2, 4, 8, or a positive multiple of 16 (rows of
 *             a matrix, moved whole).  Elements are raw bytes: the library
 *             never looks at their values, so every dtype is bit-exact.
 * Memory.     All data pointers are DEVICE pointers owned by the caller.  `in`
 *             and `out` must not overlap (the shuffle is not in place, Sec. 7)
 *             and must be aligned to min(elem_bytes, 16) bytes.
 * Streams.    `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *             default stream).  Calls are asynchronous with respect to the
 *             host and ordered on `stream`.
 * Workspace.  The library owns a small per-(device, stream) workspace: a
 *             tile-status word per tile (8 bytes per 2^11 domain indices), a
 *             tile ticket, a completion counter and an error word.  It is
 *             allocated with cudaMalloc on the first call that needs it (make
 *             that first call before capturing the stream into a CUDA graph)
 *             and reused; bshuffle_release_workspaces() frees it.  Calls
 *             that share a stream share its workspace and must not run
 *             concurrently with each other, which stream order guarantees.
 * Errors.     Every function returns BSHUFFLE_OK (0) or a negative code.
 *             Argument errors are detected on the host before any launch and
 *             leave the output untouched.  Device-side errors (a look-back
 *             wait that ran past its time limit, an out-of-range slot) are
 *             recorded in the workspace's error word and returned by
 *             bshuffle_get_error(); the kernels never trap.
 * No fallback. There is no CPU path.  Without a CUDA device every compute
 *             call returns BSHUFFLE_ERR_CUDA.
 */
#ifndef BSHUFFLE_H
#define BSHUFFLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BSHUFFLE_OK 0
#define BSHUFFLE_ERR_NULL (-1)              /* a required pointer is NULL */
#define BSHUFFLE_ERR_ELEM (-2)              /* unsupported elem_bytes / idx_bytes */
#define BSHUFFLE_ERR_ROUNDS (-3)            /* rounds > BSHUFFLE_MAX_ROUNDS */
#define BSHUFFLE_ERR_TOO_LARGE (-4)         /* n > BSHUFFLE_MAX_N */
#define BSHUFFLE_ERR_ALIAS (-5)             /* in and out overlap */
#define BSHUFFLE_ERR_ALIGN (-6)             /* pointer not aligned to min(elem_bytes, 16) */
#define BSHUFFLE_ERR_CUDA (-7)              /* a CUDA runtime call failed */
#define BSHUFFLE_ERR_LOOKBACK_TIMEOUT (-8)  /* device: a look-back wait ran out of time */
#define BSHUFFLE_ERR_DEVICE_BOUNDS (-9)     /* device: an output slot fell outside [0, n) */
#define BSHUFFLE_ERR_INVALID (-10)          /* other invalid argument (e.g. batch count) */

#define BSHUFFLE_DEFAULT_ROUNDS 24u
#define BSHUFFLE_MAX_ROUNDS 64u
/* Largest supported length: slots and domain indices are 32-bit (k <= 32). */
#define BSHUFFLE_MAX_N 4294967295ull

/* One instance of a batched shuffle (device memory, see bshuffle_batched). */
typedef struct bshuffle_desc {
    const void *in;   /* device pointer to n elements */
    void *out;        /* device pointer to n elements, disjoint from every in/out */
    uint64_t n;       /* instance length, 0 <= n <= BSHUFFLE_MAX_N */
    uint64_t seed;    /* key seed of this instance */
} bshuffle_desc;

/*
 * Y[j] = X[f(i_j)] for j in [0, n), where i_j is the j-th domain index, in
 * increasing order, whose image f(i_j) is below n (Algorithm 1, Sec. 4; f is
 * VariablePhilox of Sec. 3.2 with the keys of `seed`).
 *   in, out     device buffers of n * elem_bytes bytes each (caller-owned)
 *   n           number of elements
 *   elem_bytes  1, 2, 4, 8 or a multiple of 16
 *   seed        key seed; rounds: cipher rounds (24 recommended)
 *   stream      cudaStream_t as void*
 * Returns BSHUFFLE_OK once the kernels are enqueued.
 */
int bshuffle_permute(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                     uint32_t rounds, void *stream);

/*
 * out_idx[j] = f(i_j): the source index of each output slot of
 * bshuffle_permute with the same (n, seed, rounds), i.e. bshuffle_permute of
 * the iota input 0, 1, ..., n-1 (Algorithm 1, Sec. 4).
 *   out_idx     device buffer of n * idx_bytes bytes
 *   idx_bytes   4 (uint32 indices) or 8 (uint64 indices)
 */
int bshuffle_indices(void *out_idx, uint32_t idx_bytes, uint64_t n, uint64_t seed, uint32_t rounds,
                     void *stream);

/*
 * The inverse shuffle, a scatter through the same bijection:
 * out[f(i_j)] = in[j], so bshuffle_inverse(bshuffle_permute(x)) == x for equal
 * (n, seed, rounds).  Arguments as for bshuffle_permute.  (The paper notes
 * that a scatter is the inverse of a gather, Sec. 2.2.)
 */
int bshuffle_inverse(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                     uint32_t rounds, void *stream);

/*
 * `count` independent shuffles in one launch.  Instance t reads d_descs[t]
 * (DEVICE memory) and produces exactly bshuffle_permute(in, out, n,
 * elem_bytes, seed, rounds) for its own (in, out, n, seed).  All instances
 * share elem_bytes and rounds; no two instances' buffers may overlap.
 *   d_descs     device array of `count` bshuffle_desc (caller-owned; read by
 *               the kernels, so it must stay valid until the stream reaches
 *               the end of this call)
 *   count       1 <= count <= 2^24 (0 is a no-op)
 * The library keeps per-instance tile tables in the stream's workspace.  The
 * call enqueues a small planning kernel and one persistent shuffle kernel.
 */
int bshuffle_batched(const bshuffle_desc *d_descs, uint32_t count, uint32_t elem_bytes, uint32_t rounds,
                     void *stream);

/*
 * One shuffle split by domain range, for running its parts on several
 * devices (or one after another).  Algorithm 1 (Sec. 4) has one dependency
 * between its indices, the exclusive scan of the keep flags; split the domain
 * [0, 2^k) into consecutive ranges [first, end), and the kept indices of a
 * range fill a contiguous run of output slots that starts at the number of
 * kept indices in the ranges before it.  So:
 *   1. each part calls bshuffle_count_range for its range (or for every
 *      range: the count reads no data, so parts can also recompute the
 *      counts of their predecessors instead of exchanging them);
 *   2. the counts are scanned in range order (an all-gather of one integer
 *      per part, then an exclusive sum): part r's first slot is offset_r;
 *   3. each part calls bshuffle_permute_range with out pointing at slot
 *      offset_r of the whole output (or at a buffer of count_r elements it
 *      owns), reading the whole input (replicated, or reachable).
 * The parts together write exactly bshuffle_permute(in, out, n, ...).
 *
 * bshuffle_count_range: *d_count (one uint64 in DEVICE memory, 8-byte
 *   aligned, caller-owned) = the number of i in [first, end) with f(i) < n,
 *   on the domain of n (end is clipped to 2^k).  The count is written
 *   asynchronously on `stream` (it is zeroed first, then the GPU adds to it).
 *   For n = 2^k (k >= 4) nothing is dropped and the count is end - first,
 *   stored without evaluating the cipher.
 *   BSHUFFLE_ERR_INVALID if first > end.  No workspace.
 * bshuffle_permute_range: out[t] = in[f(i_t)] for the t-th kept domain index
 *   i_t in [first, end), in increasing order (t < the count above).  in holds
 *   all n elements; out holds out_capacity elements (the range's count, from
 *   bshuffle_count_range; 0 makes the call a no-op) and must not overlap in.
 *   A slot at or past out_capacity is not written and records
 *   BSHUFFLE_ERR_DEVICE_BOUNDS.  elem_bytes 1, 2, 4, 8 or 16; first < 2^32.
 *   Uses the stream's workspace (one status word per 2,048 indices of the
 *   range) and the fused single pass (pipelined for 4-, 8- and 16-byte
 *   elements, as in bshuffle_permute); for n = 2^k (16 <= n <= 2^31) the scan
 *   over the range is the identity, so the scan-free gather runs instead
 *   (out[t] = in[f(first + t)], the workspace's error word only).  Errors as
 *   for bshuffle_permute.
 */
int bshuffle_count_range(uint64_t n, uint64_t seed, uint32_t rounds, uint64_t first, uint64_t end,
                         uint64_t *d_count, void *stream);
int bshuffle_permute_range(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                           uint32_t rounds, uint64_t first, uint64_t end, uint64_t out_capacity, void *stream);

/*
 * The shuffle with the linear congruential bijection of Sec. 3.1 in place of
 * VariablePhilox: Y[j] = X[f(i_j)] as in bshuffle_permute, with
 * f(i) = (a i + c) mod 2^k, a odd (so f is a bijection of [0, 2^k)).  The
 * paper gives no seed-to-(a, c) mapping; here a is the first SplitMix64
 * output of `seed` with its low bit set and c the second, both reduced
 * mod 2^k (bshuffle_lcg_params, a host helper).  Fast but statistically weak:
 * at most 2^(2k-1) permutations, and Sec. 5 reports it failing the
 * chi-squared test by orders of magnitude.  Single-pass kernel only;
 * elem_bytes 1, 2, 4, 8 or 16.
 */
int bshuffle_permute_lcg(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                         void *stream);
int bshuffle_lcg_params(uint64_t seed, uint64_t n, uint64_t *a, uint64_t *c);

/*
 * Measurement entry point for the fusion experiment of Sec. 6: the output of
 * bshuffle_permute, computed with less kernel fusion.
 *   variant 0  "Bijective0": three kernels - W[i] = f(i) for the whole
 *              domain, stream compaction of W (entries below n, in order,
 *              decoupled look-back), then the gather Y[j] = X[W'[j]].
 *              Scratch 4 * 2^k + 4 * n bytes.
 *   variant 1  "Bijective1": fused, with a two-pass scan: a reduce pass
 *              evaluates f and counts per tile, the tile counts are scanned,
 *              and a second pass evaluates f again, ranks and gathers.
 *   variant 2  "Bijective2": the fused single pass (as bshuffle_permute
 *              with BSHUFFLE_STRATEGY_SINGLE_PASS).
 *   variant 3  the fused single pass with its look-back taken off the
 *              compute warps (as bshuffle_permute with
 *              BSHUFFLE_STRATEGY_PIPELINED); not in the paper.
 * Scratch lives in the stream's workspace.  elem_bytes 4, 8 or 16.
 */
int bshuffle_permute_ablation(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                              uint32_t rounds, int variant, void *stream);

/*
 * Permutation Monte Carlo statistic fused with the shuffle (an application
 * named in Sec. 1; the shuffled data never leaves registers and nothing but T
 * is written).  For b in [0, count):
 *     y = bshuffle_permute(x, n, seed = base_seed + b, rounds)
 *     T[b] = mean(y[0:n1]) - mean(y[n1:n])          (FP64 sums)
 *   x       device array of n float32 values (caller-owned, read only)
 *   n1      size of the first group, 0 < n1 < n
 *   T       device array of count doubles (caller-owned)
 * Slots fill in increasing domain order, so the kernel stops a shuffle once
 * n1 elements are kept and takes the second group's sum as the total minus
 * the first's.  Summation order differs from a sequential sum, so T agrees
 * with it to FP64 rounding (relative differences near 1e-15), not bitwise.
 * Needs no workspace.  Returns BSHUFFLE_ERR_INVALID unless 0 < n1 < n.
 */
int bshuffle_mc_group_diff(const float *x, uint64_t n, uint64_t n1, uint64_t base_seed, uint32_t count,
                           uint32_t rounds, double *T, void *stream);

/*
 * Shapley values of a weighted voting game by permutation sampling (an
 * application named in Sec. 1), fused with the shuffle; the player orders
 * are never written.  Game [quota; w_0 .. w_{n-1}]: a coalition wins when
 * its total weight reaches quota.  For s in [0, samples):
 *     order = bshuffle_indices(n, seed = seed0 + s, rounds)
 *     the player order[j] whose weight takes the running total of
 *     order[0..j-1] from below quota to at least quota is pivotal:
 *     counts[order[j]] += 1
 *   weights  device array of n uint32 weights (caller-owned, read only)
 *   counts   device array of n uint64 (caller-owned), overwritten
 * counts / samples estimates each player's Shapley value.  With quota 0 or
 * above the total weight no player is pivotal and counts stays zero.  The
 * counts are exact integers: any order of the increments gives the same
 * result.  Needs no workspace.  n = 0 is a no-op.
 */
int bshuffle_shapley_voting(const uint32_t *weights, uint64_t n, uint64_t quota, uint64_t seed0, uint64_t samples,
                            uint32_t rounds, uint64_t *counts, void *stream);

/*
 * Measurement kernel, not a shuffle API: out[i] = in[h(i)] for a fixed cheap
 * bijection h of [0, n) (three rounds of multiply-by-odd-constant and
 * xor-shift on k-bit values), with no cipher, keep test or scan.  It measures
 * the random-gather bound the paper sets for every shuffle (the "Gather"
 * column of Tables 1 and 2, Sec. 2.2).  n must be a power of two in
 * [16, 2^32]; elem_bytes 4, 8 or 16; BSHUFFLE_ERR_INVALID otherwise.
 */
int bshuffle_random_gather(const void *in, void *out, uint64_t n, uint32_t elem_bytes, void *stream);

/*
 * Measurement kernel, not a shuffle API: for every i, out[w 2^m + h_m(i -
 * w 2^m)] = in[i] with window w = i >> m and h_m the bijection of
 * bshuffle_random_gather on m = window_log2 bits.  Sequential reads and
 * random writes confined to windows of 2^m elements: the access pattern of
 * the staged path's second pass, so it measures the rate at which the L2
 * takes random writes into a resident window (the bound of that pass).
 * n must be a power of two in [16, 2^32], 4 <= window_log2 <= log2 n;
 * elem_bytes 4, 8 or 16; BSHUFFLE_ERR_INVALID otherwise.
 */
int bshuffle_window_scatter(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint32_t window_log2,
                            void *stream);

/*
 * GPU helpers for the statistical tests of Sec. 5 (not part of the shuffle).
 * bshuffle_kendall_pairs: for each p < num_pairs, out[p] = n_dis(s, t) of the
 * permutations s = perms[2p], t = perms[2p + 1] (rows of n uint32 ranks),
 * n_dis = #{i < j : (s_i < s_j) != (t_i < t_j)}, the count in the Mallows
 * kernel exp(-lambda n_dis / C(n, 2)); 1 <= n <= 4096.
 * bshuffle_invert_rows: sigma[r][idx[r][j]] = j for each of `rows` rows of
 * length n: the slot order of a shuffle (slot j holds element idx[j]) turned
 * into each element's rank, the convention of Sec. 2.  Device pointers;
 * asynchronous on `stream`.
 */
int bshuffle_kendall_pairs(const uint32_t *perms, uint32_t n, uint64_t num_pairs, uint64_t *out, void *stream);
int bshuffle_invert_rows(const uint32_t *idx, uint32_t n, uint64_t rows, uint32_t *sigma, void *stream);

/*
 * Synchronises `stream`, then returns and clears the first device-side error
 * recorded by calls on that stream since the last bshuffle_get_error:
 * BSHUFFLE_OK, BSHUFFLE_ERR_LOOKBACK_TIMEOUT or BSHUFFLE_ERR_DEVICE_BOUNDS (or
 * BSHUFFLE_ERR_CUDA if synchronising failed).  A stream without a workspace
 * has no recorded errors.  It also returns and clears an error that
 * bshuffle_permute_static recorded on the current device (that entry point
 * keeps one error word per device): pass the stream of the static call, so
 * that the call has finished when the word is read.  When both hold an
 * error, the stream workspace's is returned and both are cleared.
 */
int bshuffle_get_error(void *stream);

/*
 * The cudaError_t value (as int) of the CUDA runtime call behind the latest
 * BSHUFFLE_ERR_CUDA that a bshuffle function returned on the calling thread
 * (0 if none has), e.g. cudaErrorMemoryAllocation (2) when a workspace could
 * not be allocated or cudaErrorNoDevice (100) without a GPU.  It stays set
 * until the next BSHUFFLE_ERR_CUDA on the thread.  bshuffle_cuda_error_name
 * gives the runtime's name for such a value; never NULL.
 */
int bshuffle_last_cuda_error(void);
const char *bshuffle_cuda_error_name(int error);

/* Static English text for a return code; never NULL. */
const char *bshuffle_error_string(int code);

/*
 * Host-side helpers (no GPU needed).  The domain exponent k of length n
 * (0 for n = 0) and the round keys of a seed, exactly as the kernels use
 * them.  keys must hold `rounds` entries.  Return BSHUFFLE_OK or an error.
 */
int bshuffle_domain_bits(uint64_t n, uint32_t *k);
int bshuffle_round_keys(uint64_t seed, uint32_t rounds, uint32_t *keys);

/*
 * Frees every workspace the library allocated (all devices and streams).
 * The caller must ensure no call of this library is still running.
 */
int bshuffle_release_workspaces(void);

/*
 * How bshuffle_permute, bshuffle_inverse and bshuffle_indices move data
 * (the output is identical either way):
 *   BSHUFFLE_STRATEGY_SINGLE_PASS  one fused launch: bijection, scan with
 *       decoupled look-back, one random read and one coalesced write per
 *       element (the paper's "Bijective2", Sec. 6).  No extra memory beyond
 *       the small workspace.
 *   BSHUFFLE_STRATEGY_STAGED  for n >= 4096 and 4, 8 or 16-byte elements
 *       (other calls run the single pass).  For n = 2^k nothing is dropped,
 *       so element b belongs in slot f^-1(b) (the inverse cipher of Sec. 3.2;
 *       bshuffle_inverse uses the same passes with slot f(b)).
 *       Pass 1 reads the input sequentially, inverts the cipher and buckets
 *       (value, slot) by 8 MiB output window; pass 2 scatters each window
 *       while it is resident in L2.  Random HBM accesses are rate-limited on
 *       GB300, streaming ones are not.  Workspace n * (4 + elem_bytes) bytes
 *       plus a little, allocated on first use per stream.  Other n (the
 *       ranked form, bshuffle_permute only): element b's slot is the rank of
 *       its domain index i = f^-1(b) among the kept indices (Algorithm 1's
 *       exclusive scan); pass 1 buckets (value, i) by span of domain
 *       indices, a second kernel ranks each span's kept indices with a
 *       bitmap in shared memory, and the window scatter places the values.
 *       Workspace 2^k * (4 + elem_bytes) bytes plus a little.
 *   BSHUFFLE_STRATEGY_PIPELINED  the single pass with its look-back taken
 *       off the compute warps, for gathers and scatters of 4, 8 and 16-byte
 *       elements and for indices (other calls run the plain single pass):
 *       persistent CTAs; eight compute warps evaluate the bijection of a tile
 *       and copy its kept elements into shared memory with cp.async, then
 *       store the previous tile, which a ninth warp has meanwhile ranked
 *       with the look-back.  Same memory traffic and workspace as the single
 *       pass.
 *   BSHUFFLE_STRATEGY_AUTO (default)  staged when it applies and
 *       n * elem_bytes >= 256 MiB (for n other than 2^k: with 4- or 8-byte
 *       elements only; 16-byte elements run faster on the pipelined single
 *       pass there); otherwise, for n = 2^k >= 16, one launch
 *       without the scan (nothing is dropped, so the i-th domain index is
 *       the i-th kept one: out[i] = in[f(i)], out[f(i)] = in[i] or
 *       out[i] = f(i)); otherwise the pipelined single pass where it applies
 *       and the domain has at least 2^18 indices (2^19 for the scatter of
 *       bshuffle_inverse), else the plain one (on smaller domains a launch
 *       is all latency and the plain kernel finishes first).  If the staged
 *       workspace cannot be allocated, the scan-free launch runs instead.
 * The setting is process-wide.  Returns BSHUFFLE_ERR_INVALID for other values.
 */
#define BSHUFFLE_STRATEGY_AUTO 0
#define BSHUFFLE_STRATEGY_SINGLE_PASS 1
#define BSHUFFLE_STRATEGY_STAGED 2
#define BSHUFFLE_STRATEGY_PIPELINED 3
int bshuffle_set_strategy(int strategy);
int bshuffle_get_strategy(void);

/*
 * Tuning of the single-pass kernel used by bshuffle_permute for 4, 8 and
 * 16-byte elements.  Configuration c (0 <= c < bshuffle_tuning_configs())
 * has `block` threads per CTA, `items` domain indices per thread (one tile is
 * block * items indices) and `rounds_unrolled` rounds fixed at compile time
 * (0: the round count is read at run time; a configuration with a fixed count
 * serves only calls with that many rounds, others fall back to
 * configuration 0).  Configuration 0 is the default.  The choice is
 * process-wide per element width and changes speed only: every
 * configuration computes the same output.  bshuffle_tuning_select returns
 * BSHUFFLE_ERR_INVALID for other widths or indices; bshuffle_tuning_selected
 * returns the current choice (0 for other widths).
 */
int bshuffle_tuning_configs(void);
int bshuffle_tuning_describe(int config, int *block, int *items, int *rounds_unrolled);
int bshuffle_tuning_select(uint32_t elem_bytes, int config);
int bshuffle_tuning_selected(uint32_t elem_bytes);

/*
 * Tuning of the three kernels the default strategy runs for shuffles without
 * staging: `kernel` is BSHUFFLE_KERNEL_SINGLE_PASS (the plain fused kernel:
 * small domains, and every call under BSHUFFLE_STRATEGY_SINGLE_PASS; its
 * configurations are those of bshuffle_tuning_*), BSHUFFLE_KERNEL_PIPELINED
 * (the pipelined single pass of bshuffle_permute for 4-, 8- and 16-byte
 * elements) or BSHUFFLE_KERNEL_BATCHED (the persistent kernel of
 * bshuffle_batched for 4-, 8- and 16-byte elements).  Configuration c has
 * `threads` per CTA (the pipelined shapes: compute warps plus one look-back
 * warp), `items` domain indices per compute thread, the resident CTAs per SM
 * its register budget targets (0: not set) and the rounds unrolled at compile
 * time (24: the default count runs unrolled, other counts in a loop; 0: every
 * count runs in a loop).  Configuration 0 is the default.  Every
 * configuration computes the same output; the choice is process-wide per
 * element width and changes speed only.  Select and selected return
 * BSHUFFLE_ERR_INVALID for another kernel, width or configuration.
 */
#define BSHUFFLE_KERNEL_SINGLE_PASS 0
#define BSHUFFLE_KERNEL_PIPELINED 1
#define BSHUFFLE_KERNEL_BATCHED 2
int bshuffle_kernel_configs(int kernel);
int bshuffle_kernel_describe(int kernel, int config, int *threads, int *items, int *ctas_per_sm,
                             int *rounds_unrolled);
int bshuffle_kernel_select(int kernel, uint32_t elem_bytes, int config);
int bshuffle_kernel_selected(int kernel, uint32_t elem_bytes);

/*
 * Per-pass timing (tracing aid, off by default).  While on, bshuffle_permute
 * records CUDA events around each of its kernels on the caller's stream.
 * bshuffle_last_pass_ms synchronises `stream` and writes the durations of the
 * last bshuffle_permute call on it, in ms, to ms[0 .. capacity): one value for
 * the single pass, two for the staged path (inverse cipher + destination
 * buckets, window scatter).  Returns
 * the number of passes recorded (0 if none) or a negative error.  Do not turn
 * it on while capturing a stream.
 */
int bshuffle_set_pass_timing(int on);
int bshuffle_last_pass_ms(void *stream, float *ms, int capacity);

/*
 * Time limit of one look-back wait in nanoseconds (default 2e9).  When a
 * wait runs out the kernel records BSHUFFLE_ERR_LOOKBACK_TIMEOUT, skips its
 * stores and lets later tiles finish.  Values below 1e6 are raised to 1e6.
 */
int bshuffle_set_lookback_timeout_ns(uint64_t ns);

/*
 * Test hook: the tile with this index, in every following call, does not
 * publish its tile status, so that its successors' look-back waits run out
 * and report BSHUFFLE_ERR_LOOKBACK_TIMEOUT.  Pass -1 to switch it off
 * (the default).
 */
int bshuffle_debug_skip_publish(int64_t tile);

/*
 * Measurement aid.  A library built with BSHUFFLE_LOOKBACK_CLOCKS=1 (an nvcc
 * define; the default build has it off and pays nothing) adds, per stream,
 * the SM clock cycles its single-pass kernels wait on the inter-tile
 * look-back (the plain kernel: cycles of the look-back itself, while the
 * tile's other warps wait at the barrier; the pipelined kernel: cycles the
 * compute warps wait for a tile's rank) and the cycles their CTAs run.  This
 * call synchronises `stream`, writes both sums and clears them; their ratio
 * is the share of CTA time lost to the look-back chain of Sec. 4's single
 * pass.  Returns BSHUFFLE_ERR_INVALID (and zeros) in the default build.
 */
int bshuffle_debug_lookback_cycles(void *stream, uint64_t *lookback_cycles, uint64_t *cta_cycles);

/*
 * Allocation-free variant of bshuffle_permute, for callers that cannot
 * allocate device memory when they call: a process that has reserved all of
 * the device's memory for its own pool (cudaMalloc would fail), or a
 * latency-critical loop that cannot take the device-wide synchronisation
 * that cudaMalloc/cudaFree may cause.  The paper has no counterpart; this is
 * a deployment convenience.
 *   Output.    Identical to bshuffle_permute(in, out, n, elem_bytes, seed,
 *              rounds, stream).  The caller passes in and out as usual.
 *   Scratch.   The tile-status words and launch counters live in one
 *              file-scope device array of 512 KiB + 256 B that every GPU
 *              loading the library holds until the process exits.  No call
 *              allocates or frees device memory.
 *   Limits.    elem_bytes 1, 2, 4, 8 or 16; n <= 2^27 (134,217,728);
 *              larger n returns BSHUFFLE_ERR_TOO_LARGE.
 *   Set-up.    The first call on a device looks up the array's device
 *              address with that device current and initialises its launch
 *              tag (one small synchronous copy); make that first call before
 *              any stream capture.
 *   Sharing.   Every call on a device shares the one array, which keeps the
 *              last call's contents; each call clears the counters that must
 *              start at zero.  Calls that overlap on the GPU (e.g. on two
 *              streams at once) race and corrupt each other's output:
 *              serialise them.
 *   Errors.    Argument errors as for bshuffle_permute.  A device-side
 *              error (a look-back wait that ran out of time, an out-of-range
 *              slot) is recorded in the array's own error word, which
 *              bshuffle_get_error(stream) syncs, returns and clears for the
 *              current device.  The word keeps the first error until then.
 */
int bshuffle_permute_static(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                            uint32_t rounds, void *stream);

/* Library version as major * 10000 + minor * 100 + patch. */
int bshuffle_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BSHUFFLE_H */
