// Staged shuffle of lengths much larger than L2: the same permutation as the
// fused single pass (Algorithm 1, Sec. 4), with every HBM access sequential
// and the random accesses confined to L2-resident windows.  For n = 2^k the
// inverse shuffle (out[f(j)] = in[j]) runs the same two passes with the
// forward cipher in place of the inverse one; other n take the ranked form
// (gathers only, below).
//
// On GB300 a random 8-byte access to a multi-GiB array is bound by the HBM
// random-access rate (~47 G accesses/s), far below the streaming bandwidth, so
// the single pass that the paper designs around (one random read and one
// write per element) runs at ~10 % of HBM bandwidth.  When n = 2^k no domain
// index is dropped, slot j holds X[f(j)], and equivalently element b goes to
// slot f^-1(b): the inverse cipher of Sec. 3.2 turns the gather into a
// scatter whose source side is sequential.  Two passes:
//
//   P1  per chunk of 2,048 (or 4,096) consecutive elements b: a coalesced
//       read of X[b], the inverse cipher j = f^-1(b), and a counting sort of
//       (value, j) by destination bucket (j >> dst_shift, an output window of
//       4 MiB or more) in shared memory; each bucket's run is appended with
//       one global atomic per bucket per chunk.
//   P2  per chunk of one destination bucket: out[j] = value, random within an
//       L2-resident output window whose lines leave L2 complete.
//
// Runs are appended in a nondeterministic order, but every element is placed
// by its exact slot, so the output is deterministic and identical to the
// single pass.
//
// Sizes (measured on GB300): P2 is fastest in small windows (its random
// writes stay in L2; 4 MiB beats 8 MiB by 13 %, 32 MiB costs 50 % more), while
// P1 slows down steeply past 256 buckets per 2,048-element chunk (each chunk
// zeroes, scans and atomically appends every bucket).  staged_window_shift
// takes the smallest window (at least 4 MiB) that keeps the bucket count at
// one per 8 elements of a P1 chunk, and inputs over 2 GiB of 4- or 8-byte
// elements use 4,096-element chunks (16 items per thread), which halves the
// appends per element and allows 512 buckets.
//
// Ranked form (n not a power of two, domain 2^k > n): element b still goes to
// the slot of its domain index i = f^-1(b), but that slot is the rank of i
// among the kept indices (Algorithm 1's exclusive scan), not i itself.  P1
// buckets (value, offset of i) by span of 2^s domain indices (a span holds
// at most 2^s kept indices, so 2^k entries are reserved); P2a ranks every
// span's kept indices with a bitmap in shared memory and rewrites the offsets
// as slot offsets; P2b is the window scatter above, one bucket's output range
// at a time.
#include <atomic>
#include <cstdint>

#include <cooperative_groups.h>

#include "bshuffle_device.cuh"
#include "bshuffle_internal.h"

namespace bsh {
namespace {

using dev::kFull;

constexpr int kSBlock = 256;
constexpr int kSItems = 8;
constexpr uint32_t kSTile = kSBlock * kSItems;  // entries per CTA of P2
// P1's CTA size (overridable at build time for tuning experiments): a P1 CTA
// buckets kP1Block * ITEMS consecutive elements, ITEMS = 8 or 16.
#ifndef BSHUFFLE_STAGED_P1_BLOCK
#define BSHUFFLE_STAGED_P1_BLOCK 256
#endif
constexpr int kP1Block = BSHUFFLE_STAGED_P1_BLOCK;
constexpr int kP1Warps = kP1Block / 32;
constexpr uint32_t kP1TileSmall = kP1Block * 8;
constexpr uint32_t kP1TileLarge = kP1Block * 16;
constexpr uint32_t kStagedMinChunk = kP1TileSmall > kSTile ? kP1TileSmall : kSTile;
constexpr uint32_t kMinWindowLog2 = 22;       // 4 MiB
constexpr uint64_t kLargeInputBytes = uint64_t{1} << 31;  // above this, 16 items per P1 thread

// P1 items per thread for n elements of elem_bytes.
uint32_t p1_items_for(uint64_t n, uint32_t elem_bytes)
{
    return elem_bytes <= 8 && n * elem_bytes > kLargeInputBytes ? 16u : 8u;
}

// Exclusive scan of cnt[0..m) into start[0..m) by the whole CTA (kP1Block threads).
__device__ __forceinline__ void block_exclusive_scan(const uint32_t *cnt, uint32_t *start, uint32_t m,
                                                     uint32_t *s_warp)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t per = (m + kP1Block - 1) / kP1Block;
    const uint32_t b0 = tid * per;
    const uint32_t b1 = b0 + per < m ? b0 + per : m;
    uint32_t sum = 0;
    for (uint32_t q = b0; q < b1; ++q) sum += cnt[q];
    const uint32_t incl = dev::warp_inclusive_scan(sum);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < static_cast<uint32_t>(kP1Warps) ? s_warp[lane] : 0u;
        const uint32_t wi = dev::warp_inclusive_scan(w);
        if (lane < static_cast<uint32_t>(kP1Warps)) s_warp[lane] = wi - w;
    }
    __syncthreads();
    uint32_t run = s_warp[warp] + incl - sum;
    for (uint32_t q = b0; q < b1; ++q) {
        start[q] = run;
        run += cnt[q];
    }
}

// ------------------------------------------------------------------ P1

// FORWARD: element b goes to slot f(b) (the inverse shuffle) instead of
// f^-1(b) (the shuffle).  PADDED: the ranked form for n < 2^k, where the
// bucket is a window of domain indices and the last chunk is ragged.  The
// round keys sit in kernel parameter space, so the unrolled 24 rounds read
// them as constant operands.
template <class T, bool ODD, bool FORWARD, int ITEMS, bool PADDED>
__device__ __forceinline__ void bucket_pass(const StagedArgs &a)
{
    constexpr int kP1Items = ITEMS;
    constexpr uint32_t kP1Tile = kP1Block * ITEMS;
    // dynamic shared memory: the chunk's entries (value, output slot) sorted
    // by destination bucket, then three words per destination bucket.  The
    // bucket and the entry's staged offset are recomputed from the slot at
    // write-out: 12 bytes per uint64 entry instead of 14 or 16 made this pass
    // 3-9 % faster on GB300 (it is sensitive to its shared-memory footprint).
    extern __shared__ __align__(16) unsigned char s_raw[];
    T *s_val = reinterpret_cast<T *>(s_raw);
    uint32_t *s_dst = reinterpret_cast<uint32_t *>(s_raw + kP1Tile * sizeof(T));
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(s_raw + kP1Tile * (sizeof(T) + 4));
    uint32_t *s_start = s_cnt + a.num_dst;
    uint32_t *s_gbase = s_start + a.num_dst;
    __shared__ uint32_t s_warp[kP1Warps];

    const uint32_t tid = threadIdx.x;
    const Geometry &g = a.g;
    // n = 2^k is a multiple of kP1Tile; a padded n leaves a ragged last chunk
    const uint32_t first = blockIdx.x * kP1Tile;
    const uint32_t chunk = PADDED ? min(kP1Tile, g.n - first) : kP1Tile;
    const T *in = static_cast<const T *>(a.in);
    for (uint32_t q = tid; q < a.num_dst; q += kP1Block) s_cnt[q] = 0u;

    T val[kP1Items];
    uint32_t left[kP1Items], right[kP1Items];
#pragma unroll
    for (int j = 0; j < kP1Items; ++j) {
        const uint32_t b = first + static_cast<uint32_t>(j * kP1Block) + tid;
        if (!PADDED || b < g.n) val[j] = __ldcs(in + b);
        left[j] = b >> g.R;  // beyond a padded n: never used
        right[j] = b & g.rmask;
    }
    if constexpr (FORWARD)
        dev::cipher_items<ODD, kP1Items>(left, right, a.keys, a.rounds, g);
    else
        dev::cipher_inverse_items<ODD, kP1Items>(left, right, a.keys, a.rounds, g);
    uint32_t dst[kP1Items], slot[kP1Items];
#pragma unroll
    for (int j = 0; j < kP1Items; ++j) dst[j] = (left[j] << g.R) | right[j];  // f^-1(b) (or f(b)): its slot
    __syncthreads();  // s_cnt zeroed
#pragma unroll
    for (int j = 0; j < kP1Items; ++j)
        if (!PADDED || static_cast<uint32_t>(j * kP1Block) + tid < chunk)
            slot[j] = atomicAdd(&s_cnt[dst[j] >> a.dst_shift], 1u);
    __syncthreads();
    block_exclusive_scan(s_cnt, s_start, a.num_dst, s_warp);
    for (uint32_t q = tid; q < a.num_dst; q += kP1Block) {
        const uint32_t c = s_cnt[q];
        s_gbase[q] = c != 0u ? atomicAdd(&a.dst_cursor[q], c) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kP1Items; ++j) {
        if (PADDED && static_cast<uint32_t>(j * kP1Block) + tid >= chunk) continue;
        const uint32_t p = s_start[dst[j] >> a.dst_shift] + slot[j];
        s_val[p] = val[j];
        s_dst[p] = dst[j];
    }
    __syncthreads();
    T *dval = static_cast<T *>(a.dval);
    const uint32_t bmask = static_cast<uint32_t>((uint64_t{1} << a.dst_shift) - 1u);
#pragma unroll
    for (int j = 0; j < kP1Items; ++j) {
        const uint32_t p = static_cast<uint32_t>(j * kP1Block) + tid;
        if (PADDED && p >= chunk) continue;
        const uint32_t d = s_dst[p];
        const uint32_t q = static_cast<uint32_t>(static_cast<uint64_t>(d) >> a.dst_shift);
        const uint32_t off = s_gbase[q] + (p - s_start[q]);
        if (off <= bmask) {
            const uint64_t o = (static_cast<uint64_t>(q) << a.dst_shift) + off;
            dval[o] = s_val[p];
            a.dpos[o] = d & bmask;
        } else {
            dev::record_error(a.ws, dev::kErrDeviceBounds, (static_cast<uint64_t>(q) << a.dst_shift) + off);
        }
    }
}

template <class T, bool ODD, bool FORWARD, int ITEMS>
__global__ void __launch_bounds__(kP1Block) staged_bucket_kernel(const __grid_constant__ StagedArgs a)
{
    bucket_pass<T, ODD, FORWARD, ITEMS, false>(a);
}

// The ranked form's P1, in kernels of its own so that their register
// budgets are set apart from the 2^k form's.  With 16 items per thread and
// 4- or 8-byte elements the compiler would take 92-94 registers (2 CTAs per
// SM); capped for 3 CTAs per SM, pass 1 of the n = 2^28 + 12345 uint64
// shuffle takes 2.61 ms instead of 2.85 ms on GB300 (16-byte elements spill
// under the cap and keep 2 CTAs).
template <class T, bool ODD, int ITEMS>
__global__ void __launch_bounds__(kP1Block) staged_rank_bucket_kernel(const __grid_constant__ StagedArgs a)
{
    bucket_pass<T, ODD, false, ITEMS, true>(a);
}

#ifndef BSHUFFLE_RANKED_P1_MIN_CTAS
#define BSHUFFLE_RANKED_P1_MIN_CTAS 3
#endif
template <class T, bool ODD>
__global__ void __launch_bounds__(kP1Block, BSHUFFLE_RANKED_P1_MIN_CTAS)
    staged_rank_bucket16_kernel(const __grid_constant__ StagedArgs a)
{
    bucket_pass<T, ODD, false, 16, true>(a);
}

// ------------------------------------------------------------------ P2

// P2: each thread moves kSItems entries (reads first, then the stores).
// Measured on GB300: more independent random stores in flight per SM (16 per
// thread with paired vector loads, or more than 5 resident CTAs) slows this
// pass down; the L2 takes random 8-byte writes at a bounded rate.  The launch
// reserves shared memory to keep at most kScatterCtasPerSm CTAs per SM.
constexpr int kScatterCtasPerSm = 5;
constexpr size_t kScatterSmemReserve = (228u * 1024u) / kScatterCtasPerSm - 1024u;

template <class T>
__global__ void __launch_bounds__(kSBlock) staged_scatter_kernel(const __grid_constant__ StagedArgs a)
{
    const uint32_t n = a.g.n;  // n = 2^k <= 2^31, a multiple of kSTile
    const uint32_t first = blockIdx.x * kSTile;
    const T *dval = static_cast<const T *>(a.dval);
    T *out = static_cast<T *>(a.out);
    T v[kSItems];
    uint32_t dst[kSItems];
#pragma unroll
    for (int j = 0; j < kSItems; ++j) {
        const uint32_t e = first + static_cast<uint32_t>(j * kSBlock) + threadIdx.x;
        v[j] = __ldcs(dval + e);
        dst[j] = ((e >> a.dst_shift) << a.dst_shift) + __ldcs(a.dpos + e);
    }
#pragma unroll
    for (int j = 0; j < kSItems; ++j) {
        if (dst[j] < n) out[dst[j]] = v[j];
        else dev::record_error(a.ws, dev::kErrDeviceBounds, dst[j]);
    }
}

// ------------------------------------------------------------------ P2, ranked form (n < 2^k)
//
// Bucket q holds, in arrival order, every element b whose domain index
// i = f^-1(b) lies in the span [q 2^s, (q + 1) 2^s) (s = dst_shift), with
// i's offset in that span.  These are exactly the kept indices of the span,
// so the span's first slot is the number of entries in the buckets before
// it, and an element's slot is that base plus the number of entries of the
// bucket with a smaller offset: Algorithm 1's exclusive scan of the keep
// flags, taken over the span.  The offsets are distinct, so the count is a
// rank in a bitmap of the span.
//
// P2a ranks: a CTA builds the bitmap of 2^w of the span's indices
// (w = sub_shift <= 20) in shared memory with a 16-bit prefix per bitmap word
// and a 32-bit prefix per 2,048 words (192 KiB at w = 20), then rewrites each
// of its entries' offset in place as the entry's slot offset in the bucket's
// output range, tagged with bit 31.  When the span is larger (s > w), the
// 2^(s-w) CTAs that share it form a cluster: each reads every entry of the
// bucket, keeps those of its own part (an entry already tagged belongs to
// another part), and takes the entry counts of the parts before it from
// their shared memory.  P2a also records each bucket's first slot.
// P2b scatters: the window scatter of the 2^k form, out[base + offset] =
// value, over the bucket's entries, with every resident CTA inside one or
// two buckets at a time, so that the random writes stay in L2.
constexpr int kRankBlock = 1024;
constexpr int kRankWarps = kRankBlock / 32;
constexpr uint32_t kRankMaxSubShift = 20;
constexpr uint32_t kSuperWords = 2048;  // bitmap words per 32-bit prefix (2^16 indices)
constexpr int kRankUnroll = 4;          // uint4 loads of 4 offsets each, per thread and step
constexpr uint32_t kRanked = 0x80000000u;
// The ranked form takes 16 P1 items per thread (512 buckets) where 8 would
// leave spans over 2^BSHUFFLE_RANKED_MAX_SPAN_LOG2 domain indices.
#ifndef BSHUFFLE_RANKED_MAX_SPAN_LOG2
#define BSHUFFLE_RANKED_MAX_SPAN_LOG2 20
#endif

size_t rank_smem_bytes(uint32_t sub_shift)
{
    const size_t words = sub_shift >= 5 ? size_t{1} << (sub_shift - 5) : 1;
    const size_t supers = (words + kSuperWords - 1) / kSuperWords;
    return words * 4 + ((words * 2 + 15) & ~size_t{15}) + supers * 4;
}

// Offsets e .. e+3 of the bucket (0xffffffff past its count).
__device__ __forceinline__ uint4 load_offsets(const uint32_t *dpos, uint32_t e, uint32_t count)
{
    if (e + 4 <= count) return *reinterpret_cast<const uint4 *>(dpos + e);
    uint4 d;
    d.x = e < count ? dpos[e] : 0xffffffffu;
    d.y = e + 1 < count ? dpos[e + 1] : 0xffffffffu;
    d.z = e + 2 < count ? dpos[e + 2] : 0xffffffffu;
    d.w = e + 3 < count ? dpos[e + 3] : 0xffffffffu;
    return d;
}

__global__ void __launch_bounds__(kRankBlock) staged_rank_kernel(const __grid_constant__ StagedArgs a)
{
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) unsigned char s_raw[];
    __shared__ uint32_t s_warp[kRankWarps];
    __shared__ uint32_t s_thread_prefix[kRankBlock];
    __shared__ uint32_t s_part_count;  // entries of this CTA's part (read by later parts)
    __shared__ uint32_t s_base;        // entries of the span before this part

    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t w = a.sub_shift;
    const uint32_t parts_log2 = a.dst_shift - w;
    const uint32_t q = blockIdx.x >> parts_log2;              // bucket (span)
    const uint32_t part = blockIdx.x & ((1u << parts_log2) - 1u);
    const uint32_t words = w >= 5 ? 1u << (w - 5) : 1u;
    const uint32_t wmask = (1u << w) - 1u;
    uint32_t *s_bits = reinterpret_cast<uint32_t *>(s_raw);
    uint16_t *s_pre = reinterpret_cast<uint16_t *>(s_raw + size_t{words} * 4);
    uint32_t *s_super =
        reinterpret_cast<uint32_t *>(s_raw + size_t{words} * 4 + ((size_t{words} * 2 + 15) & ~size_t{15}));

    // the span's first slot: entries in the buckets before it
    uint32_t before = 0;
    for (uint32_t t = tid; t < q; t += kRankBlock) before += a.dst_cursor[t];
    before = __reduce_add_sync(kFull, before);
    if (lane == 0) s_warp[warp] = before;
    for (uint32_t t = tid; t < words; t += kRankBlock) s_bits[t] = 0u;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = __reduce_add_sync(kFull, s_warp[lane]);
        if (lane == 0) {
            if (part == 0) a.bucket_base[q] = v;
            s_base = 0u;
        }
    }
    const uint32_t count = a.dst_cursor[q];
    uint32_t *dpos = a.dpos + (static_cast<uint64_t>(q) << a.dst_shift);

    // the part's bitmap of kept indices
    for (uint32_t e0 = 4u * tid; e0 < count; e0 += 4u * kRankBlock * kRankUnroll) {
        uint4 d[kRankUnroll];
#pragma unroll
        for (int u = 0; u < kRankUnroll; ++u) d[u] = load_offsets(dpos, e0 + 4u * kRankBlock * u, count);
#pragma unroll
        for (int u = 0; u < kRankUnroll; ++u) {
            const uint32_t dd[4] = {d[u].x, d[u].y, d[u].z, d[u].w};
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (dd[c] != 0xffffffffu && (dd[c] >> w) == part)
                    atomicOr(&s_bits[(dd[c] & wmask) >> 5], 1u << (dd[c] & 31u));
        }
    }
    __syncthreads();

    // prefix counts: thread t owns `per` consecutive words (inside one
    // 2,048-word block), a block scan of their popcounts gives each thread's
    // exclusive prefix, and each word gets its prefix relative to its block
    const uint32_t per = words > kRankBlock ? words / kRankBlock : 1u;
    const uint32_t w0 = tid * per;
    uint32_t mine = 0;
    if (w0 < words)
        for (uint32_t u = 0; u < per; ++u) mine += __popc(s_bits[w0 + u]);
    const uint32_t incl = dev::warp_inclusive_scan(mine);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = s_warp[lane];
        const uint32_t vi = dev::warp_inclusive_scan(v);
        s_warp[lane] = vi - v;
        if (lane == 31) s_part_count = vi;
    }
    __syncthreads();
    const uint32_t excl = s_warp[warp] + incl - mine;
    s_thread_prefix[tid] = excl;
    __syncthreads();
    if (w0 < words) {
        const uint32_t block = w0 / kSuperWords;
        const uint32_t block_start = s_thread_prefix[(block * kSuperWords) / per];
        if (w0 % kSuperWords == 0) s_super[block] = block_start;
        uint32_t run = excl - block_start;
        for (uint32_t u = 0; u < per; ++u) {
            s_pre[w0 + u] = static_cast<uint16_t>(run);
            run += __popc(s_bits[w0 + u]);
        }
    }
    // the parts before this one (same cluster) hold the span's earlier slots
    if (parts_log2 != 0) {
        cg::cluster_group cluster = cg::this_cluster();
        cluster.sync();  // every part has read all offsets and counted its own
        if (tid == 0) {
            uint32_t earlier = 0;
            for (uint32_t r = 0; r < part; ++r) earlier += *cluster.map_shared_rank(&s_part_count, r);
            s_base = earlier;
        }
        cluster.sync();  // no CTA leaves while another reads its count; s_base, s_pre, s_super visible
    } else {
        __syncthreads();
    }

    // rewrite each of the part's offsets as its tagged slot offset in the bucket
    const uint32_t base = s_base;
    for (uint32_t e0 = 4u * tid; e0 < count; e0 += 4u * kRankBlock * kRankUnroll) {
        uint4 d[kRankUnroll];
#pragma unroll
        for (int u = 0; u < kRankUnroll; ++u) d[u] = load_offsets(dpos, e0 + 4u * kRankBlock * u, count);
#pragma unroll
        for (int u = 0; u < kRankUnroll; ++u) {
            uint32_t dd[4] = {d[u].x, d[u].y, d[u].z, d[u].w};
            bool mine4 = false;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                // past the count, ranked by another part, or in another part
                if (dd[c] == 0xffffffffu || (dd[c] & kRanked) != 0u || (dd[c] >> w) != part) continue;
                const uint32_t local = dd[c] & wmask;
                const uint32_t wd = local >> 5;
                const uint32_t rank = s_super[wd / kSuperWords] + s_pre[wd] +
                                      __popc(s_bits[wd] & ((1u << (local & 31u)) - 1u));
                dd[c] = kRanked | (base + rank);
                mine4 = true;
            }
            if (!mine4) continue;
            const uint32_t e = e0 + 4u * kRankBlock * u;
            if (e + 4 <= count && parts_log2 == 0) {
                *reinterpret_cast<uint4 *>(dpos + e) = make_uint4(dd[0], dd[1], dd[2], dd[3]);
            } else {
                // only this part's entries: the others belong to CTAs that may read them now
                const uint32_t old[4] = {d[u].x, d[u].y, d[u].z, d[u].w};
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (e + c < count && dd[c] != old[c]) dpos[e + c] = dd[c];
            }
        }
    }
}

// P2b of the ranked form: chunks of kSTile entries of one bucket, blockIdx.x
// over the bucket's reserved entries (chunks past the bucket's count exit),
// blockIdx.y over the buckets, so consecutive CTAs share a bucket.
template <class T>
__global__ void __launch_bounds__(kSBlock) staged_rank_scatter_kernel(const __grid_constant__ StagedArgs a)
{
    const uint32_t q = blockIdx.y;
    const uint32_t count = a.dst_cursor[q];
    const uint32_t first = blockIdx.x * kSTile;
    if (first >= count) return;
    const uint32_t base = a.bucket_base[q];
    const uint64_t span0 = static_cast<uint64_t>(q) << a.dst_shift;
    const T *dval = static_cast<const T *>(a.dval) + span0;
    const uint32_t *dpos = a.dpos + span0;
    T *out = static_cast<T *>(a.out);
    const uint32_t n = a.g.n;
    T v[kSItems];
    uint32_t off[kSItems];
#pragma unroll
    for (int j = 0; j < kSItems; ++j) {
        const uint32_t e = first + static_cast<uint32_t>(j * kSBlock) + threadIdx.x;
        off[j] = 0xffffffffu;
        if (e < count) {
            v[j] = __ldcs(dval + e);
            off[j] = __ldcs(dpos + e);
        }
    }
#pragma unroll
    for (int j = 0; j < kSItems; ++j) {
        if (off[j] == 0xffffffffu) continue;
        const uint32_t slot = base + (off[j] & ~kRanked);
        if ((off[j] & kRanked) != 0u && slot < n) out[slot] = v[j];
        else dev::record_error(a.ws, dev::kErrDeviceBounds, slot);
    }
}

// P1's dynamic shared memory for num_dst destination buckets.
template <class T, int ITEMS>
constexpr size_t p1_smem_bytes(uint32_t num_dst)
{
    return size_t{kP1Block} * ITEMS * (sizeof(T) + sizeof(uint32_t)) + 3u * num_dst * sizeof(uint32_t);
}

cudaError_t mark(cudaEvent_t *marks, int i, cudaStream_t stream)
{
    return marks != nullptr ? cudaEventRecord(marks[i], stream) : cudaSuccess;
}

// P1 with ITEMS per thread: the odd and even instances, each allowed the
// shared memory of 4096 buckets on first use on a device.
template <class T, bool FORWARD, int ITEMS, bool PADDED>
cudaError_t launch_p1(const StagedArgs &a, int device, cudaStream_t stream)
{
    using Kernel = void (*)(StagedArgs);
    Kernel odd, even;
    if constexpr (PADDED && ITEMS == 16 && sizeof(T) <= 8) {
        odd = staged_rank_bucket16_kernel<T, true>;
        even = staged_rank_bucket16_kernel<T, false>;
    } else if constexpr (PADDED) {
        odd = staged_rank_bucket_kernel<T, true, ITEMS>;
        even = staged_rank_bucket_kernel<T, false, ITEMS>;
    } else {
        odd = staged_bucket_kernel<T, true, FORWARD, ITEMS>;
        even = staged_bucket_kernel<T, false, FORWARD, ITEMS>;
    }
    static std::atomic<bool> configured[64];  // attribute set on this device
    if (!configured[device].load(std::memory_order_acquire)) {
        const int most = static_cast<int>(p1_smem_bytes<T, ITEMS>(4096));
        cudaError_t e = cudaFuncSetAttribute(odd, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(even, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        if (e != cudaSuccess) return e;
        configured[device].store(true, std::memory_order_release);
    }
    const size_t dyn = p1_smem_bytes<T, ITEMS>(a.num_dst);
    const uint64_t tile = uint64_t{kP1Block} * ITEMS;
    const unsigned chunks = static_cast<unsigned>((static_cast<uint64_t>(a.g.n) + tile - 1) / tile);
    ((a.g.k & 1u) ? odd : even)<<<chunks, kP1Block, dyn, stream>>>(a);
    return cudaGetLastError();
}

// P2 of the ranked form: P2a with one CTA per part of a span (clusters of
// the parts of one span when a span has more than one), then P2b.
template <class T>
cudaError_t launch_rank(const StagedArgs &a, int device, cudaStream_t stream)
{
    static std::atomic<bool> configured[64];  // attributes set on this device
    if (!configured[device].load(std::memory_order_acquire)) {
        cudaError_t e = cudaFuncSetAttribute(staged_rank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(rank_smem_bytes(kRankMaxSubShift)));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(staged_rank_scatter_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(kScatterSmemReserve));
        if (e != cudaSuccess) return e;
        configured[device].store(true, std::memory_order_release);
    }
    const uint32_t parts = 1u << (a.dst_shift - a.sub_shift);
    const size_t dyn = rank_smem_bytes(a.sub_shift);
    const unsigned grid = a.num_dst * parts;
    cudaError_t e = cudaSuccess;
    if (parts == 1) {
        staged_rank_kernel<<<grid, kRankBlock, dyn, stream>>>(a);
        e = cudaGetLastError();
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid, 1, 1);
        cfg.blockDim = dim3(kRankBlock, 1, 1);
        cfg.dynamicSmemBytes = dyn;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = parts;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, staged_rank_kernel, a);
    }
    if (e != cudaSuccess) return e;
    const dim3 grid2(static_cast<unsigned>(((uint64_t{1} << a.dst_shift) + kSTile - 1) / kSTile), a.num_dst, 1);
    staged_rank_scatter_kernel<T><<<grid2, kSBlock, kScatterSmemReserve, stream>>>(a);
    return cudaGetLastError();
}


template <class T, bool FORWARD>
cudaError_t launch_typed(const StagedArgs &a, uint32_t items, cudaStream_t stream, cudaEvent_t *marks)
{
    static std::atomic<bool> configured[64];  // attribute set on this device
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (!configured[device].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(staged_scatter_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kScatterSmemReserve));
        if (e != cudaSuccess) return e;
        configured[device].store(true, std::memory_order_release);
    }
    const bool padded = static_cast<uint64_t>(a.g.n) != a.g.domain;
    e = mark(marks, 0, stream);
    if (e != cudaSuccess) return e;
    if (padded) {
        if constexpr (!FORWARD)
            e = items == 16 ? launch_p1<T, false, 16, true>(a, device, stream)
                            : launch_p1<T, false, 8, true>(a, device, stream);
        else
            e = cudaErrorInvalidValue;  // the inverse shuffle has no ranked form
    } else if constexpr (sizeof(T) <= 8) {
        e = items == 16 ? launch_p1<T, FORWARD, 16, false>(a, device, stream)
                        : launch_p1<T, FORWARD, 8, false>(a, device, stream);
    } else {
        e = launch_p1<T, FORWARD, 8, false>(a, device, stream);
    }
    if (e == cudaSuccess) e = mark(marks, 1, stream);
    if (e != cudaSuccess) return e;
    if (padded) {
        e = launch_rank<T>(a, device, stream);
    } else {
        const unsigned chunks = static_cast<unsigned>(static_cast<uint64_t>(a.g.n) / kSTile);
        staged_scatter_kernel<T><<<chunks, kSBlock, kScatterSmemReserve, stream>>>(a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = mark(marks, 2, stream);
    return e;
}

// The ranked form's shape: one bucket per 8 elements of a P1 chunk (256
// buckets with 8 items per thread, 512 with 16), spans of at least 2^12
// indices, 16 items per thread where 8 would leave spans over 2^20 indices
// (one CTA then ranks a whole span up to 2^29-index domains), and at most 8
// parts of 2^20 indices per span (a portable cluster), with more buckets
// where a span would need more parts.
void rank_config(uint64_t n, uint32_t k, uint32_t elem_bytes, uint32_t *bucket_shift, uint32_t *sub_shift,
                 uint32_t *items)
{
    uint32_t it = p1_items_for(n, elem_bytes);
    if (k > 8 && k - 8 > BSHUFFLE_RANKED_MAX_SPAN_LOG2) it = 16;
    const uint32_t buckets_log2 = it == 16 ? 9u : 8u;
    uint32_t s = k > buckets_log2 ? k - buckets_log2 : 0u;
    const uint32_t floor_shift = k < 12 ? k : 12u;
    if (s < floor_shift) s = floor_shift;
    if (s > kRankMaxSubShift + 3) s = kRankMaxSubShift + 3;
    *bucket_shift = s;
    *sub_shift = s < kRankMaxSubShift ? s : kRankMaxSubShift;
    *items = it;
}

}  // namespace

uint32_t staged_tile_size() { return kStagedMinChunk; }

uint32_t staged_window_shift(uint64_t n, uint32_t elem_bytes)
{
    uint32_t lg = 0;
    while ((uint64_t{1} << lg) < n) ++lg;
    uint32_t eb_log2 = 0;
    while ((1u << eb_log2) < elem_bytes) ++eb_log2;
    // one bucket per 8 elements of a P1 chunk: 256 (or 512) buckets
    uint32_t bucket_log2 = 0;
    while ((8u << bucket_log2) < static_cast<uint32_t>(kP1Block) * p1_items_for(n, elem_bytes)) ++bucket_log2;
    uint32_t shift = lg > bucket_log2 ? lg - bucket_log2 : 0u;
    const uint32_t min_shift = kMinWindowLog2 > eb_log2 ? kMinWindowLog2 - eb_log2 : 0u;
    if (shift < min_shift) shift = min_shift;
    if (lg > 12 && shift < lg - 12) shift = lg - 12;  // at most 4096 buckets
    if (shift > lg) shift = lg;
    return shift;
}

void staged_rank_shifts(uint64_t n, uint32_t k, uint32_t elem_bytes, uint32_t *bucket_shift, uint32_t *sub_shift)
{
    uint32_t items = 0;
    rank_config(n, k, elem_bytes, bucket_shift, sub_shift, &items);
}


cudaError_t launch_staged(const StagedArgs &a, uint32_t elem_bytes, bool inverse, cudaStream_t stream,
                          cudaEvent_t *marks)
{
    uint32_t items = p1_items_for(a.g.n, elem_bytes);
    const uint64_t p1_tile = items == 16 ? kP1TileLarge : kP1TileSmall;
    if (static_cast<uint64_t>(a.g.n) != a.g.domain) {
        // ranked form: any n below its 2^k domain, gathers only
        uint32_t s = 0, w = 0;
        rank_config(a.g.n, a.g.k, elem_bytes, &s, &w, &items);
        if (inverse || a.g.n == 0 || a.g.domain > (uint64_t{1} << 32) || a.dst_shift != s || a.sub_shift != w ||
            (static_cast<uint64_t>(a.num_dst) << a.dst_shift) != a.g.domain || a.num_dst > 4096)
            return cudaErrorInvalidValue;
    } else if (a.num_dst > 4096 || a.g.domain < 2 * kStagedMinChunk || a.g.domain > (uint64_t{1} << 31) ||
               a.g.domain % p1_tile != 0 || (uint64_t{1} << a.dst_shift) < p1_tile ||
               (uint64_t{1} << a.dst_shift) < kSTile) {
        return cudaErrorInvalidValue;
    }
    switch (elem_bytes) {
    case 4: return inverse ? launch_typed<unsigned int, true>(a, items, stream, marks)
                           : launch_typed<unsigned int, false>(a, items, stream, marks);
    case 8: return inverse ? launch_typed<unsigned long long, true>(a, items, stream, marks)
                           : launch_typed<unsigned long long, false>(a, items, stream, marks);
    case 16: return inverse ? launch_typed<uint4, true>(a, items, stream, marks)
                            : launch_typed<uint4, false>(a, items, stream, marks);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bsh
