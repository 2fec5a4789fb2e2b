// Staged shuffle of power-of-two lengths much larger than L2: the same
// permutation as the fused single pass (Algorithm 1, Sec. 4), with every HBM
// access sequential and the random accesses confined to L2-resident windows.
// The inverse shuffle (out[f(j)] = in[j]) runs the same two passes with the
// forward cipher in place of the inverse one.
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
#include <atomic>
#include <cstdint>

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
// f^-1(b) (the shuffle).  The round keys sit in kernel parameter space, so
// the unrolled 24 rounds read them as constant operands.
template <class T, bool ODD, bool FORWARD, int ITEMS>
__global__ void __launch_bounds__(kP1Block) staged_bucket_kernel(const __grid_constant__ StagedArgs a)
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
    const uint32_t first = blockIdx.x * kP1Tile;  // n = 2^k is a multiple of kP1Tile
    const T *in = static_cast<const T *>(a.in);
    for (uint32_t q = tid; q < a.num_dst; q += kP1Block) s_cnt[q] = 0u;

    T val[kP1Items];
    uint32_t left[kP1Items], right[kP1Items];
#pragma unroll
    for (int j = 0; j < kP1Items; ++j) {
        const uint32_t b = first + static_cast<uint32_t>(j * kP1Block) + tid;
        val[j] = __ldcs(in + b);
        left[j] = b >> g.R;
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
    for (int j = 0; j < kP1Items; ++j) slot[j] = atomicAdd(&s_cnt[dst[j] >> a.dst_shift], 1u);
    __syncthreads();
    block_exclusive_scan(s_cnt, s_start, a.num_dst, s_warp);
    for (uint32_t q = tid; q < a.num_dst; q += kP1Block) {
        const uint32_t c = s_cnt[q];
        s_gbase[q] = c != 0u ? atomicAdd(&a.dst_cursor[q], c) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kP1Items; ++j) {
        const uint32_t p = s_start[dst[j] >> a.dst_shift] + slot[j];
        s_val[p] = val[j];
        s_dst[p] = dst[j];
    }
    __syncthreads();
    T *dval = static_cast<T *>(a.dval);
    const uint32_t bsize = 1u << a.dst_shift;
#pragma unroll
    for (int j = 0; j < kP1Items; ++j) {
        const uint32_t p = static_cast<uint32_t>(j * kP1Block) + tid;
        const uint32_t d = s_dst[p];
        const uint32_t q = d >> a.dst_shift;
        const uint32_t off = s_gbase[q] + (p - s_start[q]);
        if (off < bsize) {
            const uint32_t o = (q << a.dst_shift) + off;
            dval[o] = s_val[p];
            a.dpos[o] = d & (bsize - 1u);
        } else {
            dev::record_error(a.ws, dev::kErrDeviceBounds, (static_cast<uint64_t>(q) << a.dst_shift) + off);
        }
    }
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
template <class T, bool FORWARD, int ITEMS>
cudaError_t launch_p1(const StagedArgs &a, int device, cudaStream_t stream)
{
    static std::atomic<bool> configured[64];  // attribute set on this device
    if (!configured[device].load(std::memory_order_acquire)) {
        const int most = static_cast<int>(p1_smem_bytes<T, ITEMS>(4096));
        cudaError_t e = cudaSuccess;
        for (const void *k : {reinterpret_cast<const void *>(staged_bucket_kernel<T, true, FORWARD, ITEMS>),
                              reinterpret_cast<const void *>(staged_bucket_kernel<T, false, FORWARD, ITEMS>)})
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        if (e != cudaSuccess) return e;
        configured[device].store(true, std::memory_order_release);
    }
    const size_t dyn = p1_smem_bytes<T, ITEMS>(a.num_dst);
    const unsigned chunks = static_cast<unsigned>(static_cast<uint64_t>(a.g.n) / (uint64_t{kP1Block} * ITEMS));
    if (a.g.k & 1u)
        staged_bucket_kernel<T, true, FORWARD, ITEMS><<<chunks, kP1Block, dyn, stream>>>(a);
    else
        staged_bucket_kernel<T, false, FORWARD, ITEMS><<<chunks, kP1Block, dyn, stream>>>(a);
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
    const unsigned chunks = static_cast<unsigned>(static_cast<uint64_t>(a.g.n) / kSTile);
    e = mark(marks, 0, stream);
    if (e != cudaSuccess) return e;
    if constexpr (sizeof(T) <= 8)
        e = items == 16 ? launch_p1<T, FORWARD, 16>(a, device, stream) : launch_p1<T, FORWARD, 8>(a, device, stream);
    else
        e = launch_p1<T, FORWARD, 8>(a, device, stream);
    if (e == cudaSuccess) e = mark(marks, 1, stream);
    if (e != cudaSuccess) return e;
    staged_scatter_kernel<T><<<chunks, kSBlock, kScatterSmemReserve, stream>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = mark(marks, 2, stream);
    return e;
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

cudaError_t launch_staged(const StagedArgs &a, uint32_t elem_bytes, bool inverse, cudaStream_t stream,
                          cudaEvent_t *marks)
{
    const uint32_t items = p1_items_for(a.g.n, elem_bytes);
    const uint64_t p1_tile = items == 16 ? kP1TileLarge : kP1TileSmall;
    if (a.num_dst > 4096 || static_cast<uint64_t>(a.g.n) != a.g.domain || a.g.domain < 2 * kStagedMinChunk ||
        a.g.domain > (uint64_t{1} << 31) || a.g.domain % p1_tile != 0 || (uint64_t{1} << a.dst_shift) < p1_tile ||
        (uint64_t{1} << a.dst_shift) < kSTile)
        return cudaErrorInvalidValue;
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
