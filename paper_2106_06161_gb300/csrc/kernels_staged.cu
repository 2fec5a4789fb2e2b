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
//   P1  per chunk of 2,048 consecutive elements b: a coalesced read of X[b],
//       the inverse cipher j = f^-1(b), and a counting sort of (value, j) by
//       destination bucket (j >> dst_shift, an 8 MiB output window) in shared
//       memory; each bucket's run is appended with one global atomic per
//       bucket per chunk.
//   P2  per chunk of one destination bucket: out[j] = value, random within an
//       L2-resident output window whose lines leave L2 complete.
//
// Runs are appended in a nondeterministic order, but every element is placed
// by its exact slot, so the output is deterministic and identical to the
// single pass.
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
// buckets kP1Block * kSItems consecutive elements.
#ifndef BSHUFFLE_STAGED_P1_BLOCK
#define BSHUFFLE_STAGED_P1_BLOCK 256
#endif
constexpr int kP1Block = BSHUFFLE_STAGED_P1_BLOCK;
constexpr int kP1Warps = kP1Block / 32;
constexpr uint32_t kP1Tile = kP1Block * kSItems;
constexpr uint32_t kStagedMinChunk = kP1Tile > kSTile ? kP1Tile : kSTile;

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

// Streaming read of data used once (evict-first in L1 and L2).
// ------------------------------------------------------------------ P1

// FORWARD: element b goes to slot f(b) (the inverse shuffle) instead of
// f^-1(b) (the shuffle).
template <class T, bool ODD, bool FORWARD>
__global__ void __launch_bounds__(kP1Block) staged_bucket_kernel(const __grid_constant__ StagedArgs a)
{
    // dynamic shared memory: the chunk's sorted (value, position, bucket)
    // staging, then three words per destination bucket
    extern __shared__ __align__(16) unsigned char s_raw[];
    T *s_val = reinterpret_cast<T *>(s_raw);
    uint32_t *s_pos = reinterpret_cast<uint32_t *>(s_raw + kP1Tile * sizeof(T));
    uint16_t *s_bucket = reinterpret_cast<uint16_t *>(s_raw + kP1Tile * (sizeof(T) + 4));
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(s_raw + kP1Tile * (sizeof(T) + 6));
    uint32_t *s_start = s_cnt + a.num_dst;
    uint32_t *s_gbase = s_start + a.num_dst;
    __shared__ uint32_t s_warp[kP1Warps];

    const uint32_t tid = threadIdx.x;
    const Geometry &g = a.g;
    const uint32_t first = blockIdx.x * kP1Tile;  // n = 2^k is a multiple of kP1Tile
    const T *in = static_cast<const T *>(a.in);
    for (uint32_t q = tid; q < a.num_dst; q += kP1Block) s_cnt[q] = 0u;

    T val[kSItems];
    uint32_t left[kSItems], right[kSItems];
#pragma unroll
    for (int j = 0; j < kSItems; ++j) {
        const uint32_t b = first + static_cast<uint32_t>(j * kP1Block) + tid;
        val[j] = __ldcs(in + b);
        left[j] = b >> g.R;
        right[j] = b & g.rmask;
    }
    if constexpr (FORWARD)
        dev::cipher_items<ODD, kSItems>(left, right, a.keys, a.rounds, g);
    else
        dev::cipher_inverse_items<ODD, kSItems>(left, right, a.keys, a.rounds, g);
    uint32_t bucket[kSItems], pos[kSItems], slot[kSItems];
#pragma unroll
    for (int j = 0; j < kSItems; ++j) {
        const uint32_t dst = (left[j] << g.R) | right[j];  // f^-1(b) (or f(b)): the element's output slot
        bucket[j] = dst >> a.dst_shift;
        pos[j] = dst & ((1u << a.dst_shift) - 1u);
    }
    __syncthreads();  // s_cnt zeroed
#pragma unroll
    for (int j = 0; j < kSItems; ++j) slot[j] = atomicAdd(&s_cnt[bucket[j]], 1u);
    __syncthreads();
    block_exclusive_scan(s_cnt, s_start, a.num_dst, s_warp);
    for (uint32_t q = tid; q < a.num_dst; q += kP1Block) {
        const uint32_t c = s_cnt[q];
        s_gbase[q] = c != 0u ? atomicAdd(&a.dst_cursor[q], c) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSItems; ++j) {
        const uint32_t p = s_start[bucket[j]] + slot[j];
        s_val[p] = val[j];
        s_pos[p] = pos[j];
        s_bucket[p] = static_cast<uint16_t>(bucket[j]);
    }
    __syncthreads();
    T *dval = static_cast<T *>(a.dval);
    const uint64_t bsize = uint64_t{1} << a.dst_shift;
    for (uint32_t p = tid; p < kP1Tile; p += kP1Block) {
        const uint32_t q = s_bucket[p];
        const uint64_t off = static_cast<uint64_t>(s_gbase[q]) + (p - s_start[q]);
        const uint64_t bucket_base = static_cast<uint64_t>(q) << a.dst_shift;
        if (off < bsize) {
            dval[bucket_base + off] = s_val[p];
            a.dpos[bucket_base + off] = s_pos[p];
        } else {
            dev::record_error(a.ws, dev::kErrDeviceBounds, bucket_base + off);
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
template <class T>
constexpr size_t p1_smem_bytes(uint32_t num_dst)
{
    return kP1Tile * (sizeof(T) + sizeof(uint32_t) + sizeof(uint16_t)) + 3u * num_dst * sizeof(uint32_t);
}

cudaError_t mark(cudaEvent_t *marks, int i, cudaStream_t stream)
{
    return marks != nullptr ? cudaEventRecord(marks[i], stream) : cudaSuccess;
}

template <class T, bool FORWARD>
cudaError_t launch_typed(const StagedArgs &a, cudaStream_t stream, cudaEvent_t *marks)
{
    static bool configured[64] = {false};
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (!configured[device]) {
        e = cudaFuncSetAttribute(staged_bucket_kernel<T, true, FORWARD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(p1_smem_bytes<T>(4096)));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(staged_bucket_kernel<T, false, FORWARD>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(p1_smem_bytes<T>(4096)));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(staged_scatter_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(kScatterSmemReserve));
        if (e != cudaSuccess) return e;
        configured[device] = true;
    }
    const size_t dyn = p1_smem_bytes<T>(a.num_dst);
    const unsigned chunks = static_cast<unsigned>(static_cast<uint64_t>(a.g.n) / kSTile);
    const unsigned p1_chunks = static_cast<unsigned>(static_cast<uint64_t>(a.g.n) / kP1Tile);
    e = mark(marks, 0, stream);
    if (e != cudaSuccess) return e;
    if (a.g.k & 1u)
        staged_bucket_kernel<T, true, FORWARD><<<p1_chunks, kP1Block, dyn, stream>>>(a);
    else
        staged_bucket_kernel<T, false, FORWARD><<<p1_chunks, kP1Block, dyn, stream>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = mark(marks, 1, stream);
    if (e != cudaSuccess) return e;
    staged_scatter_kernel<T><<<chunks, kSBlock, kScatterSmemReserve, stream>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = mark(marks, 2, stream);
    return e;
}

}  // namespace

uint32_t staged_tile_size() { return kStagedMinChunk; }

cudaError_t launch_staged(const StagedArgs &a, uint32_t elem_bytes, bool inverse, cudaStream_t stream,
                          cudaEvent_t *marks)
{
    if (a.num_dst > 4096 || static_cast<uint64_t>(a.g.n) != a.g.domain || a.g.domain < 2 * kStagedMinChunk ||
        a.g.domain > (uint64_t{1} << 31) || (uint64_t{1} << a.dst_shift) < kStagedMinChunk)
        return cudaErrorInvalidValue;
    switch (elem_bytes) {
    case 4: return inverse ? launch_typed<unsigned int, true>(a, stream, marks)
                           : launch_typed<unsigned int, false>(a, stream, marks);
    case 8: return inverse ? launch_typed<unsigned long long, true>(a, stream, marks)
                           : launch_typed<unsigned long long, false>(a, stream, marks);
    case 16: return inverse ? launch_typed<uint4, true>(a, stream, marks) : launch_typed<uint4, false>(a, stream, marks);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bsh
