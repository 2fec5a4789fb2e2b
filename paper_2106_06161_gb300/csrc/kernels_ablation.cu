// The fusion ablation of Sec. 6: Algorithm 1 with less kernel fusion than the
// single-pass kernel ("Bijective2"), to measure what fusion buys on GB300.
//
//   Bijective0  three separate passes through global memory:
//                 transform   W[i] = f(i) for every domain index i
//                 compaction  J = the entries of W below n, in order (flags,
//                             in-tile scan, decoupled look-back)
//                 gather      Y[j] = X[J[j]]
//   Bijective1  transformation, compaction and gather fused, but the scan is
//               the two-pass kind (Harris et al.): a reduce pass evaluates f
//               and counts the kept indices per tile, a small scan of the tile
//               counts follows, and a second pass evaluates f again, ranks the
//               kept indices and gathers.
//
// Both produce exactly the output of bshuffle_permute.
#include <cstdint>

#include "bshuffle_device.cuh"
#include "bshuffle_internal.h"

namespace bsh {
namespace {

using dev::kFull;

constexpr int kABlock = 256;
constexpr int kAItems = 8;
constexpr int kAWarps = kABlock / 32;
constexpr uint32_t kATile = kABlock * kAItems;
constexpr int kScanThreads = 1024;

template <bool ODD>
__device__ __forceinline__ void evaluate(const AblationArgs &a, uint32_t base, uint32_t (&src)[kAItems],
                                         bool (&keep)[kAItems])
{
    uint32_t left[kAItems], right[kAItems];
#pragma unroll
    for (int j = 0; j < kAItems; ++j) {
        const uint32_t i = base + static_cast<uint32_t>(j * kABlock) + threadIdx.x;
        left[j] = i >> a.g.R;
        right[j] = i & a.g.rmask;
    }
    dev::cipher_items<ODD, kAItems>(left, right, a.keys, a.rounds, a.g);
#pragma unroll
    for (int j = 0; j < kAItems; ++j) {
        const uint32_t i = base + static_cast<uint32_t>(j * kABlock) + threadIdx.x;
        src[j] = (left[j] << a.g.R) | right[j];
        keep[j] = static_cast<uint64_t>(i) < a.g.domain && src[j] < a.g.n;
    }
}

// In-tile exclusive ranks of the kept items; returns the tile's kept count.
__device__ __forceinline__ uint32_t tile_ranks(const bool (&keep)[kAItems], uint32_t (&rank)[kAItems],
                                               uint32_t *s_counts, uint32_t *s_total)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t mask[kAItems];
#pragma unroll
    for (int j = 0; j < kAItems; ++j) mask[j] = __ballot_sync(kFull, keep[j]);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < kAItems; ++j) s_counts[j * kAWarps + warp] = __popc(mask[j]);
    }
    __syncthreads();
    if (warp == 0) {
        constexpr int E = kAItems * kAWarps;
        constexpr int C = (E + 31) / 32;
        uint32_t local[C];
        uint32_t sum = 0;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int e = static_cast<int>(lane) * C + c;
            local[c] = e < E ? s_counts[e] : 0u;
            sum += local[c];
        }
        const uint32_t incl = dev::warp_inclusive_scan(sum);
        uint32_t run = incl - sum;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int e = static_cast<int>(lane) * C + c;
            if (e < E) s_counts[e] = run;
            run += local[c];
        }
        if (lane == 31) *s_total = incl;
    }
    __syncthreads();
    const uint32_t lt = dev::lanemask_lt();
#pragma unroll
    for (int j = 0; j < kAItems; ++j) rank[j] = s_counts[j * kAWarps + warp] + __popc(mask[j] & lt);
    return *s_total;
}

// ---------------------------------------------------------------- Bijective0

template <bool ODD>
__global__ void __launch_bounds__(kABlock) transform_kernel(const __grid_constant__ AblationArgs a)
{
    const uint32_t base = blockIdx.x * kATile;
    uint32_t src[kAItems];
    bool keep[kAItems];
    evaluate<ODD>(a, base, src, keep);
#pragma unroll
    for (int j = 0; j < kAItems; ++j) {
        const uint32_t i = base + static_cast<uint32_t>(j * kABlock) + threadIdx.x;
        if (static_cast<uint64_t>(i) < a.g.domain) a.w[i] = src[j];
    }
}

__global__ void __launch_bounds__(kABlock) compact_kernel(const __grid_constant__ AblationArgs a)
{
    constexpr int ENTRIES = kAItems * kAWarps;
    __shared__ dev::TileShared<ENTRIES> st;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        st.tile = atomicAdd(&a.ws->ticket, 1u);
        st.tag = dev::ld_relaxed_gpu(&a.ws->tag);
    }
    __syncthreads();
    const uint32_t tile = st.tile, tag = st.tag;
    if (tile >= a.num_tiles) {
        if (threadIdx.x == 0) {
            dev::record_error(a.ws, dev::kErrDeviceBounds, tile);
            dev::finish_launch(a.ws, tag, gridDim.x);
        }
        return;
    }
    const uint32_t base = tile * kATile;
    uint32_t w[kAItems], mask[kAItems];
    bool keep[kAItems];
#pragma unroll
    for (int j = 0; j < kAItems; ++j) {
        const uint32_t i = base + static_cast<uint32_t>(j * kABlock) + threadIdx.x;
        const bool in_range = static_cast<uint64_t>(i) < a.g.domain;
        w[j] = in_range ? a.w[i] : 0xffffffffu;
        keep[j] = in_range && w[j] < a.g.n;
        mask[j] = __ballot_sync(kFull, keep[j]);
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < kAItems; ++j) st.counts[j * kAWarps + warp] = __popc(mask[j]);
    }
    __syncthreads();
    if (warp == 0)
        dev::tile_scan_lookback<ENTRIES>(st, dev::StatusRing{a.status, ~0ull, 63u, tag}, tile, 0, a.timeout_ns,
                                         -1, a.ws);
    __syncthreads();
    if (st.ok != 0u) {
        const uint32_t lt = dev::lanemask_lt();
#pragma unroll
        for (int j = 0; j < kAItems; ++j) {
            const uint32_t dst = st.prefix + st.counts[j * kAWarps + warp] + __popc(mask[j] & lt);
            if (keep[j]) {
                if (dst < a.g.n) a.j[dst] = w[j];
                else dev::record_error(a.ws, dev::kErrDeviceBounds, dst);
            }
        }
    }
    if (threadIdx.x == 0) dev::finish_launch(a.ws, tag, gridDim.x);
}

template <class T>
__global__ void __launch_bounds__(kABlock) gather_kernel(const __grid_constant__ AblationArgs a)
{
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kATile;
    const T *in = static_cast<const T *>(a.in);
    T *out = static_cast<T *>(a.out);
    T v[kAItems];
    bool ok[kAItems];
#pragma unroll
    for (int j = 0; j < kAItems; ++j) {
        const uint64_t e = base + static_cast<uint64_t>(j * kABlock) + threadIdx.x;
        ok[j] = false;
        if (e < a.g.n) {
            const uint32_t b = a.j[e];
            ok[j] = b < a.g.n;
            if (ok[j]) v[j] = __ldg(in + b);
            else dev::record_error(a.ws, dev::kErrDeviceBounds, e);
        }
    }
#pragma unroll
    for (int j = 0; j < kAItems; ++j) {
        const uint64_t e = base + static_cast<uint64_t>(j * kABlock) + threadIdx.x;
        if (ok[j]) out[e] = v[j];
    }
}

// ---------------------------------------------------------------- Bijective1

template <bool ODD>
__global__ void __launch_bounds__(kABlock) count_kernel(const __grid_constant__ AblationArgs a)
{
    __shared__ uint32_t s_counts[kAItems * kAWarps];
    __shared__ uint32_t s_total;
    uint32_t src[kAItems], rank[kAItems];
    bool keep[kAItems];
    evaluate<ODD>(a, blockIdx.x * kATile, src, keep);
    const uint32_t total = tile_ranks(keep, rank, s_counts, &s_total);
    if (threadIdx.x == 0) a.tile_count[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(const __grid_constant__ AblationArgs a)
{
    __shared__ uint32_t s_part[kScanThreads];
    const uint32_t tid = threadIdx.x, m = a.num_tiles;
    const uint32_t per = (m + kScanThreads - 1) / kScanThreads;
    const uint32_t b0 = tid * per;
    const uint32_t b1 = b0 + per < m ? b0 + per : m;
    uint32_t sum = 0;
    for (uint32_t t = b0; t < b1; ++t) sum += a.tile_count[t];
    s_part[tid] = sum;
    __syncthreads();
    for (uint32_t d = 1; d < kScanThreads; d <<= 1) {
        const uint32_t v = tid >= d ? s_part[tid - d] : 0u;
        __syncthreads();
        s_part[tid] += v;
        __syncthreads();
    }
    uint32_t run = s_part[tid] - sum;
    for (uint32_t t = b0; t < b1; ++t) {
        const uint32_t c = a.tile_count[t];
        a.tile_prefix[t] = run;
        run += c;
    }
}

template <class T, bool ODD>
__global__ void __launch_bounds__(kABlock) downsweep_kernel(const __grid_constant__ AblationArgs a)
{
    __shared__ uint32_t s_counts[kAItems * kAWarps];
    __shared__ uint32_t s_total;
    uint32_t src[kAItems], rank[kAItems];
    bool keep[kAItems];
    evaluate<ODD>(a, blockIdx.x * kATile, src, keep);
    const T *in = static_cast<const T *>(a.in);
    T v[kAItems];
#pragma unroll
    for (int j = 0; j < kAItems; ++j)
        if (keep[j]) v[j] = __ldg(in + src[j]);
    tile_ranks(keep, rank, s_counts, &s_total);
    const uint32_t prefix = a.tile_prefix[blockIdx.x];
    T *out = static_cast<T *>(a.out);
#pragma unroll
    for (int j = 0; j < kAItems; ++j) {
        if (keep[j]) {
            const uint32_t dst = prefix + rank[j];
            if (dst < a.g.n) out[dst] = v[j];
            else dev::record_error(a.ws, dev::kErrDeviceBounds, dst);
        }
    }
}

template <class T>
cudaError_t launch_t(const AblationArgs &a, int variant, cudaStream_t stream)
{
    const bool odd = (a.g.k & 1u) != 0u;
    const unsigned tiles = a.num_tiles;
    if (variant == 0) {
        if (odd) transform_kernel<true><<<tiles, kABlock, 0, stream>>>(a);
        else transform_kernel<false><<<tiles, kABlock, 0, stream>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        compact_kernel<<<tiles, kABlock, 0, stream>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const unsigned chunks = static_cast<unsigned>((static_cast<uint64_t>(a.g.n) + kATile - 1) / kATile);
        gather_kernel<T><<<chunks, kABlock, 0, stream>>>(a);
        return cudaGetLastError();
    }
    if (odd) count_kernel<true><<<tiles, kABlock, 0, stream>>>(a);
    else count_kernel<false><<<tiles, kABlock, 0, stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    tile_scan_kernel<<<1, kScanThreads, 0, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (odd) downsweep_kernel<T, true><<<tiles, kABlock, 0, stream>>>(a);
    else downsweep_kernel<T, false><<<tiles, kABlock, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

uint32_t ablation_tile_size() { return kATile; }

cudaError_t launch_ablation(const AblationArgs &a, uint32_t elem_bytes, int variant, cudaStream_t stream)
{
    if (variant != 0 && variant != 1) return cudaErrorInvalidValue;
    switch (elem_bytes) {
    case 4: return launch_t<unsigned int>(a, variant, stream);
    case 8: return launch_t<unsigned long long>(a, variant, stream);
    case 16: return launch_t<uint4>(a, variant, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bsh
