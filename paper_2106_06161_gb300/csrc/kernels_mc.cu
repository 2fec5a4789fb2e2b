// Permutation Monte Carlo statistic fused with the shuffle (no output write).
//
// For each instance b the input x (length n) is shuffled with seed
// base_seed + b and the statistic T_b = mean(y[0:n1]) - mean(y[n1:n]) of the
// shuffled sequence y is returned in FP64.  The shuffled values never leave
// registers: one warp owns one instance at a time and walks its domain in
// chunks of 32 * ITEMS indices in increasing order, ranking the kept indices
// with ballots and a running count (no block barrier, no inter-warp
// communication), and adds x[f(i)] to the first group's sum while the rank is
// below n1.  Slots are filled in increasing domain order, so once n1 elements
// are kept every later kept element belongs to the second group, whose sum
// is the total minus the first group's: the walk stops there.  The total is
// summed once per CTA, in the same order in every CTA.
#include <atomic>
#include <cstdint>

#include "bshuffle_device.cuh"
#include "bshuffle_internal.h"

namespace bsh {
namespace {

using dev::kFull;

constexpr int kMcBlock = 256;
constexpr int kMcWarps = kMcBlock / 32;
constexpr int kMcItems = 8;
constexpr uint32_t kMcChunk = 32 * kMcItems;

__device__ __forceinline__ double block_sum(double v, double *s_red)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(kFull, v, d);
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < static_cast<uint32_t>(kMcWarps) ? s_red[lane] : 0.0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(kFull, t, d);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

template <bool ODD>
__global__ void __launch_bounds__(kMcBlock) mc_kernel(const __grid_constant__ McArgs a)
{
    __shared__ uint32_t s_keys[kMcWarps][kMaxRounds];
    __shared__ double s_red[kMcWarps];
    __shared__ double s_total;

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t lt = dev::lanemask_lt();
    const Geometry &g = a.g;

    // sum of all of x, in the same order in every CTA
    double part = 0.0;
    for (uint32_t i = threadIdx.x; i < g.n; i += kMcBlock) part += static_cast<double>(a.x[i]);
    const double tot = block_sum(part, s_red);
    if (threadIdx.x == 0) s_total = tot;
    __syncthreads();
    const double total = s_total;
    uint32_t *keys = s_keys[warp];

    for (uint32_t inst = blockIdx.x * kMcWarps + warp; inst < a.count; inst += gridDim.x * kMcWarps) {
        for (uint32_t r = lane; r < a.rounds; r += 32) keys[r] = dev::splitmix_key(a.base_seed + inst, r);
        __syncwarp();
        uint32_t running = 0;
        double s1 = 0.0;
        for (uint64_t base = 0; base < g.domain && running < a.n1; base += kMcChunk) {
            uint32_t left[kMcItems], right[kMcItems];
#pragma unroll
            for (int j = 0; j < kMcItems; ++j) {
                const uint32_t i = static_cast<uint32_t>(base) + static_cast<uint32_t>(j * 32) + lane;
                left[j] = i >> g.R;
                right[j] = i & g.rmask;
            }
            dev::cipher_items<ODD, kMcItems>(left, right, keys, a.rounds, g);
#pragma unroll
            for (int j = 0; j < kMcItems; ++j) {
                const uint64_t i = base + static_cast<uint64_t>(j * 32) + lane;
                const uint32_t src = (left[j] << g.R) | right[j];
                const bool keep = i < g.domain && src < g.n;
                const uint32_t m = __ballot_sync(kFull, keep);
                if (keep && running + static_cast<uint32_t>(__popc(m & lt)) < a.n1) s1 += static_cast<double>(a.x[src]);
                running += static_cast<uint32_t>(__popc(m));
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s1 += __shfl_down_sync(kFull, s1, d);
        if (lane == 0)
            a.T[inst] = s1 / static_cast<double>(a.n1) - (total - s1) / static_cast<double>(g.n - a.n1);
        __syncwarp();  // every lane is done with the keys before the next instance's
    }
}

}  // namespace

cudaError_t launch_mc(const McArgs &a, cudaStream_t stream)
{
    static std::atomic<int> per_sm[64];  // CTAs to launch per device, 0 until first use
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    int ctas_cached = per_sm[device].load(std::memory_order_acquire);
    if (ctas_cached == 0) {
        int blocks = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, mc_kernel<true>, kMcBlock, 0);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        ctas_cached = (blocks > 0 ? blocks : 1) * sms;
        per_sm[device].store(ctas_cached, std::memory_order_release);
    }
    const uint32_t want = (a.count + kMcWarps - 1) / kMcWarps;  // one warp per instance
    const uint32_t grid = want < static_cast<uint32_t>(ctas_cached) ? want : ctas_cached;
    if (a.g.k & 1u)
        mc_kernel<true><<<grid, kMcBlock, 0, stream>>>(a);
    else
        mc_kernel<false><<<grid, kMcBlock, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace bsh
