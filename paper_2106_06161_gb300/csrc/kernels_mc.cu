// Permutation Monte Carlo statistic fused with the shuffle (no output write).
//
// For each instance b the input x (length n) is shuffled with seed
// base_seed + b and the statistic T_b = mean(y[0:n1]) - mean(y[n1:n]) of the
// shuffled sequence y is returned in FP64.  The shuffled values never leave
// registers: a CTA owns whole instances, walks the instance's domain in
// chunks of BLOCK * ITEMS indices in increasing order, ranks the kept indices
// with a block scan plus a running count (no inter-CTA communication), and
// adds x[f(i)] to the first group's sum while the rank is below n1.  Slots are
// filled in increasing domain order, so once n1 elements are kept every later
// kept element belongs to the second group, whose sum is the total minus the
// first group's: the walk stops there.
#include <cstdint>

#include "bshuffle_device.cuh"
#include "bshuffle_internal.h"

namespace bsh {
namespace {

using dev::kFull;

constexpr int kMcBlock = 512;
constexpr int kMcItems = 4;
constexpr int kMcWarps = kMcBlock / 32;
constexpr uint32_t kMcChunk = kMcBlock * kMcItems;

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
    __shared__ uint32_t s_keys[kMaxRounds];
    __shared__ uint32_t s_counts[kMcItems * kMcWarps];
    __shared__ uint32_t s_aggregate;
    __shared__ double s_red[kMcWarps];
    __shared__ double s_total;

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    const Geometry &g = a.g;

    // sum of all of x, in the same order in every CTA
    double part = 0.0;
    for (uint32_t i = threadIdx.x; i < g.n; i += kMcBlock) part += static_cast<double>(a.x[i]);
    const double tot = block_sum(part, s_red);
    if (threadIdx.x == 0) s_total = tot;
    __syncthreads();
    const double total = s_total;

    for (uint32_t inst = blockIdx.x; inst < a.count; inst += gridDim.x) {
        for (uint32_t r = threadIdx.x; r < a.rounds; r += kMcBlock) s_keys[r] = dev::splitmix_key(a.base_seed + inst, r);
        __syncthreads();
        uint32_t running = 0;
        double s1 = 0.0;
        for (uint64_t base = 0; base < g.domain && running < a.n1; base += kMcChunk) {
            uint32_t left[kMcItems], right[kMcItems];
#pragma unroll
            for (int j = 0; j < kMcItems; ++j) {
                const uint32_t i = static_cast<uint32_t>(base) + static_cast<uint32_t>(j * kMcBlock) + threadIdx.x;
                left[j] = i >> g.R;
                right[j] = i & g.rmask;
            }
            dev::cipher_items<ODD, kMcItems>(left, right, s_keys, a.rounds, g);
            bool keep[kMcItems];
            float v[kMcItems];
            uint32_t mask[kMcItems];
#pragma unroll
            for (int j = 0; j < kMcItems; ++j) {
                const uint64_t i = base + static_cast<uint64_t>(j * kMcBlock) + threadIdx.x;
                const uint32_t src = (left[j] << g.R) | right[j];
                keep[j] = i < g.domain && src < g.n;
                v[j] = keep[j] ? a.x[src] : 0.0f;
                mask[j] = __ballot_sync(kFull, keep[j]);
            }
            if (lane == 0) {
#pragma unroll
                for (int j = 0; j < kMcItems; ++j) s_counts[j * kMcWarps + warp] = __popc(mask[j]);
            }
            __syncthreads();
            if (warp == 0) {
                constexpr int E = kMcItems * kMcWarps;
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
                if (lane == 31) s_aggregate = incl;
            }
            __syncthreads();
            const uint32_t lt = dev::lanemask_lt();
#pragma unroll
            for (int j = 0; j < kMcItems; ++j) {
                const uint32_t rank = running + s_counts[j * kMcWarps + warp] + __popc(mask[j] & lt);
                if (keep[j] && rank < a.n1) s1 += static_cast<double>(v[j]);
            }
            running += s_aggregate;
            __syncthreads();
        }
        const double first = block_sum(s1, s_red);
        if (threadIdx.x == 0)
            a.T[inst] = first / static_cast<double>(a.n1) - (total - first) / static_cast<double>(g.n - a.n1);
    }
}

}  // namespace

cudaError_t launch_mc(const McArgs &a, cudaStream_t stream)
{
    static int per_sm[64] = {0};
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (per_sm[device] == 0) {
        int blocks = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, mc_kernel<true>, kMcBlock, 0);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        per_sm[device] = (blocks > 0 ? blocks : 1) * sms;
    }
    const uint32_t grid = a.count < static_cast<uint32_t>(per_sm[device]) ? a.count : per_sm[device];
    if (a.g.k & 1u)
        mc_kernel<true><<<grid, kMcBlock, 0, stream>>>(a);
    else
        mc_kernel<false><<<grid, kMcBlock, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace bsh
