// Shapley values of a weighted voting game by permutation sampling (an
// application named in Sec. 1), fused with the shuffle.
//
// Game [q; w_0 .. w_{n-1}]: a coalition wins when its weight reaches q.
// Sample s orders the players by the shuffle of Algorithm 1 with seed
// seed0 + s (slot j holds player f(i_j)).  The player whose weight takes the
// running total of the players before it from below q to at least q is
// pivotal; counts[player] is incremented.  counts / samples estimates the
// Shapley values.  A CTA owns whole samples: it walks the sample's domain in
// chunks of BLOCK * ITEMS indices in increasing order, forms the running
// weight with a block scan plus a carry (no inter-CTA communication), and
// stops after the chunk in which the total reaches q.  The order itself never
// leaves registers.
#include <cstdint>

#include "bshuffle_device.cuh"
#include "bshuffle_internal.h"

namespace bsh {
namespace {

using dev::kFull;

constexpr int kSvBlock = 256;
constexpr int kSvItems = 8;
constexpr int kSvWarps = kSvBlock / 32;
constexpr uint32_t kSvChunk = kSvBlock * kSvItems;

template <bool ODD>
__global__ void __launch_bounds__(kSvBlock) shapley_voting_kernel(const __grid_constant__ ShapleyArgs a)
{
    constexpr int E = kSvItems * kSvWarps;
    constexpr int C = (E + 31) / 32;
    __shared__ uint32_t s_keys[kMaxRounds];
    __shared__ uint64_t s_part[E];  // per (item, warp) weight sums, then their exclusive offsets
    __shared__ uint64_t s_chunk;    // weight of the kept players of the chunk

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    const Geometry &g = a.g;

    for (uint64_t smp = blockIdx.x; smp < a.samples; smp += gridDim.x) {
        for (uint32_t r = threadIdx.x; r < a.rounds; r += kSvBlock) s_keys[r] = dev::splitmix_key(a.seed0 + smp, r);
        __syncthreads();
        uint64_t carry = 0;  // weight of every kept player of the earlier chunks
        for (uint64_t base = 0; base < g.domain && carry < a.quota; base += kSvChunk) {
            uint32_t left[kSvItems], right[kSvItems];
#pragma unroll
            for (int j = 0; j < kSvItems; ++j) {
                const uint32_t i = static_cast<uint32_t>(base) + static_cast<uint32_t>(j * kSvBlock) + threadIdx.x;
                left[j] = i >> g.R;
                right[j] = i & g.rmask;
            }
            dev::cipher_items<ODD, kSvItems>(left, right, s_keys, a.rounds, g);
            uint32_t player[kSvItems], wt[kSvItems];
            uint64_t incl[kSvItems];
#pragma unroll
            for (int j = 0; j < kSvItems; ++j) {
                const uint64_t i = base + static_cast<uint64_t>(j * kSvBlock) + threadIdx.x;
                player[j] = (left[j] << g.R) | right[j];
                const bool keep = i < g.domain && player[j] < g.n;
                wt[j] = keep ? a.w[player[j]] : 0u;
                if (!keep) player[j] = 0xffffffffu;
            }
#pragma unroll
            for (int j = 0; j < kSvItems; ++j) {
                incl[j] = dev::warp_inclusive_scan64(wt[j]);
                if (lane == 31) s_part[j * kSvWarps + warp] = incl[j];
            }
            __syncthreads();
            if (warp == 0) {
                uint64_t local[C];
                uint64_t sum = 0;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int e = static_cast<int>(lane) * C + c;
                    local[c] = e < E ? s_part[e] : 0ull;
                    sum += local[c];
                }
                const uint64_t total = dev::warp_inclusive_scan64(sum);
                uint64_t run = total - sum;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int e = static_cast<int>(lane) * C + c;
                    if (e < E) s_part[e] = run;
                    run += local[c];
                }
                if (lane == 31) s_chunk = total;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < kSvItems; ++j) {
                const uint64_t before = carry + s_part[j * kSvWarps + warp] + incl[j] - wt[j];
                if (player[j] < g.n && before < a.quota && before + wt[j] >= a.quota)
                    atomicAdd(reinterpret_cast<unsigned long long *>(a.counts + player[j]), 1ull);
            }
            carry += s_chunk;
            __syncthreads();
        }
    }
}

}  // namespace

cudaError_t launch_shapley_voting(const ShapleyArgs &a, cudaStream_t stream)
{
    static int per_sm[64] = {0};
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (per_sm[device] == 0) {
        int blocks = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, shapley_voting_kernel<true>, kSvBlock, 0);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        per_sm[device] = (blocks > 0 ? blocks : 1) * sms;
    }
    const uint64_t cap = static_cast<uint64_t>(per_sm[device]);
    const unsigned grid = static_cast<unsigned>(a.samples < cap ? a.samples : cap);
    if (a.g.k & 1u)
        shapley_voting_kernel<true><<<grid, kSvBlock, 0, stream>>>(a);
    else
        shapley_voting_kernel<false><<<grid, kSvBlock, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace bsh
