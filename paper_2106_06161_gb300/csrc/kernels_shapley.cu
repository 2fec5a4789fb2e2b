// Shapley values of a weighted voting game by permutation sampling (an
// application named in Sec. 1), fused with the shuffle.
//
// Game [q; w_0 .. w_{n-1}]: a coalition wins when its weight reaches q.
// Sample s orders the players by the shuffle of Algorithm 1 with seed
// seed0 + s (slot j holds player f(i_j)).  The player whose weight takes the
// running total of the players before it from below q to at least q is
// pivotal; counts[player] is incremented.  counts / samples estimates the
// Shapley values.  One warp owns one sample at a time: it walks the sample's
// domain in chunks of 32 * ITEMS indices in increasing order, forms the
// running weight with warp scans plus a carry (no block barrier, no
// inter-warp communication), and stops once the total reaches q.  The order
// itself never leaves registers.
#include <atomic>
#include <cstdint>

#include "bshuffle_device.cuh"
#include "bshuffle_internal.h"

namespace bsh {
namespace {

using dev::kFull;

constexpr int kSvBlock = 256;
constexpr int kSvWarps = kSvBlock / 32;
constexpr int kSvItems = 8;
constexpr uint32_t kSvChunk = 32 * kSvItems;

template <bool ODD>
__global__ void __launch_bounds__(kSvBlock) shapley_voting_kernel(const __grid_constant__ ShapleyArgs a)
{
    __shared__ uint32_t s_keys[kSvWarps][kMaxRounds];
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    const Geometry &g = a.g;
    uint32_t *keys = s_keys[warp];

    for (uint64_t smp = static_cast<uint64_t>(blockIdx.x) * kSvWarps + warp; smp < a.samples;
         smp += static_cast<uint64_t>(gridDim.x) * kSvWarps) {
        for (uint32_t r = lane; r < a.rounds; r += 32) keys[r] = dev::splitmix_key(a.seed0 + smp, r);
        __syncwarp();
        uint64_t carry = 0;  // weight of every kept player of the earlier chunks
        for (uint64_t base = 0; base < g.domain && carry < a.quota; base += kSvChunk) {
            uint32_t left[kSvItems], right[kSvItems];
#pragma unroll
            for (int j = 0; j < kSvItems; ++j) {
                const uint32_t i = static_cast<uint32_t>(base) + static_cast<uint32_t>(j * 32) + lane;
                left[j] = i >> g.R;
                right[j] = i & g.rmask;
            }
            dev::cipher_items<ODD, kSvItems>(left, right, keys, a.rounds, g);
#pragma unroll
            for (int j = 0; j < kSvItems; ++j) {
                const uint64_t i = base + static_cast<uint64_t>(j * 32) + lane;
                const uint32_t player = (left[j] << g.R) | right[j];
                const bool keep = i < g.domain && player < g.n;
                const uint32_t wt = keep ? a.w[player] : 0u;
                const uint64_t incl = dev::warp_inclusive_scan64(wt);
                const uint64_t before = carry + incl - wt;
                if (keep && before < a.quota && before + wt >= a.quota)
                    atomicAdd(reinterpret_cast<unsigned long long *>(a.counts + player), 1ull);
                carry += __shfl_sync(kFull, incl, 31);
            }
        }
        __syncwarp();  // every lane is done with the keys before the next sample's
    }
}

}  // namespace

cudaError_t launch_shapley_voting(const ShapleyArgs &a, cudaStream_t stream)
{
    static std::atomic<int> per_sm[64];  // CTAs to launch per device, 0 until first use
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    int ctas_cached = per_sm[device].load(std::memory_order_acquire);
    if (ctas_cached == 0) {
        int blocks = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, shapley_voting_kernel<true>, kSvBlock, 0);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        ctas_cached = (blocks > 0 ? blocks : 1) * sms;
        per_sm[device].store(ctas_cached, std::memory_order_release);
    }
    const uint64_t cap = static_cast<uint64_t>(ctas_cached);
    const uint64_t want = (a.samples + kSvWarps - 1) / kSvWarps;  // one warp per sample
    const unsigned grid = static_cast<unsigned>(want < cap ? want : cap);
    if (a.g.k & 1u)
        shapley_voting_kernel<true><<<grid, kSvBlock, 0, stream>>>(a);
    else
        shapley_voting_kernel<false><<<grid, kSvBlock, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace bsh
