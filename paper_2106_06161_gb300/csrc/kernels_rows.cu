// Fused single-pass kernels for wide elements (rows of a matrix), elem_bytes a
// multiple of 16 and larger than 16: Algorithm 1 of Sec. 4 with each X[b]
// being a whole row.
//
// A CTA owns kRowsPerTile consecutive domain indices, one per thread of its
// first warps.  It evaluates the bijection, ranks the kept indices, looks back
// for the tile's global prefix, records the (source, slot) pairs in shared
// memory, and then all its warps copy whole rows with 16-byte vector loads
// and stores: rows are contiguous, so both sides of the copy are fully
// coalesced.  Tiles are small and each lane keeps up to 8 loads in flight
// (a 4 KiB row per warp step), so that enough bytes are in flight per SM to
// cover the HBM latency: with 256 rows per tile a [65536 x 1024] FP32
// shuffle had fewer than two CTAs per SM and was latency-bound.
#include <cstdint>

#include "bshuffle_device.cuh"
#include "bshuffle_internal.h"

namespace bsh {
namespace {

using dev::kFull;

constexpr int kRowBlock = 256;
constexpr int kRowsPerTile = 64;
constexpr int kRowChunkUnroll = 8;

template <Mode MODE, bool ODD>
__global__ void __launch_bounds__(kRowBlock) rows_tile_kernel(const __grid_constant__ TileArgs a)
{
    constexpr int WARPS = kRowBlock / 32;
    constexpr int TILE_WARPS = kRowsPerTile / 32;  // warps that own domain indices
    __shared__ dev::TileShared<TILE_WARPS> st;
    __shared__ uint32_t s_src[kRowsPerTile];
    __shared__ uint32_t s_dst[kRowsPerTile];

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        st.tile = atomicAdd(&a.ws->ticket, 1u);
        st.tag = dev::ld_relaxed_gpu(&a.ws->tag);
    }
    __syncthreads();
    const uint32_t tile = st.tile;
    const uint32_t tag = st.tag;
    if (tile >= a.num_tiles) {  // only a corrupted header could hand out such a ticket
        if (threadIdx.x == 0) {
            dev::record_error(a.ws, dev::kErrDeviceBounds, tile);
            dev::finish_launch(a.ws, tag, gridDim.x);
        }
        return;
    }
    const bool owner = warp < static_cast<uint32_t>(TILE_WARPS);
    const uint32_t i = tile * static_cast<uint32_t>(kRowsPerTile) + threadIdx.x;
    bool keep = false;
    uint32_t src = 0, mask = 0;
    if (owner) {
        uint32_t left[1] = {i >> a.g.R};
        uint32_t right[1] = {i & a.g.rmask};
        dev::cipher_items<ODD, 1>(left, right, a.keys, a.rounds, a.g);
        src = (left[0] << a.g.R) | right[0];
        keep = static_cast<uint64_t>(i) < a.g.domain && src < a.g.n;
        mask = __ballot_sync(kFull, keep);
        if (lane == 0) st.counts[warp] = __popc(mask);
    }
    __syncthreads();
    if (warp == 0)
        dev::tile_scan_lookback<TILE_WARPS>(st, dev::StatusRing{a.status, ~0ull, 63u, tag}, tile, 0, a.timeout_ns,
                                              a.skip_publish_tile, a.ws);
    __syncthreads();
    const uint32_t prefix = st.prefix;
    const uint32_t count = st.aggregate;
    const bool ok = st.ok != 0u;
    if (keep) {
        const uint32_t local = st.counts[warp] + __popc(mask & dev::lanemask_lt());
        const uint32_t dst = prefix + local;
        if (dst >= a.g.n) {
            dev::record_error(a.ws, dev::kErrDeviceBounds, dst);
            keep = false;
        }
        s_src[local] = keep ? src : 0xffffffffu;
        s_dst[local] = dst;
    }
    __syncthreads();

    if (ok) {
        const uint32_t chunks = a.elem_bytes / 16u;
        const uint4 *in = static_cast<const uint4 *>(a.in);
        uint4 *out = static_cast<uint4 *>(a.out);
        for (uint32_t r = warp; r < count; r += WARPS) {
            const uint32_t s = s_src[r];
            if (s == 0xffffffffu) continue;
            const uint64_t from_row = MODE == Mode::Gather ? s : s_dst[r];
            const uint64_t to_row = MODE == Mode::Gather ? s_dst[r] : s;
            const uint4 *from = in + from_row * chunks;
            uint4 *to = out + to_row * chunks;
            for (uint32_t c0 = 0; c0 < chunks; c0 += 32u * kRowChunkUnroll) {
                uint4 v[kRowChunkUnroll];
#pragma unroll
                for (int u = 0; u < kRowChunkUnroll; ++u) {
                    const uint32_t c = c0 + static_cast<uint32_t>(u) * 32u + lane;
                    if (c < chunks) v[u] = __ldg(from + c);
                }
#pragma unroll
                for (int u = 0; u < kRowChunkUnroll; ++u) {
                    const uint32_t c = c0 + static_cast<uint32_t>(u) * 32u + lane;
                    if (c < chunks) to[c] = v[u];
                }
            }
        }
    }
    if (threadIdx.x == 0) dev::finish_launch(a.ws, tag, gridDim.x);
}

}  // namespace

uint32_t rows_tile_size() { return static_cast<uint32_t>(kRowsPerTile); }

cudaError_t launch_rows(const TileArgs &a, Mode mode, cudaStream_t stream)
{
    const dim3 grid(a.num_tiles), block(kRowBlock);
    const bool odd = (a.g.k & 1u) != 0u;
    if (mode == Mode::Gather) {
        if (odd) rows_tile_kernel<Mode::Gather, true><<<grid, block, 0, stream>>>(a);
        else rows_tile_kernel<Mode::Gather, false><<<grid, block, 0, stream>>>(a);
    } else if (mode == Mode::Scatter) {
        if (odd) rows_tile_kernel<Mode::Scatter, true><<<grid, block, 0, stream>>>(a);
        else rows_tile_kernel<Mode::Scatter, false><<<grid, block, 0, stream>>>(a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace bsh
