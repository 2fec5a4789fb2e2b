// Fused single-pass kernels for wide elements (rows of a matrix), elem_bytes a
// multiple of 16 and larger than 16: Algorithm 1 of Sec. 4 with each X[b]
// being a whole row.
//
// A persistent CTA takes tiles of ROWS consecutive domain indices,
// one per thread of its first warps.  It evaluates the bijection, ranks the kept indices, looks back
// for the tile's global prefix, records the (source, slot) pairs in shared
// memory, and then all its warps copy whole rows with 16-byte vector loads
// and stores: rows are contiguous, so both sides of the copy are fully
// coalesced.  Tiles are small and each lane keeps up to 8 loads in flight
// (a 4 KiB row per warp step), so that enough bytes are in flight per SM to
// cover the HBM latency: with 256 rows per tile a [65536 x 1024] FP32
// shuffle had fewer than two CTAs per SM and was latency-bound.
#include <atomic>
#include <cstdint>

#include "bshuffle_device.cuh"
#include "bshuffle_internal.h"

namespace bsh {
namespace {

using dev::kFull;

constexpr int kRowBlock = 256;
// Rows per tile: 128 for rows of up to 2 KiB, 64 for longer ones (measured:
// [65536 x 1024] BF16 9 % faster with 128, FP32 the same with 64 or 128).
constexpr uint32_t rows_per_tile(uint32_t row_bytes) { return row_bytes <= 2048u ? 128u : 64u; }
constexpr int kRowChunkUnroll = 8;

template <Mode MODE, bool ODD, int ROWS>
__global__ void __launch_bounds__(kRowBlock) rows_tile_kernel(const __grid_constant__ TileArgs a)
{
    constexpr int WARPS = kRowBlock / 32;
    constexpr int TILE_WARPS = ROWS / 32;  // warps that own domain indices
    __shared__ dev::TileShared<TILE_WARPS> st;
    __shared__ uint32_t s_src[ROWS];
    __shared__ uint32_t s_dst[ROWS];

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) st.tag = dev::ld_relaxed_gpu(&a.ws->tag);
    // Persistent: a CTA takes tiles until the tickets run out (a ticket only
    // when it is ready to start the tile), so the last wave holds no idle SMs.
    for (;;) {
    if (threadIdx.x == 0) st.tile = atomicAdd(&a.ws->ticket, 1u);
    __syncthreads();
    const uint32_t tile = st.tile;
    const uint32_t tag = st.tag;
    if (tile >= a.num_tiles) break;
    const bool owner = warp < static_cast<uint32_t>(TILE_WARPS);
    const uint32_t i = tile * static_cast<uint32_t>(ROWS) + threadIdx.x;
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
    __syncthreads();  // the tile's shared state is reused by the next one
    }
    if (threadIdx.x == 0) dev::finish_launch(a.ws, st.tag, gridDim.x);
}

}  // namespace

uint32_t rows_tile_size(uint32_t row_bytes) { return rows_per_tile(row_bytes); }

template <int ROWS>
cudaError_t launch_rows_t(const TileArgs &a, Mode mode, cudaStream_t stream)
{
    static std::atomic<int> per_sm[64];  // CTAs to launch per device, 0 until first use
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    int ctas_cached = per_sm[device].load(std::memory_order_acquire);
    if (ctas_cached == 0) {
        int blocks = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, rows_tile_kernel<Mode::Gather, true, ROWS>,
                                                          kRowBlock, 0);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        ctas_cached = (blocks > 0 ? blocks : 1) * sms;
        per_sm[device].store(ctas_cached, std::memory_order_release);
    }
    const uint32_t ctas = a.num_tiles < static_cast<uint32_t>(ctas_cached) ? a.num_tiles : ctas_cached;
    const dim3 grid(ctas), block(kRowBlock);
    const bool odd = (a.g.k & 1u) != 0u;
    if (mode == Mode::Gather) {
        if (odd) rows_tile_kernel<Mode::Gather, true, ROWS><<<grid, block, 0, stream>>>(a);
        else rows_tile_kernel<Mode::Gather, false, ROWS><<<grid, block, 0, stream>>>(a);
    } else if (mode == Mode::Scatter) {
        if (odd) rows_tile_kernel<Mode::Scatter, true, ROWS><<<grid, block, 0, stream>>>(a);
        else rows_tile_kernel<Mode::Scatter, false, ROWS><<<grid, block, 0, stream>>>(a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_rows(const TileArgs &a, Mode mode, cudaStream_t stream)
{
    return rows_per_tile(a.elem_bytes) == 128u ? launch_rows_t<128>(a, mode, stream)
                                                : launch_rows_t<64>(a, mode, stream);
}

}  // namespace bsh
