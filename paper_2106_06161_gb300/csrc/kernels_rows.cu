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

// ------------------------------------------------------------------ two-kernel form
//
// For up to kRowsSumTiles tiles the inter-tile prefix needs no chain: the
// count kernel writes every tile's kept count (no data read), and each CTA of the copy kernel adds the counts of the tiles
// before it itself (at most a few thousand L2-resident words).  The copy
// kernel is a programmatic dependent launch: its CTAs evaluate the bijection
// and rank their tile while the count kernel runs, and wait for it
// (griddepcontrol.wait) only before reading the counts.  A gather's source
// rows depend on the tile's ranks alone, so its first loads (two rows of up
// to 2 KiB, or 4 KiB of a longer row, per warp) are in flight during that
// wait; all the CTA's threads then read the counts before its tile.  Counts
// are stored as tile-status words with tag 0, which no look-back ever
// accepts.
constexpr uint32_t kRowsSumTiles = 4096;

__device__ __forceinline__ void wait_for_prerequisite_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependent_grid() { asm volatile("griddepcontrol.launch_dependents;"); }

// The count kernel's CTAs: 1,024 threads, one domain index each, counting
// 1024 / ROWS tiles.  A [65537 x 1024] shuffle (domain 2^17) needs 128 of
// them, one resident wave, where one small CTA per tile (1,024 CTAs) took
// 4.5 us, mostly to dispatch.
constexpr int kCountBlock = 1024;

template <bool ODD, int ROWS>
__global__ void __launch_bounds__(kCountBlock) rows_count_kernel(const __grid_constant__ TileArgs a)
{
    allow_dependent_grid();
    constexpr int WARPS_PER_TILE = ROWS / 32;
    constexpr int TILES = kCountBlock / ROWS;
    __shared__ uint32_t s_count[kCountBlock / 32];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t i = blockIdx.x * static_cast<uint32_t>(kCountBlock) + threadIdx.x;
    uint32_t left[1] = {i >> a.g.R};
    uint32_t right[1] = {i & a.g.rmask};
    dev::cipher_items<ODD, 1>(left, right, a.keys, a.rounds, a.g);
    const uint32_t src = (left[0] << a.g.R) | right[0];
    const bool keep = static_cast<uint64_t>(i) < a.g.domain && src < a.g.n;
    const uint32_t c = __popc(__ballot_sync(kFull, keep));
    if (lane == 0) s_count[warp] = c;
    __syncthreads();
    if (threadIdx.x < static_cast<uint32_t>(TILES)) {
        const uint32_t tile = blockIdx.x * static_cast<uint32_t>(TILES) + threadIdx.x;
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < WARPS_PER_TILE; ++w) total += s_count[threadIdx.x * WARPS_PER_TILE + w];
        if (tile < a.num_tiles) a.status[tile] = total;  // tag 0: never read as a published status
    }
}

template <Mode MODE, bool ODD, int ROWS>
__global__ void __launch_bounds__(kRowBlock) rows_copy_kernel(const __grid_constant__ TileArgs a)
{
    constexpr int WARPS = kRowBlock / 32;
    constexpr int TILE_WARPS = ROWS / 32;
    // a gather's source rows are known before the tile's slots are: its
    // first loads are issued before the wait for the count kernel
    constexpr bool kEarlyLoads = MODE == Mode::Gather;
    __shared__ uint32_t s_counts[TILE_WARPS];
    __shared__ uint32_t s_src[ROWS];
    __shared__ uint32_t s_part[WARPS];
    __shared__ uint32_t s_total;

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t tile = blockIdx.x;
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
        if (lane == 0) s_counts[warp] = __popc(mask);
    }
    __syncthreads();
    // ranks within the tile need only this tile's counts
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int w = 0; w < TILE_WARPS; ++w) {
            const uint32_t c = s_counts[w];
            s_counts[w] = run;
            run += c;
        }
        s_total = run;
    }
    __syncthreads();
    if (keep) s_src[s_counts[warp] + __popc(mask & dev::lanemask_lt())] = src;
    __syncthreads();
    const uint32_t count = s_total;
    const uint32_t chunks = a.elem_bytes / 16u;
    const uint4 *in = static_cast<const uint4 *>(a.in);
    uint4 *out = static_cast<uint4 *>(a.out);
    const bool two_rows = chunks <= 16u * kRowChunkUnroll;
    constexpr int H = kRowChunkUnroll / 2;
    // registers of the first step: two rows of up to 2 KiB, or the first
    // 4 KiB of one longer row
    uint4 v[2][H];
    if (kEarlyLoads) {
        if (two_rows) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t r = warp + static_cast<uint32_t>(h) * WARPS;
                if (r < count) {
                    const uint4 *from = in + static_cast<uint64_t>(s_src[r]) * chunks;
#pragma unroll
                    for (int u = 0; u < H; ++u) {
                        const uint32_t c = static_cast<uint32_t>(u) * 32u + lane;
                        if (c < chunks) v[h][u] = __ldg(from + c);
                    }
                }
            }
        } else if (warp < count) {
            const uint4 *from = in + static_cast<uint64_t>(s_src[warp]) * chunks;
#pragma unroll
            for (int u = 0; u < kRowChunkUnroll; ++u) {
                const uint32_t c = static_cast<uint32_t>(u) * 32u + lane;
                if (c < chunks) v[u / H][u % H] = __ldg(from + c);
            }
        }
    }
    // the counts of the tiles before this one, summed by every thread
    wait_for_prerequisite_grid();
    {
        uint32_t sum = 0;
        for (uint32_t t = threadIdx.x; t < tile; t += kRowBlock) sum += static_cast<uint32_t>(a.status[t]);
        sum = __reduce_add_sync(kFull, sum);
        if (lane == 0) s_part[warp] = sum;
    }
    __syncthreads();
    uint32_t prefix = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) prefix += s_part[w];
    if (prefix + count > a.g.n) {  // impossible; kept as a guard, and nothing is written
        if (threadIdx.x == 0) dev::record_error(a.ws, dev::kErrDeviceBounds, prefix + count - 1u);
        return;
    }
    // row r of the tile (its rank among the kept indices) is slot prefix + r
    if (two_rows) {
        // a warp loads two rows before storing them, so that each lane keeps
        // up to 8 16-byte loads in flight
        for (uint32_t r0 = warp; r0 < count; r0 += 2u * WARPS) {
            uint64_t to_row[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t r = r0 + static_cast<uint32_t>(h) * WARPS;
                const uint32_t rr = r < count ? r : r0;
                const uint64_t from_row = MODE == Mode::Gather ? s_src[rr] : prefix + rr;
                to_row[h] = MODE == Mode::Gather ? prefix + rr : s_src[rr];
                if (kEarlyLoads && r0 == warp) continue;  // loaded before the wait
                const uint4 *from = in + from_row * chunks;
#pragma unroll
                for (int u = 0; u < H; ++u) {
                    const uint32_t c = static_cast<uint32_t>(u) * 32u + lane;
                    if (r < count && c < chunks) v[h][u] = __ldg(from + c);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t r = r0 + static_cast<uint32_t>(h) * WARPS;
                uint4 *to = out + to_row[h] * chunks;
#pragma unroll
                for (int u = 0; u < H; ++u) {
                    const uint32_t c = static_cast<uint32_t>(u) * 32u + lane;
                    if (r < count && c < chunks) to[c] = v[h][u];
                }
            }
        }
        return;
    }
    for (uint32_t r = warp; r < count; r += WARPS) {
        const uint64_t from_row = MODE == Mode::Gather ? s_src[r] : prefix + r;
        const uint64_t to_row = MODE == Mode::Gather ? prefix + r : s_src[r];
        const uint4 *from = in + from_row * chunks;
        uint4 *to = out + to_row * chunks;
        for (uint32_t c0 = 0; c0 < chunks; c0 += 32u * kRowChunkUnroll) {
            const bool preloaded = kEarlyLoads && r == warp && c0 == 0u;
            if (!preloaded) {
#pragma unroll
                for (int u = 0; u < kRowChunkUnroll; ++u) {
                    const uint32_t c = c0 + static_cast<uint32_t>(u) * 32u + lane;
                    if (c < chunks) v[u / H][u % H] = __ldg(from + c);
                }
            }
#pragma unroll
            for (int u = 0; u < kRowChunkUnroll; ++u) {
                const uint32_t c = c0 + static_cast<uint32_t>(u) * 32u + lane;
                if (c < chunks) to[c] = v[u / H][u % H];
            }
        }
    }
}

template <Mode MODE, bool ODD, int ROWS>
cudaError_t launch_two_kernel(const TileArgs &a, cudaStream_t stream)
{
    constexpr uint32_t tiles_per_count_cta = kCountBlock / ROWS;
    rows_count_kernel<ODD, ROWS><<<(a.num_tiles + tiles_per_count_cta - 1) / tiles_per_count_cta, kCountBlock, 0,
                                   stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.num_tiles, 1, 1);
    cfg.blockDim = dim3(kRowBlock, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, rows_copy_kernel<MODE, ODD, ROWS>, a);
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
    const bool odd = (a.g.k & 1u) != 0u;
    if (a.num_tiles <= kRowsSumTiles && (mode == Mode::Gather || mode == Mode::Scatter)) {
        if (mode == Mode::Gather)
            return odd ? launch_two_kernel<Mode::Gather, true, ROWS>(a, stream)
                       : launch_two_kernel<Mode::Gather, false, ROWS>(a, stream);
        return odd ? launch_two_kernel<Mode::Scatter, true, ROWS>(a, stream)
                   : launch_two_kernel<Mode::Scatter, false, ROWS>(a, stream);
    }
    const uint32_t ctas = a.num_tiles < static_cast<uint32_t>(ctas_cached) ? a.num_tiles : ctas_cached;
    const dim3 grid(ctas), block(kRowBlock);
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
