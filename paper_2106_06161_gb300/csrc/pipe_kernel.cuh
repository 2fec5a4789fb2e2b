// Pipelined single pass of Algorithm 1 (gather and scatter of 4-, 8- and
// 16-byte elements, and the index output): the same output as the fused tile
// kernel, with the inter-tile look-back taken off the compute warps' path.
//
// In the plain fused kernel every warp of a tile waits while one warp looks
// back, and under a full load of random gathers a look-back takes several
// L2 round trips.  Here a persistent CTA holds NCW compute warps and one
// look-back warp, and the compute warps run one tile ahead of their stores:
//
//   compute warps, iteration i (buffer i % 2): take a ticket, evaluate the
//     bijection, start copying the kept elements X[f(i)] into the buffer
//     with cp.async (one copy group per thread and tile; the index and
//     scatter modes store the image itself), store the keep ballots and
//     publish the tile aggregate (the last compute warp to add its count
//     does it); then store tile i - 1: wait for its rank (look-back warp)
//     and for this thread's own copy group of that tile, and write each
//     element this thread gathered to its slot (scatter: read the element of
//     that slot and write it to the image).
//   look-back warp, tile i: wait for the ballots, form the in-tile offsets,
//     look back, publish the inclusive prefix and hand the prefix to the
//     compute warps.
//
// Tickets stay in order of readiness: a tile's aggregate is published by the
// compute warps right after its ballots, never after another tile's
// look-back, and the compute warps wait for a rank only after that.  The
// smallest unfinished ticket therefore always makes progress.  Every wait is
// bounded.
//
// The kernel template and its launch, shared by the translation units that
// instantiate its shapes (kernels_pipe.cu: the default shape for every mode;
// kernels_pipe_tuned.cu: the other shapes of the gather, for the autotuner).
#pragma once

#include <atomic>
#include <cstdint>
#include <type_traits>

#include "bshuffle_device.cuh"
#include "bshuffle_internal.h"

namespace bsh {
namespace pipe {

using dev::kFull;

template <int NCW, int ITEMS>
struct PipeShared {
    static constexpr int E = NCW * ITEMS;
    uint64_t full[2];            // compute -> look-back: ballots of the buffer's tile written
    uint64_t ranked[2];          // look-back -> compute: offsets and prefix of that tile ready
    unsigned long long aggc[2];  // (compute warps done << 32) | kept count, per buffer
    uint32_t masks[2][E];        // keep ballot per (item, compute warp)
    uint32_t offs[2][E];         // exclusive in-tile offsets
    uint32_t prefix[2];          // exclusive prefix of the tile over all earlier tiles
    uint32_t ok[2];              // look-back finished in time
    uint32_t ticket[2];
    uint32_t tag;
    uint32_t abort;
};

// What a tile buffer holds per domain index: the gathered element (gather),
// the image itself (indices), or the image as a 32-bit target slot (scatter:
// out[f(i_j)] = in[j] reads its element once the tile's ranks are known).
template <class T, Mode MODE>
using PipeSlot = typename std::conditional<MODE == Mode::Scatter, uint32_t, T>::type;

// MINB: resident CTAs per SM the register budget targets; UNROLL: the
// default round count runs fully unrolled (else every count runs in a loop).
// RANGE: Algorithm 1 restricted to the domain indices [range_first,
// range_end) (tiles counted from range_first), writing the range's kept
// elements to out[0 .. count), at most range_cap of them.
template <class T, Mode MODE, bool ODD, int NCW, int ITEMS, int MINB, bool UNROLL, bool RANGE = false>
__global__ void __launch_bounds__((NCW + 1) * 32, MINB) pipe_tile_kernel(const __grid_constant__ TileArgs a)
{
    using S = PipeSlot<T, MODE>;
    constexpr uint32_t NCT = NCW * 32;  // compute threads
    constexpr uint32_t TILE = NCT * ITEMS;
    constexpr int E = NCW * ITEMS;
    __shared__ PipeShared<NCW, ITEMS> sh;
    const long long c_start = dev::clock_mark();
    extern __shared__ __align__(16) unsigned char pipe_dyn[];
    S *vals = reinterpret_cast<S *>(pipe_dyn);  // [2][TILE], natural (item, thread) order

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    // a wait for the other role gets room for one full look-back timeout
    const uint64_t role_limit = 2 * a.timeout_ns + 1000000000ull;
    // slots a range launch may write
    const uint32_t range_limit = RANGE && a.range_cap < a.g.n ? static_cast<uint32_t>(a.range_cap) : a.g.n;

    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            dev::mbar_init(&sh.full[b], NCW);
            dev::mbar_init(&sh.ranked[b], 1);
            sh.aggc[b] = 0ull;
        }
        sh.tag = dev::ld_relaxed_gpu(&a.ws->tag);
        sh.abort = 0u;
    }
    __syncthreads();
    const uint32_t tag = sh.tag;
    const dev::StatusRing ring{a.status, ~0ull, 63u, tag};
    volatile uint32_t *abort = &sh.abort;

    if (warp < NCW) {
        // ---------------------------------------------------------- compute
        const uint32_t ct = threadIdx.x;
        const uint32_t lt = dev::lanemask_lt();
        const T *in = static_cast<const T *>(a.in);
        T *out = static_cast<T *>(a.out);
        for (uint32_t iter = 0;; ++iter) {
            const int b = static_cast<int>(iter & 1u);
            if (ct == 0) sh.ticket[b] = *abort == 0u ? atomicAdd(&a.ws->ticket, 1u) : 0xffffffffu;
            dev::compute_sync(NCT);
            const uint32_t tile = sh.ticket[b];
            const bool stop = tile >= a.num_tiles;
            if (!stop) {
                const uint32_t base = (RANGE ? a.range_first : 0u) + tile * TILE;
                uint32_t left[ITEMS], right[ITEMS];
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) {
                    const uint32_t i = base + static_cast<uint32_t>(j) * NCT + ct;
                    left[j] = i >> a.g.R;
                    right[j] = i & a.g.rmask;
                }
                if constexpr (UNROLL)
                    dev::cipher_items<ODD, ITEMS>(left, right, a.keys, a.rounds, a.g);
                else
                    dev::cipher_items_loop<ODD, ITEMS>(left, right, a.keys, a.rounds, a.g);
                S *buf = vals + static_cast<size_t>(b) * TILE;
                uint32_t count = 0;
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) {
                    const uint32_t i = base + static_cast<uint32_t>(j) * NCT + ct;
                    const uint32_t src = (left[j] << a.g.R) | right[j];
                    bool in_domain;
                    if constexpr (RANGE)
                        in_domain = uint64_t{a.range_first} + uint64_t{tile} * TILE + static_cast<uint32_t>(j) * NCT +
                                        ct <
                                    a.range_end;
                    else
                        in_domain = static_cast<uint64_t>(i) < a.g.domain;
                    const bool keep = in_domain && src < a.g.n;
                    if (keep) {
                        S *slot = buf + static_cast<uint32_t>(j) * NCT + ct;
                        if constexpr (MODE == Mode::Gather)
                            dev::cp_async<sizeof(T)>(slot, in + src);
                        else
                            *slot = static_cast<S>(src);
                    }
                    const uint32_t m = __ballot_sync(kFull, keep);
                    count += __popc(m);
                    if (lane == 0) sh.masks[b][j * NCW + warp] = m;
                }
                if (lane == 0) {
                    const unsigned long long v = atomicAdd(&sh.aggc[b], (1ull << 32) | count);
                    if ((v >> 32) == NCW - 1 && static_cast<int64_t>(tile) != a.skip_publish_tile) {
                        const uint32_t total = static_cast<uint32_t>(v) + count;
                        dev::st_relaxed_gpu(ring.slot(tile), dev::status_word(tag, tile == 0u, total));
                    }
                }
            }
            dev::cp_async_commit();
            __syncwarp();
            if (lane == 0) dev::mbar_arrive(&sh.full[b]);
            if (iter > 0) {
                // store the previous tile (buffer b ^ 1) once it is ranked
                const int pb = b ^ 1;
                const long long w0 = dev::clock_mark();
                const bool ranked = dev::mbar_wait(&sh.ranked[pb], ((iter - 1u) >> 1) & 1u, role_limit, abort);
                if (ct == 0) dev::clock_add(&a.ws->lookback_cycles, w0);  // the compute warps wait on the rank
                if (!ranked) {
                    if (lane == 0) dev::record_error(a.ws, dev::kErrLookbackTimeout, iter);
                    *abort = 1u;
                }
                dev::cp_async_wait_prior();  // this thread's copies of the previous tile have landed
                if (ranked && sh.ok[pb] != 0u) {
                    const S *pbuf = vals + static_cast<size_t>(pb) * TILE;
                    const uint32_t prefix = sh.prefix[pb];
                    if constexpr (MODE == Mode::Scatter) {
                        // coalesced reads of this tile's slots, then the random writes
                        uint32_t target[ITEMS];
                        T val[ITEMS];
#pragma unroll
                        for (int j = 0; j < ITEMS; ++j) {
                            const uint32_t e = static_cast<uint32_t>(j) * NCW + warp;
                            const uint32_t m = sh.masks[pb][e];
                            target[j] = 0xffffffffu;
                            if ((m >> lane) & 1u) {
                                const uint32_t dst = prefix + sh.offs[pb][e] + __popc(m & lt);
                                if (dst < a.g.n) {
                                    target[j] = pbuf[static_cast<uint32_t>(j) * NCT + ct];
                                    val[j] = __ldg(in + dst);
                                } else {
                                    dev::record_error(a.ws, dev::kErrDeviceBounds, dst);
                                }
                            }
                        }
#pragma unroll
                        for (int j = 0; j < ITEMS; ++j)
                            if (target[j] < a.g.n) out[target[j]] = val[j];
                    } else {
#pragma unroll
                        for (int j = 0; j < ITEMS; ++j) {
                            const uint32_t e = static_cast<uint32_t>(j) * NCW + warp;
                            const uint32_t m = sh.masks[pb][e];
                            if ((m >> lane) & 1u) {
                                const uint32_t dst = prefix + sh.offs[pb][e] + __popc(m & lt);
                                if (RANGE ? dst < range_limit : dst < a.g.n)
                                    out[dst] = pbuf[static_cast<uint32_t>(j) * NCT + ct];
                                else dev::record_error(a.ws, dev::kErrDeviceBounds, dst);
                            }
                        }
                    }
                }
            }
            if (stop) break;
        }
        dev::cp_async_wait_all();
    } else {
        // -------------------------------------------------------- look-back
        for (uint32_t iter = 0;; ++iter) {
            const int b = static_cast<int>(iter & 1u);
            const uint32_t parity = (iter >> 1) & 1u;
            // lane 0 waits, so that the warp leaves the loop as one
            bool full = false;
            if (lane == 0) {
                full = dev::mbar_wait(&sh.full[b], parity, role_limit, abort);
                if (!full) {
                    dev::record_error(a.ws, dev::kErrLookbackTimeout, iter);
                    *abort = 1u;
                }
            }
            if (!__shfl_sync(kFull, full, 0)) break;
            (void)dev::mbar_test(&sh.full[b], parity);  // completed phase: every lane acquires it
            const uint32_t tile = sh.ticket[b];
            if (tile >= a.num_tiles) break;
            constexpr int C = (E + 31) / 32;
            uint32_t local[C];
            uint32_t sum = 0;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int e = static_cast<int>(lane) * C + c;
                local[c] = e < E ? static_cast<uint32_t>(__popc(sh.masks[b][e])) : 0u;
                sum += local[c];
            }
            const uint32_t incl = dev::warp_inclusive_scan(sum);
            uint32_t run = incl - sum;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int e = static_cast<int>(lane) * C + c;
                if (e < E) sh.offs[b][e] = run;
                run += local[c];
            }
            const uint32_t aggregate = __shfl_sync(kFull, incl, 31);
            uint32_t prefix = 0;
            bool ok = true;
            if (tile > 0u) {
                prefix = dev::lookback(ring, tile, 0, a.timeout_ns, ok);
                if (lane == 0 && static_cast<int64_t>(tile) != a.skip_publish_tile)
                    dev::st_relaxed_gpu(ring.slot(tile), dev::status_word(tag, true, prefix + aggregate));
                if (lane == 0 && !ok) dev::record_error(a.ws, dev::kErrLookbackTimeout, tile);
            }
            if (lane == 0) {
                sh.prefix[b] = prefix;
                sh.ok[b] = ok ? 1u : 0u;
                sh.aggc[b] = 0ull;
            }
            __syncwarp();
            if (lane == 0) dev::mbar_arrive(&sh.ranked[b]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        dev::clock_add(&a.ws->cta_cycles, c_start);
        dev::finish_launch(a.ws, tag, gridDim.x);
    }
}

// Launch one shape: persistent CTAs, as many as fit on the device (cached
// per device and parity on first use), never more than the tiles.
template <class T, Mode MODE, int NCW, int ITEMS, int MINB, bool UNROLL, bool RANGE = false>
cudaError_t launch_shape(const TileArgs &a, cudaStream_t stream)
{
    constexpr int THREADS = (NCW + 1) * 32;
    constexpr size_t DYN = sizeof(PipeSlot<T, MODE>) * 2 * (NCW * 32 * ITEMS);
    static std::atomic<int> per_sm[64][2];  // CTAs to launch per device and parity, 0 until first use
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    const bool odd = (a.g.k & 1u) != 0u;
    auto kernel = odd ? pipe_tile_kernel<T, MODE, true, NCW, ITEMS, MINB, UNROLL, RANGE>
                      : pipe_tile_kernel<T, MODE, false, NCW, ITEMS, MINB, UNROLL, RANGE>;
    std::atomic<int> &slot = per_sm[device][odd ? 1 : 0];
    int ctas = slot.load(std::memory_order_acquire);
    if (ctas == 0) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(DYN));
        if (e != cudaSuccess) return e;
        int blocks = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, THREADS, DYN);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        ctas = (blocks > 0 ? blocks : 1) * sms;
        slot.store(ctas, std::memory_order_release);
    }
    const uint32_t grid = a.num_tiles < static_cast<uint32_t>(ctas) ? a.num_tiles : static_cast<uint32_t>(ctas);
    kernel<<<grid, THREADS, DYN, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace pipe
}  // namespace bsh
