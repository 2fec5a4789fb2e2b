// The fused single-pass tile kernel (Algorithm 1 of Sec. 4 fused as in the
// paper's "Bijective2", Sec. 6), shared by the translation units that
// instantiate its configurations.
//
// One CTA owns one tile of BLOCK * ITEMS consecutive domain indices, taken
// from a global ticket so that every predecessor of a tile is already
// running (the look-back never waits on a CTA that has not started).
// Thread t evaluates the indices base + j * BLOCK + t (j < ITEMS): for a fixed
// j a warp covers 32 consecutive indices, so its kept elements land in
// consecutive output slots and its stores coalesce without a shared-memory
// staging step.
//   1. bijection: ITEMS cipher evaluations per thread, in registers;
//   2. gather:    the kept sources are loaded right away (Gather mode), so the
//                 random reads are in flight during the scan and look-back;
//   3. scan:      warp ballots + popc, one warp scans the per-(item, warp)
//                 counts, publishes the tile aggregate and looks back;
//   4. store:     out[prefix + rank] = value (Gather, Index) or
//                 out[source] = in[prefix + rank] (Scatter).
// ROUNDS = 0 reads the round count at run time; ROUNDS > 0 unrolls exactly
// that many rounds (valid only for calls with rounds == ROUNDS).  BIJ selects
// the bijection: VariablePhilox (Sec. 3.2) or the LCG of Sec. 3.1,
// b = (a i + c) mod 2^k with a odd.  RANGE restricts the launch to the domain
// indices [range_first, range_end) (tiles counted from range_first), whose
// kept elements fill out[0 .. count): one part of a shuffle split by domain
// range.
#pragma once

#include <cstdint>

#include "bshuffle_device.cuh"
#include "bshuffle_internal.h"

namespace bsh {
namespace elem {

using dev::kFull;

enum Bijection : int { kVarPhilox = 0, kLcg = 1 };

template <class T>
__device__ __forceinline__ T load_nc(const T *p)
{
    return __ldg(p);
}

template <class T, Mode MODE, bool ODD, int BLOCK, int ITEMS, int ROUNDS, int BIJ = kVarPhilox, bool RANGE = false>
__global__ void __launch_bounds__(BLOCK) elem_tile_kernel(const __grid_constant__ TileArgs a)
{
    constexpr int WARPS = BLOCK / 32;
    constexpr int ENTRIES = ITEMS * WARPS;
    __shared__ dev::TileShared<ENTRIES> st;
    const long long c0 = dev::clock_mark();

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
    const uint32_t base = (RANGE ? a.range_first : 0u) + tile * static_cast<uint32_t>(BLOCK * ITEMS);

    // 1. bijection
    uint32_t left[ITEMS], right[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t i = base + static_cast<uint32_t>(j * BLOCK) + threadIdx.x;
        left[j] = i >> a.g.R;
        right[j] = i & a.g.rmask;
    }
    if constexpr (BIJ == kVarPhilox) {
        if constexpr (ROUNDS > 0)
            dev::cipher_items_fixed<ODD, ITEMS, ROUNDS>(left, right, a.keys, a.g);
        else
            dev::cipher_items<ODD, ITEMS>(left, right, a.keys, a.rounds, a.g);
    }

    uint32_t src[ITEMS];
    bool keep[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t i = base + static_cast<uint32_t>(j * BLOCK) + threadIdx.x;
        if constexpr (BIJ == kLcg) {
            const uint32_t dmask = a.g.k >= 32 ? 0xffffffffu : ((1u << a.g.k) - 1u);
            src[j] = (a.lcg_a * i + a.lcg_c) & dmask;  // mod 2^k of the 32-bit wrap is mod 2^k
        } else {
            src[j] = (left[j] << a.g.R) | right[j];
        }
        if constexpr (RANGE) {  // 64-bit: the last tile of a range may pass 2^32
            const uint64_t i64 = uint64_t{a.range_first} + uint64_t{tile} * (BLOCK * ITEMS) +
                                 static_cast<uint64_t>(j * BLOCK) + threadIdx.x;
            keep[j] = i64 < a.range_end && src[j] < a.g.n;
        } else {
            keep[j] = static_cast<uint64_t>(i) < a.g.domain && src[j] < a.g.n;
        }
    }

    // 2. random reads issued before the scan
    T val[ITEMS];
    if constexpr (MODE == Mode::Gather) {
        const T *in = static_cast<const T *>(a.in);
#pragma unroll
        for (int j = 0; j < ITEMS; ++j)
            if (keep[j]) val[j] = load_nc(in + src[j]);
    }

    // 3. in-tile ranks and the tile's global prefix
    uint32_t mask[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) mask[j] = __ballot_sync(kFull, keep[j]);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) st.counts[j * WARPS + warp] = __popc(mask[j]);
    }
    __syncthreads();
    if (warp == 0)
        dev::tile_scan_lookback<ENTRIES>(st, dev::StatusRing{a.status, ~0ull, 63u, tag}, tile, 0, a.timeout_ns,
                                         a.skip_publish_tile, a.ws);
    __syncthreads();
    const uint32_t prefix = st.prefix;
    const bool ok = st.ok != 0u;

    // 4. compacted output
    if (ok) {
        const uint32_t lt = dev::lanemask_lt();
        // a range's slots end at the caller's output capacity
        uint32_t limit = a.g.n;
        if constexpr (RANGE)
            if (a.range_cap < limit) limit = static_cast<uint32_t>(a.range_cap);
        uint32_t dst[ITEMS];
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            dst[j] = prefix + st.counts[j * WARPS + warp] + __popc(mask[j] & lt);
            if (keep[j] && dst[j] >= limit) {
                dev::record_error(a.ws, dev::kErrDeviceBounds, dst[j]);
                keep[j] = false;
            }
        }
        if constexpr (MODE == Mode::Gather) {
            T *out = static_cast<T *>(a.out);
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if (keep[j]) out[dst[j]] = val[j];
        } else if constexpr (MODE == Mode::Index32 || MODE == Mode::Index64) {
            T *out = static_cast<T *>(a.out);
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if (keep[j]) out[dst[j]] = static_cast<T>(src[j]);
        } else {  // Scatter: coalesced read of slot dst, random write to src
            const T *in = static_cast<const T *>(a.in);
            T *out = static_cast<T *>(a.out);
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if (keep[j]) val[j] = load_nc(in + dst[j]);
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if (keep[j]) out[src[j]] = val[j];
        }
    }
    if (threadIdx.x == 0) {
        dev::clock_add(&a.ws->cta_cycles, c0);
        dev::finish_launch(a.ws, tag, gridDim.x);
    }
}

// Launch one configuration; the caller has checked rounds against ROUNDS.
template <class T, Mode MODE, int BLOCK, int ITEMS, int ROUNDS>
cudaError_t launch_config(const TileArgs &a, cudaStream_t stream)
{
    const dim3 grid(a.num_tiles), block(BLOCK);
    if (a.g.k & 1u)
        elem_tile_kernel<T, MODE, true, BLOCK, ITEMS, ROUNDS><<<grid, block, 0, stream>>>(a);
    else
        elem_tile_kernel<T, MODE, false, BLOCK, ITEMS, ROUNDS><<<grid, block, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace elem
}  // namespace bsh
