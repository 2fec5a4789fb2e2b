// Device building blocks of the fused bijective shuffle (sm_103a):
//   * the VariablePhilox round (Sec. 3.2) on 32-bit registers,
//   * the tile-status protocol of single-pass decoupled look-back
//     (Merrill and Garland 2016, the scan the paper fuses in Sec. 4 / Sec. 6),
//   * the in-tile scan of keep flags (Algorithm 1's exclusive scan).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bshuffle_internal.h"

namespace bsh {
namespace dev {

// Philox multiplier M0 of Listing 1 (chosen by Salmon et al.).
constexpr uint64_t kM0 = 0xD2B74407B1CE6E93ull;
constexpr uint32_t kFull = 0xffffffffu;

// Error codes written into WsHeader::error (same values as bshuffle.h).
constexpr int kErrLookbackTimeout = -8;
constexpr int kErrDeviceBounds = -9;

// ------------------------------------------------------------------ cipher

// One VariablePhilox round on the split state (left: L bits, right: R bits).
// The 64-bit product M0 * left supplies F (its high word, XORed with the
// round key and the right half into the new left half, L' = F_k(L) xor R)
// and the bijection B (its low word).  For odd k, G shifts B up one bit and
// moves the top bit b of the old right half (bit L) in underneath, so the new
// right half carries L + 1 bits.
// The right half is never masked between rounds: the next round reads only
// its low L bits (masked into the new left half) and, for odd k, exactly its
// bit L (the funnel shift below), so bits above its width are don't-care.
// The caller masks it once after the last round.
// odd_mul = 2^(31 - L) arrives as a run-time value, so the product
// right * odd_mul (which puts bit L at bit 31) stays a multiply on the FMA
// pipe instead of a shift on the busier ALU pipe (measured: odd-k rounds 17 %
// faster on GB300).
template <bool ODD>
__device__ __forceinline__ void cipher_round(uint32_t &left, uint32_t &right, uint32_t key, uint32_t odd_mul,
                                             uint32_t lmask)
{
    const uint64_t prod = kM0 * static_cast<uint64_t>(left);
    const uint32_t hi = static_cast<uint32_t>(prod >> 32);
    const uint32_t lo = static_cast<uint32_t>(prod);
    const uint32_t new_left = (hi ^ key ^ right) & lmask;
    // odd k: (lo << 1) | bit L of right
    right = ODD ? __funnelshift_l(right * odd_mul, lo, 1u) : lo;
    left = new_left;
}

// The round count of Sec. 3.2 and the library's default.  cipher_items and
// cipher_inverse_items run exactly this many rounds fully unrolled (no loop
// control, keys[r] at fixed offsets: 12 % faster index generation on GB300)
// and any other count in a loop.
constexpr uint32_t kUnrolledRounds = 24;

// ITEMS independent evaluations, rounds outer so that the ITEMS dependency
// chains interleave and each round key is loaded once per thread.
template <bool ODD, int ITEMS>
__device__ __forceinline__ void cipher_items_loop(uint32_t (&left)[ITEMS], uint32_t (&right)[ITEMS],
                                                  const uint32_t *keys, uint32_t rounds, const Geometry &g)
{
    const uint32_t odd_mul = g.odd_mul, lmask = g.lmask, rmask = g.rmask;
    for (uint32_t r = 0; r < rounds; ++r) {
        const uint32_t key = keys[r];
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) cipher_round<ODD>(left[j], right[j], key, odd_mul, lmask);
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) right[j] &= rmask;
}

// The same with the round count fixed at compile time (fully unrolled; keys
// in kernel parameter space become constant-bank operands).
template <bool ODD, int ITEMS, int ROUNDS>
__device__ __forceinline__ void cipher_items_fixed(uint32_t (&left)[ITEMS], uint32_t (&right)[ITEMS],
                                                   const uint32_t *keys, const Geometry &g)
{
    const uint32_t odd_mul = g.odd_mul, lmask = g.lmask, rmask = g.rmask;
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) cipher_round<ODD>(left[j], right[j], keys[r], odd_mul, lmask);
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) right[j] &= rmask;
}

template <bool ODD, int ITEMS>
__device__ __forceinline__ void cipher_items(uint32_t (&left)[ITEMS], uint32_t (&right)[ITEMS],
                                             const uint32_t *keys, uint32_t rounds, const Geometry &g)
{
    if (rounds == kUnrolledRounds)
        cipher_items_fixed<ODD, ITEMS, kUnrolledRounds>(left, right, keys, g);
    else
        cipher_items_loop<ODD, ITEMS>(left, right, keys, rounds, g);
}

// Inverse of M0 modulo 2^64 (Newton's iteration; M0 is odd).
constexpr uint64_t inverse_mod_2_64(uint64_t a)
{
    uint64_t x = a;  // correct to 3 bits: a * a = 1 mod 8 for odd a
    for (int i = 0; i < 5; ++i) x *= 2 - a * x;
    return x;
}
constexpr uint32_t kM0InvLo = static_cast<uint32_t>(inverse_mod_2_64(kM0));
static_assert(static_cast<uint32_t>(kM0) * kM0InvLo == 1u, "M0 inverse");

// One inverse round, following the inversion steps of Sec. 3.2: recover
// (B_k(L), b) from the new right half (G^-1: for odd k the odd bit b sits at
// the bottom and B_k(L) above it), L = B_k^-1(B_k(L)) by multiplying with
// M0^-1 modulo 2^L, and R = F_k(L) xor L' from the recomputed high product
// word.  The left half must be exact; the right half may carry don't-care
// bits above its width (only its low L + 1 bits are read, and the product
// with M0^-1 is masked to L bits), so it is masked once after the last round.
// For odd k the round moves b to bit L with a multiply by lift_mul = 2^L, a
// run-time value, so that it runs on the FMA pipe: with a shift, the ALU pipe
// bound odd-k inverse rounds (measured on GB300: 2.22 -> 1.87 ms per 2^28
// evaluations at k = 29).
template <bool ODD>
__device__ __forceinline__ void cipher_inverse_round(uint32_t &left, uint32_t &right, uint32_t key,
                                                     uint32_t lift_mul, uint32_t lmask)
{
    const uint32_t bl = ODD ? (right >> 1) : right;
    const uint32_t old_left = (bl * kM0InvLo) & lmask;
    const uint32_t hi = __umulhi(static_cast<uint32_t>(kM0), old_left) + static_cast<uint32_t>(kM0 >> 32) * old_left;
    const uint32_t x = left ^ hi ^ key;
    // odd k: R in the low L bits and b (bit 0 of the old right half) at bit L
    right = ODD ? ((x & lmask) | ((right * lift_mul) & ~lmask)) : x;
    left = old_left;
}

// ITEMS independent inverse evaluations, rounds in reverse key order.
template <bool ODD, int ITEMS>
__device__ __forceinline__ void cipher_inverse_items_loop(uint32_t (&left)[ITEMS], uint32_t (&right)[ITEMS],
                                                          const uint32_t *keys, uint32_t rounds, const Geometry &g)
{
    const uint32_t lift_mul = g.lift_mul, lmask = g.lmask;
    for (uint32_t r = rounds; r-- > 0;) {
        const uint32_t key = keys[r];
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) cipher_inverse_round<ODD>(left[j], right[j], key, lift_mul, lmask);
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) right[j] &= g.rmask;
}

template <bool ODD, int ITEMS, int ROUNDS>
__device__ __forceinline__ void cipher_inverse_items_fixed(uint32_t (&left)[ITEMS], uint32_t (&right)[ITEMS],
                                                           const uint32_t *keys, const Geometry &g)
{
#pragma unroll
    for (int r = ROUNDS - 1; r >= 0; --r) {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) cipher_inverse_round<ODD>(left[j], right[j], keys[r], g.lift_mul, g.lmask);
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) right[j] &= g.rmask;
}

template <bool ODD, int ITEMS>
__device__ __forceinline__ void cipher_inverse_items(uint32_t (&left)[ITEMS], uint32_t (&right)[ITEMS],
                                                     const uint32_t *keys, uint32_t rounds, const Geometry &g)
{
    if (rounds == kUnrolledRounds)
        cipher_inverse_items_fixed<ODD, ITEMS, kUnrolledRounds>(left, right, keys, g);
    else
        cipher_inverse_items_loop<ODD, ITEMS>(left, right, keys, rounds, g);
}

// ------------------------------------------------------------------ memory helpers

__device__ __forceinline__ uint64_t ld_relaxed_gpu(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_gpu(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Look-back clocks (a measurement build, off by default): with
// BSHUFFLE_LOOKBACK_CLOCKS=1 the single-pass kernels add the SM clock cycles
// their tiles wait on the look-back, and the cycles their CTAs run, to the
// workspace header, so that the share of time lost to the inter-tile chain
// is measured directly.  Otherwise these helpers compile to nothing.
#ifndef BSHUFFLE_LOOKBACK_CLOCKS
#define BSHUFFLE_LOOKBACK_CLOCKS 0
#endif
constexpr bool kLookbackClocks = BSHUFFLE_LOOKBACK_CLOCKS != 0;

__device__ __forceinline__ long long clock_mark()
{
    if constexpr (kLookbackClocks) return clock64();
    return 0;
}

__device__ __forceinline__ void clock_add(unsigned long long *acc, long long since)
{
    if constexpr (kLookbackClocks) atomicAdd(acc, static_cast<unsigned long long>(clock64() - since));
}

__device__ __forceinline__ void record_error(WsHeader *ws, int code, uint64_t info)
{
    if (atomicCAS(&ws->error, 0, code) == 0)
        atomicExch(reinterpret_cast<unsigned long long *>(&ws->error_info),
                   static_cast<unsigned long long>(info));
}

// ------------------------------------------------------------------ tile status

// A tile-status word: tag (31 bits) | inclusive flag (1 bit) | value (32 bits).
// The tag identifies the launch; a word with another tag reads as "not yet
// published".  value is the tile's aggregate (flag 0) or its inclusive
// prefix (flag 1).
__device__ __forceinline__ uint64_t status_word(uint32_t tag, bool inclusive, uint32_t value)
{
    return (static_cast<uint64_t>(tag) << 33) | (static_cast<uint64_t>(inclusive) << 32) | value;
}

__device__ __forceinline__ uint32_t next_tag(uint32_t tag)
{
    return tag >= 0x7fffffffu ? 1u : tag + 1u;
}

// Round key r of a seed: the low 32 bits of the (r + 1)-th SplitMix64 output
// started from the seed (Steele, Lea, Flood 2014), computed directly from r
// so that every lane can derive its own key.
__device__ __forceinline__ uint32_t splitmix_key(uint64_t seed, uint32_t r)
{
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (static_cast<uint64_t>(r) + 1ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return static_cast<uint32_t>(z ^ (z >> 31));
}

__device__ __forceinline__ uint64_t warp_inclusive_scan64(uint64_t v)
{
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t u = __shfl_up_sync(kFull, v, d);
        if (lane >= static_cast<uint32_t>(d)) v += u;
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t v)
{
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(kFull, v, d);
        if (lane >= static_cast<uint32_t>(d)) v += u;
    }
    return v;
}

// Where the tile-status words of a launch live and how they are tagged.
// Tile q's word is words[q & mask] and carries tag base_tag + (q >> shift).
// A plain launch uses one word per tile (mask = all ones, shift = 63) and the
// launch tag; the persistent batched launch reuses a ring of 2^shift words,
// cleared at the start of the launch, and tags each pass over the ring with
// its generation so that a word left by tile q - 2^shift never reads as
// tile q's.
struct StatusRing {
    uint64_t *words;
    uint64_t mask;
    uint32_t shift;
    uint32_t base_tag;
    __device__ __forceinline__ uint64_t *slot(uint64_t q) const { return words + (q & mask); }
    __device__ __forceinline__ uint32_t tag(uint64_t q) const
    {
        return base_tag + static_cast<uint32_t>(q >> shift);
    }
};

// Decoupled look-back by one warp: the exclusive prefix of tile `tile` over
// the tiles first .. tile-1.  Each pass reads the 32 nearest predecessors,
// waits until all of them are published, sums back to the nearest inclusive
// prefix and stops there, else adds all 32 aggregates and moves on.  A wait
// is bounded: after timeout_ns without progress `ok` is cleared and the
// partial sum is returned.
__device__ __forceinline__ uint32_t lookback(const StatusRing &ring, uint64_t tile, uint64_t first,
                                             uint64_t timeout_ns, bool &ok)
{
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t exclusive = 0;
    int64_t pred = static_cast<int64_t>(tile) - 1;
    uint64_t wait_start = 0;
    bool waiting = false;
    uint32_t backoff = 0;
    uint32_t spins = 0;
    ok = true;
    while (true) {
        const int64_t idx = pred - static_cast<int64_t>(lane);
        bool ready = true;
        uint64_t s = status_word(0u, true, 0u);  // before the first tile: prefix 0
        if (idx >= static_cast<int64_t>(first)) {
            const uint64_t q = static_cast<uint64_t>(idx);
            s = ld_relaxed_gpu(ring.slot(q));
            ready = static_cast<uint32_t>(s >> 33) == ring.tag(q);
        }
        if (__all_sync(kFull, ready)) {
            const uint32_t incl = __ballot_sync(kFull, static_cast<uint32_t>(s >> 32) & 1u);
            uint32_t v = static_cast<uint32_t>(s);
            if (incl != 0u && static_cast<int>(lane) > __ffs(incl) - 1) v = 0u;
            exclusive += __reduce_add_sync(kFull, v);
            if (incl != 0u) break;
            pred -= 32;
            waiting = false;
            backoff = 0;
            continue;
        }
        uint64_t now = 0;
        if (lane == 0) now = global_ns();
        now = __shfl_sync(kFull, now, 0);
        if (!waiting) {
            waiting = true;
            wait_start = now;
        } else if (now - wait_start > timeout_ns || ++spins > (1u << 26)) {
            ok = false;
            break;
        }
        __nanosleep(32u << (backoff < 5u ? backoff : 5u));
        ++backoff;
    }
    return exclusive;
}

// Shared state of one tile.
template <int ENTRIES>
struct TileShared {
    uint32_t counts[ENTRIES];  // per (item, warp) keep counts, then their exclusive offsets
    uint32_t tile;             // this CTA's tile ticket
    uint32_t tag;              // launch tag
    uint32_t prefix;           // exclusive prefix of the tile over all earlier tiles
    uint32_t aggregate;        // kept elements in the tile
    uint32_t ok;               // look-back finished in time
};

// Run by one full warp after every warp has written its counts: exclusive
// scan of the ENTRIES counts in place, publication of the tile aggregate,
// look-back, publication of the inclusive prefix.  Publishing is skipped for
// the tile `skip_tile` (test hook).
template <int ENTRIES>
__device__ __forceinline__ void tile_scan_lookback(TileShared<ENTRIES> &st, const StatusRing &ring, uint64_t tile,
                                                   uint64_t first, uint64_t timeout_ns, int64_t skip_tile,
                                                   WsHeader *ws)
{
    constexpr int C = (ENTRIES + 31) / 32;
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t local[C];
    uint32_t sum = 0;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int e = static_cast<int>(lane) * C + c;
        local[c] = e < ENTRIES ? st.counts[e] : 0u;
        sum += local[c];
    }
    const uint32_t incl = warp_inclusive_scan(sum);
    uint32_t run = incl - sum;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int e = static_cast<int>(lane) * C + c;
        if (e < ENTRIES) st.counts[e] = run;
        run += local[c];
    }
    const uint32_t aggregate = __shfl_sync(kFull, incl, 31);
    const bool publish = static_cast<int64_t>(tile) != skip_tile;
    const uint32_t tag = ring.tag(tile);
    if (lane == 0 && publish) st_relaxed_gpu(ring.slot(tile), status_word(tag, tile == first, aggregate));
    uint32_t exclusive = 0;
    bool ok = true;
    if (tile > first) {
        const long long c0 = clock_mark();
        exclusive = lookback(ring, tile, first, timeout_ns, ok);
        if (lane == 0) clock_add(&ws->lookback_cycles, c0);
        if (lane == 0 && publish) st_relaxed_gpu(ring.slot(tile), status_word(tag, true, exclusive + aggregate));
        if (lane == 0 && !ok) record_error(ws, kErrLookbackTimeout, tile);
    }
    if (lane == 0) {
        st.prefix = exclusive;
        st.aggregate = aggregate;
        st.ok = ok ? 1u : 0u;
    }
}

// Called by one thread per CTA once the CTA no longer reads the header: the
// last CTA of the launch resets the ticket and the counter and advances the
// tag, leaving the header ready for the next launch on the stream.
__device__ __forceinline__ void finish_launch(WsHeader *ws, uint32_t tag, uint32_t ctas)
{
    __threadfence();
    const uint32_t d = atomicAdd(&ws->done, 1u);
    if (d == ctas - 1u) {
        atomicExch(&ws->ticket, 0u);
        atomicExch(&ws->done, 0u);
        atomicExch(&ws->tag, next_tag(tag));
        __threadfence();
    }
}

// ------------------------------------------------------------------ async copies and mbarriers
// Helpers of the pipelined kernels: shared-memory mbarriers, cp.async copies
// global -> shared, and a named barrier over a subset of the CTA's warps.

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile(
        "{\n\t.reg .b64 state;\n\t"
        "mbarrier.arrive.shared.b64 state, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0u;
}

// Waits for the completion of the barrier phase of parity `parity`; gives up
// (false) after `limit_ns` or when another role has raised `abort`.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns,
                                          const volatile uint32_t *abort)
{
    uint64_t start = 0;
    uint32_t spins = 0;
    while (!mbar_test(bar, parity)) {
        if (*abort != 0u) return false;
        const uint64_t now = global_ns();
        if (start == 0) {
            start = now;
        } else if (now - start > limit_ns || ++spins > (1u << 26)) {
            return false;
        }
    }
    return true;
}

// 16-byte copies bypass L1 (.cg): for random 16-byte gathers, allocating in
// L1 made the pipelined kernel 1.57x slower on GB300.  .cg takes 16 bytes
// only, so smaller copies allocate (.ca).
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst_smem, const void *src)
{
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async copies 4, 8 or 16 bytes");
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst_smem)), "l"(src), "n"(BYTES)
                     : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Waits until every copy group of this thread but the most recent one has landed.
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Barrier 1 over the compute warps only.
__device__ __forceinline__ void compute_sync(uint32_t threads)
{
    asm volatile("bar.sync 1, %0;" ::"r"(threads) : "memory");
}

}  // namespace dev
}  // namespace bsh
