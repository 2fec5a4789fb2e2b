// Many independent shuffles in one persistent launch.
//
// Every instance t (its own input, output, length n_t and seed) is cut into
// tiles of the same size as the plain element kernel's.  The tiles of all
// instances form one global sequence, instance after instance, handed out by
// a global ticket to a grid of persistent CTAs (a few per SM).  A CTA maps its
// ticket to (instance, tile) by a warp-cooperative search of the tile prefix
// table, derives the instance's round keys from its seed, and runs the same
// fused pipeline as the plain kernel: bijection, gather, in-tile scan, and a
// decoupled look-back that stops at the instance's first tile.  The output of
// each instance is exactly that of a plain call with the same arguments.
//
// A small planning kernel (one CTA) runs first: it validates the descriptors,
// computes every instance's domain exponent and tile count, scans the tile
// counts, and clears the status ring used by the look-back.
#include <atomic>
#include <cstdint>

#include "bshuffle_device.cuh"
#include "bshuffle_internal.h"

namespace bsh {
namespace {

using dev::kFull;

// CTA shape of the persistent kernel (overridable at build time for tuning
// experiments): threads, domain indices per thread, and the resident CTAs
// per SM that the register budget targets for elements of up to 4 bytes
// (8- and 16-byte elements hold more live data and target fewer).
#ifndef BSHUFFLE_BATCH_BLOCK
#define BSHUFFLE_BATCH_BLOCK 256
#endif
#ifndef BSHUFFLE_BATCH_ITEMS
#define BSHUFFLE_BATCH_ITEMS 8
#endif
#ifndef BSHUFFLE_BATCH_MIN_CTAS
#define BSHUFFLE_BATCH_MIN_CTAS 5
#endif
constexpr int kBBlock = BSHUFFLE_BATCH_BLOCK;
constexpr int kBItems = BSHUFFLE_BATCH_ITEMS;
constexpr int kBMinCtas = BSHUFFLE_BATCH_MIN_CTAS;
constexpr int min_ctas_for(unsigned elem_bytes)
{
    return elem_bytes <= 4 ? kBMinCtas : (elem_bytes == 8 ? (kBMinCtas > 3 ? 3 : kBMinCtas) : 2);
}
constexpr uint32_t kTile = kBBlock * kBItems;
constexpr uint32_t kRingShift = 16;
constexpr uint64_t kRingWords = uint64_t{1} << kRingShift;
constexpr int kPlanThreads = 1024;
constexpr int kErrInvalid = -10;
constexpr int kErrAlign = -6;

__device__ __forceinline__ uint32_t domain_bits_dev(uint64_t n)
{
    if (n == 0) return 0;
    const uint32_t k = 64u - static_cast<uint32_t>(__clzll(n - 1));  // ceil(log2 n) for n >= 2
    return n == 1 ? 4u : (k < 4u ? 4u : k);
}

__global__ void __launch_bounds__(kPlanThreads) batch_plan_kernel(const __grid_constant__ BatchArgs a)
{
    __shared__ uint64_t s_sums[kPlanThreads];
    const uint32_t tid = threadIdx.x;
    for (uint64_t w = tid; w < kRingWords; w += kPlanThreads) a.status[w] = 0ull;

    const uint32_t per = (a.count + kPlanThreads - 1) / kPlanThreads;
    const uint32_t begin = tid * per;
    const uint32_t end = begin + per < a.count ? begin + per : a.count;
    uint64_t sum = 0;
    for (uint32_t t = begin; t < end; ++t) {
        const BatchDesc d = a.descs[t];
        uint32_t k = domain_bits_dev(d.n);
        bool bad = false;
        if (d.n > 4294967295ull) {
            dev::record_error(a.ws, kErrInvalid, t);
            bad = true;
        } else if (d.n > 0 && (d.in == nullptr || d.out == nullptr)) {
            dev::record_error(a.ws, kErrInvalid, t);
            bad = true;
        } else if (d.n > 0) {
            const uint64_t al = a.elem_bytes < 16u ? a.elem_bytes : 16u;
            if (reinterpret_cast<uintptr_t>(d.in) % al != 0 || reinterpret_cast<uintptr_t>(d.out) % al != 0) {
                dev::record_error(a.ws, kErrAlign, t);
                bad = true;
            }
        }
        if (bad) k = 0;
        const uint64_t tiles = k == 0 ? 0 : ((uint64_t{1} << k) + a.tile - 1) / a.tile;
        a.plan[t].k = k;
        a.plan[t].tiles = static_cast<uint32_t>(tiles);
        sum += tiles;
    }
    s_sums[tid] = sum;
    __syncthreads();
    // exclusive scan of the per-thread sums (Hillis-Steele over 1024 entries)
    for (int d = 1; d < kPlanThreads; d <<= 1) {
        const uint64_t v = tid >= static_cast<uint32_t>(d) ? s_sums[tid - d] : 0ull;
        __syncthreads();
        s_sums[tid] += v;
        __syncthreads();
    }
    uint64_t run = s_sums[tid] - sum;
    for (uint32_t t = begin; t < end; ++t) {
        a.plan[t].first_tile = run;
        a.tile_prefix[t] = run;
        run += a.plan[t].tiles;
    }
    if (tid == kPlanThreads - 1) {
        uint64_t total = s_sums[tid];
        if (total > 0xfff00000ull) {  // tickets are 32-bit
            dev::record_error(a.ws, kErrInvalid, total);
            total = 0;
        }
        a.tile_prefix[a.count] = total;
        *a.total_tiles = total;
    }
}

// The instance owning global tile g: the largest t in [lo, hi) with
// tile_prefix[t] <= g, given tile_prefix[lo] <= g.  Warp-cooperative.  The
// first probe reads the 32 entries after lo (one coalesced load): a CTA's
// successive tickets are a grid's width apart, so the owner of its next
// ticket is usually among the next few instances.  Wider ranges are then
// split into 32 parts per pass.
__device__ __forceinline__ uint32_t find_instance(const uint64_t *prefix, uint32_t lo, uint32_t hi, uint64_t g)
{
    const uint32_t lane = threadIdx.x & 31u;
    {
        const uint32_t m = lo + lane;
        const bool le = m < hi && prefix[m] <= g;
        const uint32_t ball = __ballot_sync(kFull, le);
        const uint32_t top = 31u - static_cast<uint32_t>(__clz(ball));  // lane 0 always qualifies
        if (top < 31u || lo + 32u >= hi) return lo + top;
        lo += 31u;
    }
    while (hi - lo > 32u) {
        const uint32_t span = hi - lo;
        const uint32_t m = lo + static_cast<uint32_t>((static_cast<uint64_t>(span) * lane) / 32u);
        const bool le = prefix[m] <= g;
        const uint32_t ball = __ballot_sync(kFull, le);
        const int top = 31 - __clz(ball);  // lane 0 always qualifies (prefix[lo] <= g)
        const uint32_t new_lo = lo + static_cast<uint32_t>((static_cast<uint64_t>(span) * top) / 32u);
        const uint32_t new_hi = top == 31 ? hi : lo + static_cast<uint32_t>((static_cast<uint64_t>(span) * (top + 1)) / 32u);
        lo = new_lo;
        hi = new_hi;
    }
    const uint32_t m = lo + lane;
    const bool le = m < hi && prefix[m] <= g;
    const uint32_t ball = __ballot_sync(kFull, le);
    return lo + static_cast<uint32_t>(31 - __clz(ball));
}

struct BatchJob {
    const void *in;
    void *out;
    uint64_t first;  // global index of the instance's first tile
    uint64_t end;    // one past its last tile
    Geometry g;
    uint64_t seed;
    uint32_t instance;
    uint32_t ticket;
};

// CTA state, double-buffered: the job of the CTA's next ticket is resolved
// into one buffer while the tile of the other is still being stored.
template <int ENTRIES>
struct BatchShared {
    dev::TileShared<ENTRIES> st[2];
    uint32_t keys[2][kMaxRounds];
    BatchJob job[2];
};

// Run by one full warp: turns ticket `ticket` into its job (instance,
// geometry, round keys) in buffer `nb`.  `prev` is the job of the CTA's
// previous ticket (null before the first one); a CTA's tickets grow, so the
// owner is `prev`'s instance or a later one.
template <class SH>
__device__ __forceinline__ void resolve_job(const BatchArgs &a, uint32_t ticket, uint64_t total,
                                            const BatchJob *prev, SH &sh, int nb)
{
    const uint32_t lane = threadIdx.x & 31u;
    BatchJob &job = sh.job[nb];
    if (ticket >= total) {
        if (lane == 0) job.ticket = ticket;
        return;
    }
    uint64_t seed;
    if (prev != nullptr && ticket < prev->end) {
        seed = prev->seed;
        if (lane == 0) {
            job = *prev;
            job.ticket = ticket;
        }
    } else {
        const uint32_t lo = prev != nullptr ? prev->instance + 1u : 0u;
        const uint32_t t = find_instance(a.tile_prefix, lo, a.count, ticket);
        const BatchDesc d = a.descs[t];
        const BatchPlan p = a.plan[t];
        seed = d.seed;
        if (lane == 0) {
            const uint32_t k = p.k;
            job.in = d.in;
            job.out = d.out;
            job.first = p.first_tile;
            job.end = p.first_tile + p.tiles;
            job.g.n = static_cast<uint32_t>(d.n);
            job.g.k = k;
            job.g.L = k / 2;
            job.g.R = k - k / 2;
            job.g.lmask = (1u << (k / 2)) - 1u;
            job.g.rmask = (k - k / 2) >= 32 ? 0xffffffffu : ((1u << (k - k / 2)) - 1u);
            job.g.domain = uint64_t{1} << k;
            job.g.odd_mul = 1u << (31u - k / 2);
            job.g.lift_mul = 1u << (k / 2);
            job.seed = d.seed;
            job.instance = t;
            job.ticket = ticket;
        }
    }
    for (uint32_t r = lane; r < a.rounds; r += 32) sh.keys[nb][r] = dev::splitmix_key(seed, r);
}

// One tile of job `b`, then the CTA's next ticket.  The next ticket is taken
// only after the look-back: a CTA that held a ticket while its current tile
// still waited on other tiles would make every later tile wait for it.  Warp
// 1 takes it and resolves it into buffer b ^ 1 while the other warps store.
template <class T, bool ODD, int ITEMS, int ENTRIES>
__device__ __forceinline__ void batch_tile(const BatchArgs &a, const BatchJob &job, BatchShared<ENTRIES> &sh, int b,
                                           const dev::StatusRing &ring, uint64_t total)
{
    constexpr int WARPS = kBBlock / 32;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    const Geometry &g = job.g;
    const uint64_t tile = job.ticket;
    const uint32_t base = static_cast<uint32_t>(tile - job.first) * kTile;
    dev::TileShared<ENTRIES> &st = sh.st[b];

    uint32_t left[ITEMS], right[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t i = base + static_cast<uint32_t>(j * kBBlock) + threadIdx.x;
        left[j] = i >> g.R;
        right[j] = i & g.rmask;
    }
    dev::cipher_items<ODD, ITEMS>(left, right, sh.keys[b], a.rounds, g);
    uint32_t src[ITEMS];
    bool keep[ITEMS];
    T val[ITEMS];
    const T *in = static_cast<const T *>(job.in);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t i = base + static_cast<uint32_t>(j * kBBlock) + threadIdx.x;
        src[j] = (left[j] << g.R) | right[j];
        keep[j] = static_cast<uint64_t>(i) < g.domain && src[j] < g.n;
        if (keep[j]) val[j] = __ldg(in + src[j]);
    }
    uint32_t mask[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) mask[j] = __ballot_sync(kFull, keep[j]);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) st.counts[j * WARPS + warp] = __popc(mask[j]);
    }
    __syncthreads();
    if (warp == 0)
        dev::tile_scan_lookback<ENTRIES>(st, ring, tile, job.first, a.timeout_ns, a.skip_publish_tile, a.ws);
    __syncthreads();
    uint32_t next = 0;
    if (threadIdx.x == 32) next = atomicAdd(&a.ws->batch_ticket, 1u);
    if (st.ok != 0u) {
        const uint32_t prefix = st.prefix;
        const uint32_t lt = dev::lanemask_lt();
        T *out = static_cast<T *>(job.out);
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const uint32_t dst = prefix + st.counts[j * WARPS + warp] + __popc(mask[j] & lt);
            if (keep[j]) {
                if (dst < g.n) out[dst] = val[j];
                else dev::record_error(a.ws, dev::kErrDeviceBounds, dst);
            }
        }
    }
    if (warp == 1) resolve_job(a, __shfl_sync(kFull, next, 0), total, &sh.job[b], sh, b ^ 1);
    __syncthreads();
}

// Persistent CTAs, a few per SM, take tickets in order and only when they
// are ready to start the tile, so the smallest unfinished ticket always
// belongs to a running CTA whose look-back depends only on smaller tickets:
// every wait ends.
template <class T>
__global__ void __launch_bounds__(kBBlock, min_ctas_for(sizeof(T))) batch_tile_kernel(const __grid_constant__ BatchArgs a)
{
    constexpr int ENTRIES = kBItems * (kBBlock / 32);
    __shared__ BatchShared<ENTRIES> sh;
    const dev::StatusRing ring{a.status, kRingWords - 1, kRingShift, 1u};
    const uint64_t total = *reinterpret_cast<volatile const uint64_t *>(a.total_tiles);
    const uint32_t warp = threadIdx.x >> 5;

    if (warp == 1) {
        uint32_t t0 = 0;
        if ((threadIdx.x & 31u) == 0) t0 = atomicAdd(&a.ws->batch_ticket, 1u);
        resolve_job(a, __shfl_sync(kFull, t0, 0), total, nullptr, sh, 0);
    }
    __syncthreads();
    for (int b = 0;; b ^= 1) {
        const BatchJob job = sh.job[b];
        if (job.ticket >= total) break;
        if (job.g.k & 1u)
            batch_tile<T, true, kBItems, ENTRIES>(a, job, sh, b, ring, total);
        else
            batch_tile<T, false, kBItems, ENTRIES>(a, job, sh, b, ring, total);
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t d = atomicAdd(&a.ws->batch_done, 1u);
        if (d == gridDim.x - 1u) {
            atomicExch(&a.ws->batch_ticket, 0u);
            atomicExch(&a.ws->batch_done, 0u);
            __threadfence();
        }
    }
}

// ------------------------------------------------------------------ pipelined
// The batched shuffle with the look-back taken off the compute warps (the
// schedule of kernels_pipe.cu): eight compute warps evaluate the bijection of
// tile i, copy its kept elements into a shared buffer with cp.async and
// publish its aggregate, then store tile i - 1 once a ninth warp has ranked
// it (look-back bounded by the instance's first tile).  After its stores,
// warp 0 takes the next ticket and resolves its instance.  Tickets are taken
// only when the CTA no longer waits on other tiles, and aggregates never wait
// on a look-back.  Used for 4-, 8- and 16-byte elements.
// Shapes (kBatchConfigs): NW compute warps of ITEMS indices per thread, MINB
// resident CTAs per SM targeted, UNROLL the default 24 rounds unrolled.
// Shape 0 (8 x 8, 3 CTAs per SM) is the default.
template <int E>
struct BatchPipeShared {
    uint64_t full[2];            // compute -> look-back: ballots of the buffer's tile written
    uint64_t ranked[2];          // look-back -> compute: offsets and prefix ready
    unsigned long long aggc[2];  // (compute warps done << 32) | kept count
    BatchJob job[2];
    uint32_t keys[2][kMaxRounds];
    uint32_t masks[2][E];
    uint32_t offs[2][E];
    uint32_t prefix[2];
    uint32_t ok[2];
    uint32_t abort;
};

template <class T, int NW, int ITEMS, int MINB, bool UNROLL>
__global__ void __launch_bounds__((NW + 1) * 32, MINB) batch_pipe_kernel(const __grid_constant__ BatchArgs a)
{
    constexpr int kPipeWarps = NW;
    constexpr int kPipeItems = ITEMS;
    constexpr uint32_t kPTile = NW * 32 * ITEMS;
    constexpr uint32_t NCT = kPipeWarps * 32;
    constexpr int E = NW * ITEMS;
    __shared__ BatchPipeShared<E> sh;
    extern __shared__ __align__(16) unsigned char batch_dyn[];
    T *vals = reinterpret_cast<T *>(batch_dyn);  // [2][kPTile]
    const dev::StatusRing ring{a.status, kRingWords - 1, kRingShift, 1u};
    const uint64_t total = *reinterpret_cast<volatile const uint64_t *>(a.total_tiles);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    const uint64_t role_limit = 2 * a.timeout_ns + 1000000000ull;
    volatile uint32_t *abort = &sh.abort;

    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            dev::mbar_init(&sh.full[b], kPipeWarps);
            dev::mbar_init(&sh.ranked[b], 1);
            sh.aggc[b] = 0ull;
        }
        sh.abort = 0u;
    }
    if (warp == 0) {
        uint32_t t0 = 0;
        if (lane == 0) t0 = atomicAdd(&a.ws->batch_ticket, 1u);
        resolve_job(a, __shfl_sync(kFull, t0, 0), total, nullptr, sh, 0);
    }
    __syncthreads();

    if (warp < kPipeWarps) {
        // ---------------------------------------------------------- compute
        const uint32_t ct = threadIdx.x;
        const uint32_t lt = dev::lanemask_lt();
        T *prev_out = nullptr;  // the previous tile's output and length
        uint32_t prev_n = 0;
        for (uint32_t iter = 0;; ++iter) {
            const int b = static_cast<int>(iter & 1u);
            const int pb = b ^ 1;
            const BatchJob job = sh.job[b];
            const uint32_t tile = job.ticket;
            const bool stop = tile >= total;
            if (!stop) {
                const Geometry &g = job.g;
                const uint32_t base = (tile - static_cast<uint32_t>(job.first)) * kPTile;
                uint32_t left[kPipeItems], right[kPipeItems];
#pragma unroll
                for (int j = 0; j < kPipeItems; ++j) {
                    const uint32_t i = base + static_cast<uint32_t>(j) * NCT + ct;
                    left[j] = i >> g.R;
                    right[j] = i & g.rmask;
                }
                if constexpr (UNROLL) {
                    if (g.k & 1u)
                        dev::cipher_items<true, kPipeItems>(left, right, sh.keys[b], a.rounds, g);
                    else
                        dev::cipher_items<false, kPipeItems>(left, right, sh.keys[b], a.rounds, g);
                } else {
                    if (g.k & 1u)
                        dev::cipher_items_loop<true, kPipeItems>(left, right, sh.keys[b], a.rounds, g);
                    else
                        dev::cipher_items_loop<false, kPipeItems>(left, right, sh.keys[b], a.rounds, g);
                }
                const T *in = static_cast<const T *>(job.in);
                T *buf = vals + static_cast<size_t>(b) * kPTile;
                uint32_t count = 0;
#pragma unroll
                for (int j = 0; j < kPipeItems; ++j) {
                    const uint32_t i = base + static_cast<uint32_t>(j) * NCT + ct;
                    const uint32_t src = (left[j] << g.R) | right[j];
                    const bool keep = static_cast<uint64_t>(i) < g.domain && src < g.n;
                    if (keep) dev::cp_async<sizeof(T)>(buf + static_cast<uint32_t>(j) * NCT + ct, in + src);
                    const uint32_t m = __ballot_sync(kFull, keep);
                    count += __popc(m);
                    if (lane == 0) sh.masks[b][j * kPipeWarps + warp] = m;
                }
                if (lane == 0) {
                    const unsigned long long v = atomicAdd(&sh.aggc[b], (1ull << 32) | count);
                    if ((v >> 32) == kPipeWarps - 1 && static_cast<int64_t>(tile) != a.skip_publish_tile) {
                        const uint32_t sum = static_cast<uint32_t>(v) + count;
                        dev::st_relaxed_gpu(ring.slot(tile), dev::status_word(ring.tag(tile), tile == job.first, sum));
                    }
                }
            }
            dev::cp_async_commit();
            __syncwarp();
            if (lane == 0) dev::mbar_arrive(&sh.full[b]);
            uint32_t next = 0xffffffffu;
            if (iter > 0) {
                const bool ranked = dev::mbar_wait(&sh.ranked[pb], ((iter - 1u) >> 1) & 1u, role_limit, abort);
                if (!ranked) {
                    if (lane == 0) dev::record_error(a.ws, dev::kErrLookbackTimeout, iter);
                    *abort = 1u;
                }
                // the previous tile's look-back is over: take the next ticket now
                if (ct == 0 && !stop && *abort == 0u) next = atomicAdd(&a.ws->batch_ticket, 1u);
                dev::cp_async_wait_prior();
                if (ranked && sh.ok[pb] != 0u) {
                    const T *pbuf = vals + static_cast<size_t>(pb) * kPTile;
                    const uint32_t prefix = sh.prefix[pb];
#pragma unroll
                    for (int j = 0; j < kPipeItems; ++j) {
                        const uint32_t e = static_cast<uint32_t>(j) * kPipeWarps + warp;
                        const uint32_t m = sh.masks[pb][e];
                        if ((m >> lane) & 1u) {
                            const uint32_t dst = prefix + sh.offs[pb][e] + __popc(m & lt);
                            if (dst < prev_n) prev_out[dst] = pbuf[static_cast<uint32_t>(j) * NCT + ct];
                            else dev::record_error(a.ws, dev::kErrDeviceBounds, dst);
                        }
                    }
                }
            } else if (ct == 0 && !stop) {
                next = atomicAdd(&a.ws->batch_ticket, 1u);
            }
            if (stop) break;
            prev_out = static_cast<T *>(job.out);
            prev_n = job.g.n;
            if (warp == 0) resolve_job(a, __shfl_sync(kFull, next, 0), total, &sh.job[b], sh, pb);
            dev::compute_sync(NCT);
        }
        dev::cp_async_wait_all();
    } else {
        // -------------------------------------------------------- look-back
        for (uint32_t iter = 0;; ++iter) {
            const int b = static_cast<int>(iter & 1u);
            const uint32_t parity = (iter >> 1) & 1u;
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
            const uint32_t tile = sh.job[b].ticket;
            if (tile >= total) break;
            const uint64_t first = sh.job[b].first;
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
            if (tile > first) {
                prefix = dev::lookback(ring, tile, first, a.timeout_ns, ok);
                if (lane == 0 && static_cast<int64_t>(tile) != a.skip_publish_tile)
                    dev::st_relaxed_gpu(ring.slot(tile), dev::status_word(ring.tag(tile), true, prefix + aggregate));
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
        __threadfence();
        const uint32_t d = atomicAdd(&a.ws->batch_done, 1u);
        if (d == gridDim.x - 1u) {
            atomicExch(&a.ws->batch_ticket, 0u);
            atomicExch(&a.ws->batch_done, 0u);
            __threadfence();
        }
    }
}

template <class T, int NW, int ITEMS, int MINB, bool UNROLL>
cudaError_t launch_pipe_typed(const BatchArgs &a, cudaStream_t stream)
{
    constexpr int THREADS = (NW + 1) * 32;
    constexpr uint32_t TILE = NW * 32 * ITEMS;
    constexpr size_t DYN = 2 * sizeof(T) * TILE;
    const auto kernel = batch_pipe_kernel<T, NW, ITEMS, MINB, UNROLL>;
    static std::atomic<int> per_sm[64];  // CTAs to launch per device, 0 until first use
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    int ctas_cached = per_sm[device].load(std::memory_order_acquire);
    if (ctas_cached == 0) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(DYN));
        if (e != cudaSuccess) return e;
        int blocks = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, THREADS, DYN);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        ctas_cached = (blocks > 0 ? blocks : 1) * sms;
        per_sm[device].store(ctas_cached, std::memory_order_release);
    }
    BatchArgs b = a;
    b.grid = static_cast<uint32_t>(ctas_cached);
    b.tile = TILE;
    batch_plan_kernel<<<1, kPlanThreads, 0, stream>>>(b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kernel<<<b.grid, THREADS, DYN, stream>>>(b);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_typed(const BatchArgs &a, cudaStream_t stream)
{
    static std::atomic<int> per_sm[64];  // CTAs to launch per device, 0 until first use
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    int ctas_cached = per_sm[device].load(std::memory_order_acquire);
    if (ctas_cached == 0) {
        int blocks = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, batch_tile_kernel<T>, kBBlock, 0);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        ctas_cached = (blocks > 0 ? blocks : 1) * sms;
        per_sm[device].store(ctas_cached, std::memory_order_release);
    }
    BatchArgs b = a;
    b.grid = static_cast<uint32_t>(ctas_cached);
    b.tile = kTile;
    batch_plan_kernel<<<1, kPlanThreads, 0, stream>>>(b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batch_tile_kernel<T><<<b.grid, kBBlock, 0, stream>>>(b);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_pipe_config(const BatchArgs &a, int config, cudaStream_t stream)
{
    static_assert(kNumBatchConfigs == 6, "shapes instantiated here");
    switch (config) {
    case 0: return launch_pipe_typed<T, 8, 8, 3, true>(a, stream);
    case 1: return launch_pipe_typed<T, 8, 4, 4, true>(a, stream);
    case 2: return launch_pipe_typed<T, 8, 16, 2, true>(a, stream);
    case 3: return launch_pipe_typed<T, 4, 8, 5, true>(a, stream);
    case 4: return launch_pipe_typed<T, 16, 4, 2, true>(a, stream);
    case 5: return launch_pipe_typed<T, 8, 8, 3, false>(a, stream);
    default: return cudaErrorInvalidValue;
    }
}

std::atomic<int> g_batch_selected[3];  // 4, 8, 16 bytes

int batch_slot(uint32_t elem_bytes) { return elem_bytes == 4 ? 0 : elem_bytes == 8 ? 1 : elem_bytes == 16 ? 2 : -1; }

}  // namespace

const PipeConfig kBatchConfigs[kNumBatchConfigs] = {
    {8, 8, 3, 1}, {8, 4, 4, 1}, {8, 16, 2, 1}, {4, 8, 5, 1}, {16, 4, 2, 1}, {8, 8, 3, 0},
};

int select_batch_config(uint32_t elem_bytes, int config)
{
    const int slot = batch_slot(elem_bytes);
    if (slot < 0 || config < 0 || config >= kNumBatchConfigs) return -1;
    g_batch_selected[slot].store(config);
    return 0;
}

int selected_batch_config(uint32_t elem_bytes)
{
    const int slot = batch_slot(elem_bytes);
    return slot < 0 ? 0 : g_batch_selected[slot].load();
}

uint64_t batch_ring_words() { return kRingWords; }

cudaError_t launch_batched(const BatchArgs &a, cudaStream_t stream)
{
    const int config = selected_batch_config(a.elem_bytes);
    switch (a.elem_bytes) {
    case 1: return launch_typed<unsigned char>(a, stream);
    case 2: return launch_typed<unsigned short>(a, stream);
    case 4: return launch_pipe_config<unsigned int>(a, config, stream);
    case 8: return launch_pipe_config<unsigned long long>(a, config, stream);
    case 16: return launch_pipe_config<uint4>(a, config, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bsh
