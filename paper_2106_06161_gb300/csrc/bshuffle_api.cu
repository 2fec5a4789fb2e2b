// C ABI of libbshuffle: argument checking, the key schedule, the per-stream
// workspace and the launches.  The data path is entirely on the GPU; this
// file never touches element data.
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include <cuda_runtime.h>

#include "../../include/bshuffle.h"
#include "bshuffle_device.cuh"
#include "bshuffle_internal.h"

namespace {

using bsh::Geometry;
using bsh::Mode;
using bsh::TileArgs;
using bsh::WsHeader;

constexpr uint32_t kKMin = 4;                 // domain floor 2^4 (see bshuffle.h)
constexpr size_t kHeaderBytes = 256;          // header slot, keeps the status array aligned
constexpr uint64_t kMinStatusWords = 4096;

std::atomic<uint64_t> g_timeout_ns{2000000000ull};
std::atomic<int64_t> g_skip_publish{-1};
std::atomic<int> g_strategy{BSHUFFLE_STRATEGY_AUTO};
std::atomic<int> g_pass_timing{0};
// Auto strategy: the staged path from this many input bytes on.
constexpr uint64_t kStagedMinBytes = uint64_t{1} << 28;
// Auto strategy: lengths that are not powers of two take the staged path's
// ranked form for 4- and 8-byte elements (from the same input size), else the
// pipelined single pass.  Measured on GB300 against the pipelined single
// pass: uint64 at 2^25 + 1, 2^26 + 1, 2^27 + 1, 2^28 + 12345: 0.535 / 1.19 /
// 2.17 / 5.09 ms against 0.583 / 1.35 / 2.79 / 5.86 ms; uint32 at
// 2^28 + 12345 and 2^29 + 3: 4.70 / 9.18 ms against 5.52 / 11.24 ms.  With
// 16-byte elements the ranked form lost (7.6 against 6.2 ms at 2^28 + 12345).
bool ranked_by_default(uint32_t elem_bytes) { return elem_bytes == 4 || elem_bytes == 8; }
// Auto strategy: the pipelined single pass from these domain exponents on.
// On smaller domains a launch is all latency, and the plain kernel, without
// the hand-offs between compute warps and look-back warp, finishes first:
// back-to-back calls at n = 2^m + 1 (4, 8 and 16-byte elements, GB300) took
// ~8.2 us plain against ~10.2 us pipelined up to m = 14, and the pipelined
// kernel first won at a 2^18 domain for gathers and indices and at 2^19 for
// the scatter of bshuffle_inverse.
constexpr uint32_t kPipeMinKGather = 18;
constexpr uint32_t kPipeMinKScatter = 19;

// ------------------------------------------------------------------ host math

uint32_t domain_bits_of(uint64_t n)
{
    if (n == 0) return 0;
    uint32_t k = 0;
    while (k < 64 && (uint64_t{1} << k) < n) ++k;
    return k < kKMin ? kKMin : k;
}

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the round-key schedule.
uint64_t splitmix64(uint64_t &state)
{
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void fill_keys(uint64_t seed, uint32_t rounds, uint32_t *keys)
{
    uint64_t state = seed;
    for (uint32_t r = 0; r < rounds; ++r) keys[r] = static_cast<uint32_t>(splitmix64(state));
}

Geometry geometry_of(uint64_t n)
{
    Geometry g{};
    g.n = static_cast<uint32_t>(n);
    g.k = domain_bits_of(n);
    g.L = g.k / 2;
    g.R = g.k - g.L;
    g.lmask = (1u << g.L) - 1u;
    g.rmask = g.R >= 32 ? 0xffffffffu : ((1u << g.R) - 1u);
    g.domain = uint64_t{1} << g.k;
    g.odd_mul = 1u << (31u - g.L);
    g.lift_mul = 1u << g.L;
    return g;
}

// ------------------------------------------------------------------ workspace

struct Workspace {
    void *base = nullptr;
    uint64_t status_words = 0;
    void *aux = nullptr;       // batched plan tables
    size_t aux_bytes = 0;
    void *staged = nullptr;    // staged-path buffers
    size_t staged_bytes = 0;
    cudaEvent_t marks[3] = {};  // per-pass timing of the last permute (when enabled)
    int marks_recorded = 0;     // 0: none, 2: single pass, 3: staged
    WsHeader *header() const { return static_cast<WsHeader *>(base); }
    uint64_t *status() const
    {
        return reinterpret_cast<uint64_t *>(static_cast<char *>(base) + kHeaderBytes);
    }
};

std::mutex g_mutex;
std::map<std::pair<int, uintptr_t>, Workspace> g_workspaces;

// The CUDA error behind the latest BSHUFFLE_ERR_CUDA returned on this thread
// (bshuffle_last_cuda_error).
thread_local int g_last_cuda_error = 0;

int cuda_fail(cudaError_t e)
{
    const cudaError_t pending = cudaGetLastError();  // clears the sticky launch error of this thread
    g_last_cuda_error = static_cast<int>(e != cudaSuccess ? e : (pending != cudaSuccess ? pending : cudaErrorUnknown));
    return BSHUFFLE_ERR_CUDA;
}

// Reads and clears the error word of the allocation-free entry point's
// scratch on `device`, if that scratch has been set up (defined with it below).
int static_take_error(int device, cudaStream_t stream, int *code);

uint64_t round_up_pow2(uint64_t v)
{
    uint64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Returns the stream's workspace with room for `words` tile-status words,
// allocating or growing it (growing synchronises the stream first).
int acquire_workspace(cudaStream_t stream, uint64_t words, Workspace **out)
{
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail(e);
    std::lock_guard<std::mutex> lock(g_mutex);
    Workspace &ws = g_workspaces[{device, reinterpret_cast<uintptr_t>(stream)}];
    if (ws.base != nullptr && ws.status_words >= words) {
        *out = &ws;
        return BSHUFFLE_OK;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return cuda_fail(e);
    if (cap != cudaStreamCaptureStatusNone) return BSHUFFLE_ERR_INVALID;  // allocate before capture

    const uint64_t cap_words = round_up_pow2(words < kMinStatusWords ? kMinStatusWords : words);
    WsHeader keep{};
    keep.tag = 1;
    if (ws.base != nullptr) {
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(e);
        e = cudaMemcpy(&keep, ws.base, sizeof(keep), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e);
        cudaFree(ws.base);
        ws.base = nullptr;
        ws.status_words = 0;
        keep.ticket = 0;
        keep.done = 0;
        keep.batch_ticket = 0;
        keep.batch_done = 0;
        keep.tag = 1;  // the new status array is zeroed: tag 0 never matches
    }
    void *base = nullptr;
    const size_t bytes = kHeaderBytes + cap_words * sizeof(uint64_t);
    e = cudaMalloc(&base, bytes);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaMemsetAsync(base, 0, bytes, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base, &keep, sizeof(keep), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaFree(base);
        return cuda_fail(e);
    }
    ws.base = base;
    ws.status_words = cap_words;
    *out = &ws;
    return BSHUFFLE_OK;
}

// ------------------------------------------------------------------ checks

bool valid_elem(uint32_t elem_bytes)
{
    return elem_bytes == 1 || elem_bytes == 2 || elem_bytes == 4 || elem_bytes == 8 ||
           (elem_bytes != 0 && elem_bytes % 16 == 0);
}

uint32_t align_of(uint32_t elem_bytes) { return elem_bytes < 16 ? elem_bytes : 16; }

int check_buffers(const void *in, const void *out, uint64_t n, uint32_t elem_bytes)
{
    if (in == nullptr || out == nullptr) return BSHUFFLE_ERR_NULL;
    if (elem_bytes != 0 && n > UINT64_MAX / elem_bytes) return BSHUFFLE_ERR_TOO_LARGE;
    const uint64_t bytes = n * elem_bytes;
    const uintptr_t a = reinterpret_cast<uintptr_t>(in), b = reinterpret_cast<uintptr_t>(out);
    const uint32_t al = align_of(elem_bytes);
    if (a % al != 0 || b % al != 0) return BSHUFFLE_ERR_ALIGN;
    if (a < b + bytes && b < a + bytes) return BSHUFFLE_ERR_ALIAS;
    return BSHUFFLE_OK;
}

int check_common(uint64_t n, uint32_t rounds)
{
    if (rounds > BSHUFFLE_MAX_ROUNDS) return BSHUFFLE_ERR_ROUNDS;
    if (n > BSHUFFLE_MAX_N) return BSHUFFLE_ERR_TOO_LARGE;
    return BSHUFFLE_OK;
}

// The workspace's timing events when per-pass timing is on (else null).
cudaEvent_t *timing_marks(Workspace *ws)
{
    if (g_pass_timing.load() == 0) return nullptr;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (ws->marks[0] == nullptr) {
        for (cudaEvent_t &ev : ws->marks)
            if (cudaEventCreate(&ev) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
    }
    return ws->marks;
}

// One fused launch over the whole domain of n.
// Which single-pass kernel run_fused launches for a gather.
enum class FusedKernel { ByStrategy, Plain, Pipelined };

int run_fused(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed, uint32_t rounds,
              Mode mode, void *stream_ptr, FusedKernel which = FusedKernel::ByStrategy)
{
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    TileArgs a{};
    a.in = in;
    a.out = out;
    a.g = geometry_of(n);
    a.rounds = rounds;
    a.elem_bytes = elem_bytes;
    a.skip_publish_tile = g_skip_publish.load();
    a.timeout_ns = g_timeout_ns.load();
    fill_keys(seed, rounds, a.keys);
    const bool rows = (mode == Mode::Gather || mode == Mode::Scatter) && elem_bytes > 16;
    const int strategy = g_strategy.load();
    // n = 2^k: nothing is dropped and the scan is the identity, so by default
    // the scan-free kernels run (same output, no look-back)
    if (which == FusedKernel::ByStrategy && strategy == BSHUFFLE_STRATEGY_AUTO && a.g.domain == n) {
        Workspace *ws = nullptr;
        const int rc = acquire_workspace(stream, 1, &ws);
        if (rc != BSHUFFLE_OK) return rc;
        a.ws = ws->header();
        a.status = ws->status();
        cudaEvent_t *marks = mode == Mode::Gather ? timing_marks(ws) : nullptr;
        if (marks != nullptr && cudaEventRecord(marks[0], stream) != cudaSuccess) return cuda_fail(cudaErrorUnknown);
        const cudaError_t e = bsh::launch_direct(a, mode, elem_bytes, stream);
        if (e != cudaSuccess) return cuda_fail(e);
        if (marks != nullptr) {
            if (cudaEventRecord(marks[1], stream) != cudaSuccess) return cuda_fail(cudaErrorUnknown);
            ws->marks_recorded = 2;
        } else if (mode == Mode::Gather) {
            ws->marks_recorded = 0;
        }
        return BSHUFFLE_OK;
    }
    // the pipelined kernel: on request for every call it serves, and by
    // default for those over domains of at least 2^18 (2^19 for the scatter)
    const bool pipe_by_default = a.g.k >= (mode == Mode::Scatter ? kPipeMinKScatter : kPipeMinKGather);
    const bool pipe = !rows && bsh::pipe_supports(mode, elem_bytes) &&
                      (which == FusedKernel::Pipelined ||
                       (which == FusedKernel::ByStrategy &&
                        (strategy == BSHUFFLE_STRATEGY_PIPELINED ||
                         (strategy == BSHUFFLE_STRATEGY_AUTO && pipe_by_default))));
    const int config = rows ? 0 : bsh::elem_config_for(elem_bytes, mode, rounds);
    const int pipe_config = pipe ? bsh::pipe_config_for(elem_bytes, mode) : 0;
    const uint64_t tile = rows   ? bsh::rows_tile_size(elem_bytes)
                          : pipe ? bsh::pipe_tile_size(elem_bytes, pipe_config)
                                 : bsh::elem_tile_size(config);
    const uint64_t tiles = (a.g.domain + tile - 1) / tile;
    a.num_tiles = static_cast<uint32_t>(tiles);
    Workspace *ws = nullptr;
    const int rc = acquire_workspace(stream, tiles, &ws);
    if (rc != BSHUFFLE_OK) return rc;
    a.ws = ws->header();
    a.status = ws->status();
    cudaEvent_t *marks = mode == Mode::Gather ? timing_marks(ws) : nullptr;
    if (marks != nullptr && cudaEventRecord(marks[0], stream) != cudaSuccess) return cuda_fail(cudaErrorUnknown);
    const cudaError_t e = rows   ? bsh::launch_rows(a, mode, stream)
                          : pipe ? bsh::launch_pipe(a, mode, elem_bytes, pipe_config, stream)
                                 : bsh::launch_elem(a, mode, elem_bytes, config, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    if (marks != nullptr) {
        if (cudaEventRecord(marks[1], stream) != cudaSuccess) return cuda_fail(cudaErrorUnknown);
        ws->marks_recorded = 2;
    } else if (mode == Mode::Gather) {
        ws->marks_recorded = 0;
    }
    return BSHUFFLE_OK;
}

uint32_t ceil_log2(uint64_t v)
{
    uint32_t k = 0;
    while ((uint64_t{1} << k) < v) ++k;
    return k;
}

// Grows the stream's staged buffers to `bytes`.  Returns BSHUFFLE_ERR_CUDA
// (after clearing the CUDA error) if the allocation fails.
int acquire_staged(cudaStream_t stream, Workspace *ws, size_t bytes)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (ws->staged != nullptr && ws->staged_bytes >= bytes) return BSHUFFLE_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return cuda_fail(e);
    if (cap != cudaStreamCaptureStatusNone) return BSHUFFLE_ERR_INVALID;
    if (ws->staged != nullptr) {
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(e);
        cudaFree(ws->staged);
        ws->staged = nullptr;
        ws->staged_bytes = 0;
    }
    const size_t granule = size_t{1} << 26;
    const size_t want = (bytes + granule - 1) / granule * granule;
    void *p = nullptr;
    e = cudaMalloc(&p, want);
    if (e != cudaSuccess) return cuda_fail(e);
    ws->staged = p;
    ws->staged_bytes = want;
    return BSHUFFLE_OK;
}

// The staged path (kernels_staged.cu) for n = 2^k: same output as the fused
// single pass.  Returns BSHUFFLE_ERR_CUDA without launching anything if its
// buffers cannot be allocated.
int run_staged(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed, uint32_t rounds,
               void *stream_ptr, bool inverse = false)
{
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    bsh::StagedArgs a{};
    a.in = in;
    a.out = out;
    a.g = geometry_of(n);
    // n < 2^k: the ranked form (gathers only), buckets are spans of domain indices
    const bool padded = a.g.domain != n;
    if (padded && inverse) return BSHUFFLE_ERR_INVALID;
    a.rounds = rounds;
    fill_keys(seed, rounds, a.keys);
    if (padded) {
        uint32_t shift = 0, sub = 0;
        bsh::staged_rank_shifts(n, a.g.k, elem_bytes, &shift, &sub);
        a.dst_shift = shift;
        a.sub_shift = sub;
        a.num_dst = static_cast<uint32_t>(a.g.domain >> shift);
    } else {
        const uint32_t shift = bsh::staged_window_shift(n, elem_bytes);
        a.dst_shift = shift;
        a.sub_shift = shift;
        a.num_dst = static_cast<uint32_t>((n + (uint64_t{1} << shift) - 1) >> shift);
    }

    // every bucket reserves its whole span: 2^k entries for the ranked form
    const uint64_t entries = padded ? a.g.domain : n;
    auto up = [](size_t v) { return (v + 255) & ~static_cast<size_t>(255); };
    const size_t off_dval = 0;
    const size_t off_dpos = up(off_dval + entries * elem_bytes);
    const size_t off_cursor = up(off_dpos + entries * sizeof(uint32_t));
    const size_t off_base = up(off_cursor + a.num_dst * sizeof(uint32_t));
    const size_t total = up(off_base + a.num_dst * sizeof(uint32_t));

    Workspace *ws = nullptr;
    int rc = acquire_workspace(stream, kMinStatusWords, &ws);
    if (rc != BSHUFFLE_OK) return rc;
    rc = acquire_staged(stream, ws, total);
    if (rc != BSHUFFLE_OK) return rc;
    char *base = static_cast<char *>(ws->staged);
    a.dval = base + off_dval;
    a.dpos = reinterpret_cast<uint32_t *>(base + off_dpos);
    a.dst_cursor = reinterpret_cast<uint32_t *>(base + off_cursor);
    a.bucket_base = reinterpret_cast<uint32_t *>(base + off_base);
    a.ws = ws->header();
    cudaError_t e = cudaMemsetAsync(a.dst_cursor, 0, a.num_dst * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return cuda_fail(e);
    cudaEvent_t *marks = timing_marks(ws);
    e = bsh::launch_staged(a, elem_bytes, inverse, stream, marks);
    if (e != cudaSuccess) return cuda_fail(e);
    ws->marks_recorded = marks != nullptr ? 3 : 0;
    return BSHUFFLE_OK;
}

// The staged path needs n = 2^k (nothing dropped, so the inverse cipher gives
// every element's slot) and 4, 8 or 16-byte elements.
bool staged_eligible(uint64_t n, uint32_t elem_bytes)
{
    return (elem_bytes == 4 || elem_bytes == 8 || elem_bytes == 16) && n >= 2 * bsh::staged_tile_size() &&
           (n & (n - 1)) == 0;
}

// Its ranked form serves the other lengths of the shuffle (not the inverse):
// the slot of a kept domain index is its rank among the kept indices.
bool ranked_eligible(uint64_t n, uint32_t elem_bytes)
{
    return (elem_bytes == 4 || elem_bytes == 8 || elem_bytes == 16) && n >= 2 * bsh::staged_tile_size() &&
           (n & (n - 1)) != 0;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

int bshuffle_version(void) { return 100; }

int bshuffle_domain_bits(uint64_t n, uint32_t *k)
{
    if (k == nullptr) return BSHUFFLE_ERR_NULL;
    if (n > BSHUFFLE_MAX_N) return BSHUFFLE_ERR_TOO_LARGE;
    *k = domain_bits_of(n);
    return BSHUFFLE_OK;
}

int bshuffle_round_keys(uint64_t seed, uint32_t rounds, uint32_t *keys)
{
    if (rounds > BSHUFFLE_MAX_ROUNDS) return BSHUFFLE_ERR_ROUNDS;
    if (keys == nullptr && rounds > 0) return BSHUFFLE_ERR_NULL;
    fill_keys(seed, rounds, keys);
    return BSHUFFLE_OK;
}

int bshuffle_permute(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed, uint32_t rounds,
                     void *stream)
{
    int rc = check_common(n, rounds);
    if (rc != BSHUFFLE_OK) return rc;
    if (!valid_elem(elem_bytes)) return BSHUFFLE_ERR_ELEM;
    if (n == 0) return BSHUFFLE_OK;
    rc = check_buffers(in, out, n, elem_bytes);
    if (rc != BSHUFFLE_OK) return rc;
    const int strategy = g_strategy.load();
    const bool staged =
        (strategy == BSHUFFLE_STRATEGY_STAGED && (staged_eligible(n, elem_bytes) || ranked_eligible(n, elem_bytes))) ||
        (strategy == BSHUFFLE_STRATEGY_AUTO && n * elem_bytes >= kStagedMinBytes &&
         (staged_eligible(n, elem_bytes) || (ranked_by_default(elem_bytes) && ranked_eligible(n, elem_bytes))));
    if (staged) {
        rc = run_staged(in, out, n, elem_bytes, seed, rounds, stream);
        if (rc == BSHUFFLE_OK || strategy == BSHUFFLE_STRATEGY_STAGED) return rc;
        // auto: the staged buffers could not be had; the single pass needs none
    }
    return run_fused(in, out, n, elem_bytes, seed, rounds, Mode::Gather, stream);
}

int bshuffle_inverse(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed, uint32_t rounds,
                     void *stream)
{
    int rc = check_common(n, rounds);
    if (rc != BSHUFFLE_OK) return rc;
    if (!valid_elem(elem_bytes)) return BSHUFFLE_ERR_ELEM;
    if (n == 0) return BSHUFFLE_OK;
    rc = check_buffers(in, out, n, elem_bytes);
    if (rc != BSHUFFLE_OK) return rc;
    const int strategy = g_strategy.load();
    if ((strategy == BSHUFFLE_STRATEGY_AUTO || strategy == BSHUFFLE_STRATEGY_STAGED) &&
        staged_eligible(n, elem_bytes) && (strategy == BSHUFFLE_STRATEGY_STAGED || n * elem_bytes >= kStagedMinBytes)) {
        rc = run_staged(in, out, n, elem_bytes, seed, rounds, stream, true);
        if (rc == BSHUFFLE_OK || strategy == BSHUFFLE_STRATEGY_STAGED) return rc;
        // auto: the staged buffers could not be had; the single pass needs none
    }
    return run_fused(in, out, n, elem_bytes, seed, rounds, Mode::Scatter, stream);
}

int bshuffle_indices(void *out_idx, uint32_t idx_bytes, uint64_t n, uint64_t seed, uint32_t rounds, void *stream)
{
    int rc = check_common(n, rounds);
    if (rc != BSHUFFLE_OK) return rc;
    if (idx_bytes != 4 && idx_bytes != 8) return BSHUFFLE_ERR_ELEM;
    if (n == 0) return BSHUFFLE_OK;
    if (out_idx == nullptr) return BSHUFFLE_ERR_NULL;
    if (reinterpret_cast<uintptr_t>(out_idx) % idx_bytes != 0) return BSHUFFLE_ERR_ALIGN;
    return run_fused(nullptr, out_idx, n, idx_bytes, seed, rounds, idx_bytes == 4 ? Mode::Index32 : Mode::Index64,
                     stream);
}

int bshuffle_batched(const bshuffle_desc *d_descs, uint32_t count, uint32_t elem_bytes, uint32_t rounds, void *stream)
{
    if (rounds > BSHUFFLE_MAX_ROUNDS) return BSHUFFLE_ERR_ROUNDS;
    if (count == 0) return BSHUFFLE_OK;
    if (d_descs == nullptr) return BSHUFFLE_ERR_NULL;
    if (elem_bytes != 1 && elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8 && elem_bytes != 16)
        return BSHUFFLE_ERR_ELEM;
    if (count > (1u << 24)) return BSHUFFLE_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(d_descs) % alignof(bshuffle_desc) != 0) return BSHUFFLE_ERR_ALIGN;
    static_assert(sizeof(bshuffle_desc) == sizeof(bsh::BatchDesc), "descriptor layouts differ");

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace *ws = nullptr;
    int rc = acquire_workspace(s, kMinStatusWords, &ws);
    if (rc != BSHUFFLE_OK) return rc;
    auto up = [](size_t v) { return (v + 255) & ~static_cast<size_t>(255); };
    const size_t plan_off = 0;
    const size_t prefix_off = up(plan_off + sizeof(bsh::BatchPlan) * count);
    const size_t total_off = up(prefix_off + sizeof(uint64_t) * (static_cast<size_t>(count) + 1));
    const size_t ring_off = up(total_off + sizeof(uint64_t));
    const size_t need = ring_off + sizeof(uint64_t) * bsh::batch_ring_words();
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (ws->aux_bytes < need) {
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            cudaError_t e = cudaStreamIsCapturing(s, &cap);
            if (e != cudaSuccess) return cuda_fail(e);
            if (cap != cudaStreamCaptureStatusNone) return BSHUFFLE_ERR_INVALID;
            if (ws->aux != nullptr) {
                e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) return cuda_fail(e);
                cudaFree(ws->aux);
                ws->aux = nullptr;
                ws->aux_bytes = 0;
            }
            const size_t bytes = round_up_pow2(need);
            e = cudaMalloc(&ws->aux, bytes);
            if (e != cudaSuccess) {
                ws->aux = nullptr;
                return cuda_fail(e);
            }
            ws->aux_bytes = bytes;
        }
    }
    char *aux = static_cast<char *>(ws->aux);
    bsh::BatchArgs a{};
    a.descs = reinterpret_cast<const bsh::BatchDesc *>(d_descs);
    a.plan = reinterpret_cast<bsh::BatchPlan *>(aux + plan_off);
    a.tile_prefix = reinterpret_cast<uint64_t *>(aux + prefix_off);
    a.total_tiles = reinterpret_cast<uint64_t *>(aux + total_off);
    a.status = reinterpret_cast<uint64_t *>(aux + ring_off);
    a.count = count;
    a.rounds = rounds;
    a.elem_bytes = elem_bytes;
    a.timeout_ns = g_timeout_ns.load();
    a.skip_publish_tile = g_skip_publish.load();
    a.ws = ws->header();
    const cudaError_t e = bsh::launch_batched(a, s);
    return e == cudaSuccess ? BSHUFFLE_OK : cuda_fail(e);
}

int bshuffle_permute_ablation(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                              uint32_t rounds, int variant, void *stream_ptr)
{
    int rc = check_common(n, rounds);
    if (rc != BSHUFFLE_OK) return rc;
    if (elem_bytes != 4 && elem_bytes != 8 && elem_bytes != 16) return BSHUFFLE_ERR_ELEM;
    if (variant < 0 || variant > 3) return BSHUFFLE_ERR_INVALID;
    if (n == 0) return BSHUFFLE_OK;
    rc = check_buffers(in, out, n, elem_bytes);
    if (rc != BSHUFFLE_OK) return rc;
    if (variant >= 2)
        return run_fused(in, out, n, elem_bytes, seed, rounds, Mode::Gather, stream_ptr,
                         variant == 2 ? FusedKernel::Plain : FusedKernel::Pipelined);

    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    bsh::AblationArgs a{};
    a.in = in;
    a.out = out;
    a.g = geometry_of(n);
    a.rounds = rounds;
    a.timeout_ns = g_timeout_ns.load();
    fill_keys(seed, rounds, a.keys);
    const uint64_t tile = bsh::ablation_tile_size();
    const uint64_t tiles = (a.g.domain + tile - 1) / tile;
    a.num_tiles = static_cast<uint32_t>(tiles);
    auto up = [](size_t v) { return (v + 255) & ~static_cast<size_t>(255); };
    const size_t bytes = variant == 0 ? up(a.g.domain * sizeof(uint32_t)) + up(n * sizeof(uint32_t))
                                      : 2 * up(tiles * sizeof(uint32_t));
    Workspace *ws = nullptr;
    rc = acquire_workspace(stream, tiles, &ws);
    if (rc != BSHUFFLE_OK) return rc;
    rc = acquire_staged(stream, ws, bytes);
    if (rc != BSHUFFLE_OK) return rc;
    char *base = static_cast<char *>(ws->staged);
    if (variant == 0) {
        a.w = reinterpret_cast<uint32_t *>(base);
        a.j = reinterpret_cast<uint32_t *>(base + up(a.g.domain * sizeof(uint32_t)));
    } else {
        a.tile_count = reinterpret_cast<uint32_t *>(base);
        a.tile_prefix = reinterpret_cast<uint32_t *>(base + up(tiles * sizeof(uint32_t)));
    }
    a.ws = ws->header();
    a.status = ws->status();
    const cudaError_t e = bsh::launch_ablation(a, elem_bytes, variant, stream);
    return e == cudaSuccess ? BSHUFFLE_OK : cuda_fail(e);
}

int bshuffle_count_range(uint64_t n, uint64_t seed, uint32_t rounds, uint64_t first, uint64_t end,
                         uint64_t *d_count, void *stream_ptr)
{
    int rc = check_common(n, rounds);
    if (rc != BSHUFFLE_OK) return rc;
    if (d_count == nullptr) return BSHUFFLE_ERR_NULL;
    if (reinterpret_cast<uintptr_t>(d_count) % alignof(uint64_t) != 0) return BSHUFFLE_ERR_ALIGN;
    if (first > end) return BSHUFFLE_ERR_INVALID;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(uint64_t), stream);
    if (e != cudaSuccess) return cuda_fail(e);
    if (n == 0) return BSHUFFLE_OK;
    const Geometry g = geometry_of(n);
    if (end > g.domain) end = g.domain;
    if (first >= end) return BSHUFFLE_OK;
    if (g.domain == n) {
        // n = 2^k: nothing is dropped, the count is the range's length
        e = bsh::launch_store_count(reinterpret_cast<unsigned long long *>(d_count), end - first, stream);
        return e == cudaSuccess ? BSHUFFLE_OK : cuda_fail(e);
    }
    uint32_t keys[BSHUFFLE_MAX_ROUNDS];
    fill_keys(seed, rounds, keys);
    e = bsh::launch_count_range(g, keys, rounds, first, end, reinterpret_cast<unsigned long long *>(d_count),
                                stream);
    return e == cudaSuccess ? BSHUFFLE_OK : cuda_fail(e);
}

int bshuffle_permute_range(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                           uint32_t rounds, uint64_t first, uint64_t end, uint64_t out_capacity, void *stream_ptr)
{
    int rc = check_common(n, rounds);
    if (rc != BSHUFFLE_OK) return rc;
    if (elem_bytes != 1 && elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8 && elem_bytes != 16)
        return BSHUFFLE_ERR_ELEM;
    if (first > end) return BSHUFFLE_ERR_INVALID;
    if (n == 0) return BSHUFFLE_OK;
    const Geometry g = geometry_of(n);
    if (end > g.domain) end = g.domain;
    if (first >= end) return BSHUFFLE_OK;
    if (in == nullptr || out == nullptr) return BSHUFFLE_ERR_NULL;
    const uint32_t al = align_of(elem_bytes);
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(in), b0 = reinterpret_cast<uintptr_t>(out);
    if (a0 % al != 0 || b0 % al != 0) return BSHUFFLE_ERR_ALIGN;
    if (out_capacity == 0) return BSHUFFLE_OK;
    if (out_capacity > n) out_capacity = n;
    if (a0 < b0 + out_capacity * elem_bytes && b0 < a0 + n * elem_bytes) return BSHUFFLE_ERR_ALIAS;

    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    TileArgs a{};
    a.in = in;
    a.out = out;
    a.g = g;
    a.rounds = rounds;
    a.elem_bytes = elem_bytes;
    a.range_first = static_cast<uint32_t>(first);
    a.range_end = end;
    a.range_cap = out_capacity;
    a.skip_publish_tile = g_skip_publish.load();
    a.timeout_ns = g_timeout_ns.load();
    fill_keys(seed, rounds, a.keys);
    // n = 2^k: every index is kept, the scan over the range is the identity,
    // and the scan-free gather serves the range (the workspace only takes its
    // error word)
    const bool direct = g.domain == n && n >= 16 && n <= (uint64_t{1} << 31);
    const uint64_t tile = bsh::elem_tile_size(0);
    const uint64_t tiles = direct ? 1 : (end - first + tile - 1) / tile;
    a.num_tiles = static_cast<uint32_t>(tiles);
    Workspace *ws = nullptr;
    rc = acquire_workspace(stream, tiles, &ws);
    if (rc != BSHUFFLE_OK) return rc;
    a.ws = ws->header();
    a.status = ws->status();
    const cudaError_t e = direct ? bsh::launch_direct_range(a, elem_bytes, stream)
                                 : bsh::launch_permute_range(a, elem_bytes, stream);
    return e == cudaSuccess ? BSHUFFLE_OK : cuda_fail(e);
}

int bshuffle_lcg_params(uint64_t seed, uint64_t n, uint64_t *a, uint64_t *c)
{
    if (a == nullptr || c == nullptr) return BSHUFFLE_ERR_NULL;
    if (n > BSHUFFLE_MAX_N) return BSHUFFLE_ERR_TOO_LARGE;
    const uint32_t k = domain_bits_of(n);
    const uint64_t mask = k >= 64 ? ~uint64_t{0} : ((uint64_t{1} << k) - 1);
    uint64_t state = seed;
    *a = (splitmix64(state) | 1) & mask;
    *c = splitmix64(state) & mask;
    return BSHUFFLE_OK;
}

int bshuffle_permute_lcg(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                         void *stream_ptr)
{
    int rc = check_common(n, 0);
    if (rc != BSHUFFLE_OK) return rc;
    if (elem_bytes != 1 && elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8 && elem_bytes != 16)
        return BSHUFFLE_ERR_ELEM;
    if (n == 0) return BSHUFFLE_OK;
    rc = check_buffers(in, out, n, elem_bytes);
    if (rc != BSHUFFLE_OK) return rc;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    TileArgs a{};
    a.in = in;
    a.out = out;
    a.g = geometry_of(n);
    a.elem_bytes = elem_bytes;
    a.skip_publish_tile = g_skip_publish.load();
    a.timeout_ns = g_timeout_ns.load();
    uint64_t la = 0, lc = 0;
    bshuffle_lcg_params(seed, n, &la, &lc);
    a.lcg_a = static_cast<uint32_t>(la);
    a.lcg_c = static_cast<uint32_t>(lc);
    const uint64_t tile = bsh::elem_tile_size(0);
    const uint64_t tiles = (a.g.domain + tile - 1) / tile;
    a.num_tiles = static_cast<uint32_t>(tiles);
    Workspace *ws = nullptr;
    rc = acquire_workspace(stream, tiles, &ws);
    if (rc != BSHUFFLE_OK) return rc;
    a.ws = ws->header();
    a.status = ws->status();
    const cudaError_t e = bsh::launch_gather_lcg(a, elem_bytes, stream);
    return e == cudaSuccess ? BSHUFFLE_OK : cuda_fail(e);
}

int bshuffle_mc_group_diff(const float *x, uint64_t n, uint64_t n1, uint64_t base_seed, uint32_t count,
                           uint32_t rounds, double *T, void *stream)
{
    if (rounds > BSHUFFLE_MAX_ROUNDS) return BSHUFFLE_ERR_ROUNDS;
    if (n > BSHUFFLE_MAX_N) return BSHUFFLE_ERR_TOO_LARGE;
    if (count == 0) return BSHUFFLE_OK;
    if (x == nullptr || T == nullptr) return BSHUFFLE_ERR_NULL;
    if (n1 == 0 || n1 >= n) return BSHUFFLE_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(x) % alignof(float) != 0 || reinterpret_cast<uintptr_t>(T) % alignof(double) != 0)
        return BSHUFFLE_ERR_ALIGN;
    bsh::McArgs a{};
    a.x = x;
    a.T = T;
    a.g = geometry_of(n);
    a.n1 = static_cast<uint32_t>(n1);
    a.count = count;
    a.rounds = rounds;
    a.base_seed = base_seed;
    const cudaError_t e = bsh::launch_mc(a, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? BSHUFFLE_OK : cuda_fail(e);
}

int bshuffle_shapley_voting(const uint32_t *weights, uint64_t n, uint64_t quota, uint64_t seed0, uint64_t samples,
                            uint32_t rounds, uint64_t *counts, void *stream)
{
    if (rounds > BSHUFFLE_MAX_ROUNDS) return BSHUFFLE_ERR_ROUNDS;
    if (n > BSHUFFLE_MAX_N) return BSHUFFLE_ERR_TOO_LARGE;
    if (n == 0) return BSHUFFLE_OK;
    if (weights == nullptr || counts == nullptr) return BSHUFFLE_ERR_NULL;
    if (reinterpret_cast<uintptr_t>(weights) % 4 != 0 || reinterpret_cast<uintptr_t>(counts) % 8 != 0)
        return BSHUFFLE_ERR_ALIGN;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(counts, 0, n * sizeof(uint64_t), s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (quota == 0 || samples == 0) return BSHUFFLE_OK;
    bsh::ShapleyArgs a{};
    a.w = weights;
    a.counts = counts;
    a.g = geometry_of(n);
    a.quota = quota;
    a.seed0 = seed0;
    a.samples = samples;
    a.rounds = rounds;
    e = bsh::launch_shapley_voting(a, s);
    return e == cudaSuccess ? BSHUFFLE_OK : cuda_fail(e);
}

int bshuffle_random_gather(const void *in, void *out, uint64_t n, uint32_t elem_bytes, void *stream)
{
    if (elem_bytes != 4 && elem_bytes != 8 && elem_bytes != 16) return BSHUFFLE_ERR_ELEM;
    if (n == 0) return BSHUFFLE_OK;
    if (n < 16 || n > (uint64_t{1} << 32) || (n & (n - 1)) != 0) return BSHUFFLE_ERR_INVALID;
    const int rc = check_buffers(in, out, n, elem_bytes);
    if (rc != BSHUFFLE_OK) return rc;
    uint32_t k = 0;
    while ((uint64_t{1} << k) < n) ++k;
    const cudaError_t e = bsh::launch_random_gather(in, out, k, elem_bytes, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? BSHUFFLE_OK : cuda_fail(e);
}

int bshuffle_window_scatter(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint32_t window_log2,
                            void *stream)
{
    if (elem_bytes != 4 && elem_bytes != 8 && elem_bytes != 16) return BSHUFFLE_ERR_ELEM;
    if (n == 0) return BSHUFFLE_OK;
    if (n < 16 || n > (uint64_t{1} << 32) || (n & (n - 1)) != 0) return BSHUFFLE_ERR_INVALID;
    uint32_t k = 0;
    while ((uint64_t{1} << k) < n) ++k;
    if (window_log2 < 4 || window_log2 > k) return BSHUFFLE_ERR_INVALID;
    const int rc = check_buffers(in, out, n, elem_bytes);
    if (rc != BSHUFFLE_OK) return rc;
    const cudaError_t e =
        bsh::launch_window_scatter(in, out, k, window_log2, elem_bytes, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? BSHUFFLE_OK : cuda_fail(e);
}

int bshuffle_kendall_pairs(const uint32_t *perms, uint32_t n, uint64_t num_pairs, uint64_t *out, void *stream)
{
    if (num_pairs == 0) return BSHUFFLE_OK;
    if (perms == nullptr || out == nullptr) return BSHUFFLE_ERR_NULL;
    if (n == 0 || n > bsh::kendall_max_n()) return BSHUFFLE_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(perms) % 4 != 0 || reinterpret_cast<uintptr_t>(out) % 8 != 0)
        return BSHUFFLE_ERR_ALIGN;
    const cudaError_t e = bsh::launch_kendall_pairs(perms, n, num_pairs, out, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? BSHUFFLE_OK : cuda_fail(e);
}

int bshuffle_invert_rows(const uint32_t *idx, uint32_t n, uint64_t rows, uint32_t *sigma, void *stream)
{
    if (rows == 0) return BSHUFFLE_OK;
    if (idx == nullptr || sigma == nullptr) return BSHUFFLE_ERR_NULL;
    if (n == 0) return BSHUFFLE_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(idx) % 4 != 0 || reinterpret_cast<uintptr_t>(sigma) % 4 != 0)
        return BSHUFFLE_ERR_ALIGN;
    const uint64_t a = reinterpret_cast<uintptr_t>(idx), b = reinterpret_cast<uintptr_t>(sigma);
    const uint64_t bytes = rows * n * 4;
    if (a < b + bytes && b < a + bytes) return BSHUFFLE_ERR_ALIAS;
    const cudaError_t e = bsh::launch_invert_rows(idx, n, rows, sigma, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? BSHUFFLE_OK : cuda_fail(e);
}

int bshuffle_get_error(void *stream_ptr)
{
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e);
    int code = BSHUFFLE_OK;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        auto it = g_workspaces.find({device, reinterpret_cast<uintptr_t>(stream)});
        if (it != g_workspaces.end() && it->second.base != nullptr) {
            WsHeader h{};
            e = cudaMemcpy(&h, it->second.base, sizeof(h), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e);
            if (h.error != 0) {
                const size_t off = offsetof(WsHeader, error);
                const size_t len = offsetof(WsHeader, error_info) + sizeof(h.error_info) - off;
                e = cudaMemsetAsync(static_cast<char *>(it->second.base) + off, 0, len, stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
                if (e != cudaSuccess) return cuda_fail(e);
                code = h.error;
            }
        }
    }
    // errors of bshuffle_permute_static on this device (its scratch is per device)
    int static_code = BSHUFFLE_OK;
    const int rc = static_take_error(device, stream, &static_code);
    if (rc != BSHUFFLE_OK) return rc;
    return code != BSHUFFLE_OK ? code : static_code;
}

int bshuffle_last_cuda_error(void) { return g_last_cuda_error; }

const char *bshuffle_cuda_error_name(int error)
{
    return cudaGetErrorName(static_cast<cudaError_t>(error));
}

const char *bshuffle_error_string(int code)
{
    switch (code) {
    case BSHUFFLE_OK: return "success";
    case BSHUFFLE_ERR_NULL: return "a required pointer is NULL";
    case BSHUFFLE_ERR_ELEM: return "unsupported element width (use 1, 2, 4, 8 or a multiple of 16 bytes; indices 4 or 8)";
    case BSHUFFLE_ERR_ROUNDS: return "too many cipher rounds (at most 64)";
    case BSHUFFLE_ERR_TOO_LARGE: return "length above the supported maximum (2^32 - 1 elements)";
    case BSHUFFLE_ERR_ALIAS: return "input and output buffers overlap (the shuffle is not in place)";
    case BSHUFFLE_ERR_ALIGN: return "buffer not aligned to min(element width, 16) bytes";
    case BSHUFFLE_ERR_CUDA: return "a CUDA runtime call failed (no device, launch failure or stream error)";
    case BSHUFFLE_ERR_LOOKBACK_TIMEOUT: return "device: a look-back wait ran past its time limit; output is invalid";
    case BSHUFFLE_ERR_DEVICE_BOUNDS: return "device: an output slot fell outside [0, n); output is invalid";
    case BSHUFFLE_ERR_INVALID: return "invalid argument or state (batch count, or workspace growth during graph capture)";
    default: return "unknown bshuffle error code";
    }
}

int bshuffle_release_workspaces(void)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    int rc = BSHUFFLE_OK;
    for (auto &kv : g_workspaces) {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cudaSetDevice(kv.first.first) != cudaSuccess) rc = BSHUFFLE_ERR_CUDA;
        if (kv.second.base != nullptr && cudaFree(kv.second.base) != cudaSuccess) rc = BSHUFFLE_ERR_CUDA;
        if (kv.second.aux != nullptr && cudaFree(kv.second.aux) != cudaSuccess) rc = BSHUFFLE_ERR_CUDA;
        if (kv.second.staged != nullptr && cudaFree(kv.second.staged) != cudaSuccess) rc = BSHUFFLE_ERR_CUDA;
        for (cudaEvent_t ev : kv.second.marks)
            if (ev != nullptr) cudaEventDestroy(ev);
        cudaSetDevice(cur);
    }
    g_workspaces.clear();
    return rc;
}

int bshuffle_set_strategy(int strategy)
{
    if (strategy != BSHUFFLE_STRATEGY_AUTO && strategy != BSHUFFLE_STRATEGY_SINGLE_PASS &&
        strategy != BSHUFFLE_STRATEGY_STAGED && strategy != BSHUFFLE_STRATEGY_PIPELINED)
        return BSHUFFLE_ERR_INVALID;
    g_strategy.store(strategy);
    return BSHUFFLE_OK;
}

int bshuffle_get_strategy(void) { return g_strategy.load(); }

int bshuffle_tuning_configs(void) { return bsh::kNumElemConfigs; }

int bshuffle_tuning_describe(int config, int *block, int *items, int *rounds_unrolled)
{
    if (config < 0 || config >= bsh::kNumElemConfigs) return BSHUFFLE_ERR_INVALID;
    if (block == nullptr || items == nullptr || rounds_unrolled == nullptr) return BSHUFFLE_ERR_NULL;
    *block = bsh::kElemConfigs[config].block;
    *items = bsh::kElemConfigs[config].items;
    *rounds_unrolled = bsh::kElemConfigs[config].rounds;
    return BSHUFFLE_OK;
}

int bshuffle_tuning_select(uint32_t elem_bytes, int config)
{
    return bsh::select_elem_config(elem_bytes, config) == 0 ? BSHUFFLE_OK : BSHUFFLE_ERR_INVALID;
}

int bshuffle_tuning_selected(uint32_t elem_bytes) { return bsh::selected_elem_config(elem_bytes); }

int bshuffle_kernel_configs(int kernel)
{
    switch (kernel) {
    case BSHUFFLE_KERNEL_SINGLE_PASS: return bsh::kNumElemConfigs;
    case BSHUFFLE_KERNEL_PIPELINED: return bsh::kNumPipeConfigs;
    case BSHUFFLE_KERNEL_BATCHED: return bsh::kNumBatchConfigs;
    default: return BSHUFFLE_ERR_INVALID;
    }
}

int bshuffle_kernel_describe(int kernel, int config, int *threads, int *items, int *ctas_per_sm,
                             int *rounds_unrolled)
{
    const int count = bshuffle_kernel_configs(kernel);
    if (count < 0 || config < 0 || config >= count) return BSHUFFLE_ERR_INVALID;
    if (threads == nullptr || items == nullptr || ctas_per_sm == nullptr || rounds_unrolled == nullptr)
        return BSHUFFLE_ERR_NULL;
    if (kernel == BSHUFFLE_KERNEL_SINGLE_PASS) {
        *threads = bsh::kElemConfigs[config].block;
        *items = bsh::kElemConfigs[config].items;
        *ctas_per_sm = 0;
        *rounds_unrolled = bsh::kElemConfigs[config].rounds;
        return BSHUFFLE_OK;
    }
    const bsh::PipeConfig &c =
        kernel == BSHUFFLE_KERNEL_PIPELINED ? bsh::kPipeConfigs[config] : bsh::kBatchConfigs[config];
    *threads = (c.warps + 1) * 32;
    *items = c.items;
    *ctas_per_sm = c.ctas_per_sm;
    *rounds_unrolled = c.unroll != 0 ? static_cast<int>(BSHUFFLE_DEFAULT_ROUNDS) : 0;
    return BSHUFFLE_OK;
}

int bshuffle_kernel_select(int kernel, uint32_t elem_bytes, int config)
{
    int rc = -1;
    switch (kernel) {
    case BSHUFFLE_KERNEL_SINGLE_PASS: rc = bsh::select_elem_config(elem_bytes, config); break;
    case BSHUFFLE_KERNEL_PIPELINED: rc = bsh::select_pipe_config(elem_bytes, config); break;
    case BSHUFFLE_KERNEL_BATCHED: rc = bsh::select_batch_config(elem_bytes, config); break;
    default: break;
    }
    return rc == 0 ? BSHUFFLE_OK : BSHUFFLE_ERR_INVALID;
}

int bshuffle_kernel_selected(int kernel, uint32_t elem_bytes)
{
    switch (kernel) {
    case BSHUFFLE_KERNEL_SINGLE_PASS: return bsh::selected_elem_config(elem_bytes);
    case BSHUFFLE_KERNEL_PIPELINED: return bsh::selected_pipe_config(elem_bytes);
    case BSHUFFLE_KERNEL_BATCHED: return bsh::selected_batch_config(elem_bytes);
    default: return BSHUFFLE_ERR_INVALID;
    }
}

int bshuffle_set_pass_timing(int on)
{
    g_pass_timing.store(on != 0 ? 1 : 0);
    return BSHUFFLE_OK;
}

int bshuffle_last_pass_ms(void *stream_ptr, float *ms, int capacity)
{
    if (ms == nullptr && capacity > 0) return BSHUFFLE_ERR_NULL;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e);
    std::lock_guard<std::mutex> lock(g_mutex);
    auto it = g_workspaces.find({device, reinterpret_cast<uintptr_t>(stream)});
    if (it == g_workspaces.end() || it->second.marks_recorded < 2) return 0;
    const int passes = it->second.marks_recorded - 1;
    for (int i = 0; i < passes && i < capacity; ++i) {
        e = cudaEventElapsedTime(&ms[i], it->second.marks[i], it->second.marks[i + 1]);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return passes;
}

int bshuffle_set_lookback_timeout_ns(uint64_t ns)
{
    g_timeout_ns.store(ns < 1000000ull ? 1000000ull : ns);
    return BSHUFFLE_OK;
}

int bshuffle_debug_lookback_cycles(void *stream_ptr, uint64_t *lookback_cycles, uint64_t *cta_cycles)
{
    if (lookback_cycles == nullptr || cta_cycles == nullptr) return BSHUFFLE_ERR_NULL;
    *lookback_cycles = 0;
    *cta_cycles = 0;
    if (BSHUFFLE_LOOKBACK_CLOCKS == 0) return BSHUFFLE_ERR_INVALID;  // not a measurement build
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e);
    std::lock_guard<std::mutex> lock(g_mutex);
    auto it = g_workspaces.find({device, reinterpret_cast<uintptr_t>(stream)});
    if (it == g_workspaces.end() || it->second.base == nullptr) return BSHUFFLE_OK;
    WsHeader h{};
    e = cudaMemcpy(&h, it->second.base, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    *lookback_cycles = h.lookback_cycles;
    *cta_cycles = h.cta_cycles;
    const size_t off = offsetof(WsHeader, lookback_cycles);
    e = cudaMemsetAsync(static_cast<char *>(it->second.base) + off, 0, 2 * sizeof(unsigned long long), stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    return e == cudaSuccess ? BSHUFFLE_OK : cuda_fail(e);
}

int bshuffle_debug_skip_publish(int64_t tile)
{
    g_skip_publish.store(tile < 0 ? -1 : tile);
    return BSHUFFLE_OK;
}

}  // extern "C"

// ====================================================================== allocation-free entry point
//
// bshuffle_permute_static runs the same element kernel as bshuffle_permute,
// but its scratch (launch counters, tag, error word and the tile-status
// words) lives in the file-scope device array below instead of a cudaMalloc'd
// per-stream workspace.  It is meant for callers that cannot allocate device
// memory at call time: a process that has already reserved all device memory
// for its own pool (so cudaMalloc would fail), or a latency-critical loop that
// cannot afford the device-wide synchronisation cudaMalloc/cudaFree may
// cause.

namespace {

constexpr uint64_t kStaticTiles = 65536;                       // tile-status words
constexpr uint64_t kStaticMaxN = kStaticTiles * 2048;          // 2^27 elements (2048 per tile)
constexpr size_t kStaticBytes = kHeaderBytes + kStaticTiles * sizeof(uint64_t);  // 512 KiB + 256 B

// Held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void *g_static_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device, set up once per
// device: the symbol's address is looked up with that device current (in
// host code the array's name is only a host-side stand-in) and its launch tag
// is set to 1, so that the zero-initialised status words never read as
// published.
int static_scratch(void **out)
{
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail(e);
    if (device < 0 || device >= kMaxDevices) return BSHUFFLE_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (g_static_addr[device] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e);
        WsHeader h{};
        h.tag = 1;
        e = cudaMemcpy(p, &h, sizeof(h), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e);
        g_static_addr[device] = p;
    }
    *out = g_static_addr[device];
    return BSHUFFLE_OK;
}

int static_take_error(int device, cudaStream_t stream, int *code)
{
    *code = BSHUFFLE_OK;
    if (device < 0 || device >= kMaxDevices) return BSHUFFLE_OK;
    void *p = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mutex);
        p = g_static_addr[device];
    }
    if (p == nullptr) return BSHUFFLE_OK;  // never used on this device
    WsHeader h{};
    cudaError_t e = cudaMemcpy(&h, p, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    if (h.error != 0) {
        const size_t off = offsetof(WsHeader, error);
        const size_t len = offsetof(WsHeader, error_info) + sizeof(h.error_info) - off;
        e = cudaMemsetAsync(static_cast<char *>(p) + off, 0, len, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(e);
        *code = h.error;
    }
    return BSHUFFLE_OK;
}

}  // namespace

extern "C" int bshuffle_permute_static(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                                       uint32_t rounds, void *stream_ptr)
{
    int rc = check_common(n, rounds);
    if (rc != BSHUFFLE_OK) return rc;
    if (elem_bytes != 1 && elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8 && elem_bytes != 16)
        return BSHUFFLE_ERR_ELEM;
    if (n == 0) return BSHUFFLE_OK;
    if (n > kStaticMaxN) return BSHUFFLE_ERR_TOO_LARGE;
    rc = check_buffers(in, out, n, elem_bytes);
    if (rc != BSHUFFLE_OK) return rc;

    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    TileArgs a{};
    a.in = in;
    a.out = out;
    a.g = geometry_of(n);
    a.rounds = rounds;
    a.elem_bytes = elem_bytes;
    a.skip_publish_tile = g_skip_publish.load();
    a.timeout_ns = g_timeout_ns.load();
    fill_keys(seed, rounds, a.keys);
    const uint64_t tile = bsh::elem_tile_size(0);
    const uint64_t tiles = (a.g.domain + tile - 1) / tile;
    if (tiles > kStaticTiles) return BSHUFFLE_ERR_TOO_LARGE;
    a.num_tiles = static_cast<uint32_t>(tiles);

    void *scratch = nullptr;
    rc = static_scratch(&scratch);
    if (rc != BSHUFFLE_OK) return rc;
    a.ws = static_cast<WsHeader *>(scratch);
    a.status = reinterpret_cast<uint64_t *>(static_cast<char *>(scratch) + kHeaderBytes);
    // The tile ticket and the completion counter must start at zero; the
    // status words carry the launch tag and need no clearing.
    cudaError_t e = cudaMemsetAsync(scratch, 0, 2 * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return cuda_fail(e);
    e = bsh::launch_elem(a, Mode::Gather, elem_bytes, 0, stream);
    return e == cudaSuccess ? BSHUFFLE_OK : cuda_fail(e);
}
