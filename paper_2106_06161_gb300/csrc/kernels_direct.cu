// Power-of-two lengths without the scan.  When n = 2^k (k >= 4) the domain is
// exactly [0, n): every image f(i) is below n, nothing is dropped, and the
// exclusive scan of Algorithm 1 (Sec. 4) is the identity, rank(i) = i.  The
// fused kernels' look-back then adds only latency, so these kernels write
//   Gather   out[i] = in[f(i)]        (bshuffle_permute)
//   Scatter  out[f(i)] = in[i]        (bshuffle_inverse)
//   Index    out[i] = f(i)            (bshuffle_indices)
// with the same bijection (Sec. 3.2), hence the same output as every other
// path, and no inter-CTA dependency at all.
//
// Elements of 1 to 16 bytes: each thread evaluates ITEMS indices (rounds
// outer, so the ITEMS cipher chains interleave) and issues all its loads
// before its stores.  Rows (elem_bytes a multiple of 16 above 16): a warp
// owns kRowsPerWarp consecutive rows, evaluates their images in its lanes,
// and copies the rows one after another with 16-byte vectors, up to 8 in
// flight per lane; both sides of every row copy are contiguous.
#include <cstdint>
#include <type_traits>

#include "bshuffle_device.cuh"
#include "bshuffle_internal.h"

namespace bsh {
namespace {

using dev::kFull;

constexpr int kDBlock = 256;
constexpr int kDItems = 8;
constexpr uint32_t kRowsPerWarp = 8;
constexpr int kRowChunkUnroll = 8;

template <bool ODD, int ITEMS>
__device__ __forceinline__ void images(const TileArgs &a, const uint32_t (&i)[ITEMS], uint32_t (&f)[ITEMS])
{
    uint32_t left[ITEMS], right[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        left[j] = i[j] >> a.g.R;
        right[j] = i[j] & a.g.rmask;
    }
    dev::cipher_items<ODD, ITEMS>(left, right, a.keys, a.rounds, a.g);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) f[j] = (left[j] << a.g.R) | right[j];
}

template <class T, Mode MODE, bool ODD>
__global__ void __launch_bounds__(kDBlock) direct_elem_kernel(const __grid_constant__ TileArgs a)
{
    const uint32_t n = a.g.n;  // == 2^k <= 2^31
    const uint32_t base = blockIdx.x * static_cast<uint32_t>(kDBlock * kDItems) + threadIdx.x;
    uint32_t i[kDItems], f[kDItems];
#pragma unroll
    for (int j = 0; j < kDItems; ++j) i[j] = base + static_cast<uint32_t>(j * kDBlock);
    images<ODD, kDItems>(a, i, f);

    if constexpr (MODE == Mode::Index32 || MODE == Mode::Index64) {
        using I = typename std::conditional<MODE == Mode::Index32, uint32_t, unsigned long long>::type;
        I *out = static_cast<I *>(a.out);
#pragma unroll
        for (int j = 0; j < kDItems; ++j)
            if (i[j] < n) out[i[j]] = static_cast<I>(f[j]);
    } else {
        const T *in = static_cast<const T *>(a.in);
        T *out = static_cast<T *>(a.out);
        T v[kDItems];
#pragma unroll
        for (int j = 0; j < kDItems; ++j) {
            if (i[j] < n && f[j] < n) v[j] = MODE == Mode::Gather ? __ldg(in + f[j]) : __ldg(in + i[j]);
        }
#pragma unroll
        for (int j = 0; j < kDItems; ++j) {
            if (i[j] >= n) continue;
            if (f[j] >= n) {  // impossible for a bijection of [0, n); kept as a guard
                dev::record_error(a.ws, dev::kErrDeviceBounds, f[j]);
                continue;
            }
            if (MODE == Mode::Gather) out[i[j]] = v[j];
            else out[f[j]] = v[j];
        }
    }
}

// The gather restricted to the domain range [range_first, range_end) of a
// power-of-two length: every index is kept, so the range's t-th index
// range_first + t fills out[t] (the exclusive scan over the range is the
// identity too).  A slot at or past range_cap is not written and records a
// bounds error.
template <class T, bool ODD>
__global__ void __launch_bounds__(kDBlock) direct_range_kernel(const __grid_constant__ TileArgs a)
{
    const uint32_t n = a.g.n;  // == 2^k <= 2^31
    const uint64_t len = a.range_end - a.range_first;
    const uint64_t t0 = uint64_t{blockIdx.x} * (kDBlock * kDItems) + threadIdx.x;
    uint32_t i[kDItems], f[kDItems];
#pragma unroll
    for (int j = 0; j < kDItems; ++j) {
        const uint64_t t = t0 + static_cast<uint64_t>(j * kDBlock);
        i[j] = t < len ? a.range_first + static_cast<uint32_t>(t) : 0u;
    }
    images<ODD, kDItems>(a, i, f);
    const T *in = static_cast<const T *>(a.in);
    T *out = static_cast<T *>(a.out);
    T v[kDItems];
#pragma unroll
    for (int j = 0; j < kDItems; ++j) {
        const uint64_t t = t0 + static_cast<uint64_t>(j * kDBlock);
        if (t < len && t < a.range_cap && f[j] < n) v[j] = __ldg(in + f[j]);
    }
#pragma unroll
    for (int j = 0; j < kDItems; ++j) {
        const uint64_t t = t0 + static_cast<uint64_t>(j * kDBlock);
        if (t >= len) continue;
        if (t >= a.range_cap || f[j] >= n) {  // f[j] >= n is impossible for a bijection; kept as a guard
            dev::record_error(a.ws, dev::kErrDeviceBounds, t);
            continue;
        }
        out[t] = v[j];
    }
}

template <Mode MODE, bool ODD>
__global__ void __launch_bounds__(kDBlock) direct_rows_kernel(const __grid_constant__ TileArgs a)
{
    const uint32_t n = a.g.n;  // == 2^k >= 16, a multiple of kRowsPerWarp
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = blockIdx.x * static_cast<uint32_t>(kDBlock / 32) + (threadIdx.x >> 5);
    const uint32_t row0 = warp * kRowsPerWarp;
    if (row0 >= n) return;  // the whole warp leaves together
    uint32_t i[1] = {row0 + (lane % kRowsPerWarp)};
    uint32_t f[1];
    images<ODD, 1>(a, i, f);
    if (f[0] >= n) dev::record_error(a.ws, dev::kErrDeviceBounds, f[0]);  // impossible; kept as a guard

    const uint32_t chunks = a.elem_bytes / 16u;
    const uint4 *in = static_cast<const uint4 *>(a.in);
    uint4 *out = static_cast<uint4 *>(a.out);
    if (chunks <= 16u * kRowChunkUnroll) {
        // rows of up to 2 KiB: two rows loaded before they are stored, so
        // that each lane keeps up to 8 16-byte loads in flight
        constexpr int H = kRowChunkUnroll / 2;
        for (uint32_t r = 0; r < kRowsPerWarp; r += 2) {
            uint4 v[2][H];
            uint64_t to_row[2];
            bool live[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t fr = __shfl_sync(kFull, f[0], r + h);
                live[h] = fr < n;
                const uint64_t from_row = MODE == Mode::Gather ? fr : row0 + r + h;
                to_row[h] = MODE == Mode::Gather ? row0 + r + h : fr;
                const uint4 *src = in + from_row * chunks;
#pragma unroll
                for (int u = 0; u < H; ++u) {
                    const uint32_t c = static_cast<uint32_t>(u) * 32u + lane;
                    if (live[h] && c < chunks) v[h][u] = __ldg(src + c);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint4 *dst = out + to_row[h] * chunks;
#pragma unroll
                for (int u = 0; u < H; ++u) {
                    const uint32_t c = static_cast<uint32_t>(u) * 32u + lane;
                    if (live[h] && c < chunks) dst[c] = v[h][u];
                }
            }
        }
        return;
    }
    for (uint32_t r = 0; r < kRowsPerWarp; ++r) {
        const uint32_t fr = __shfl_sync(kFull, f[0], r);
        if (fr >= n) continue;
        const uint64_t from_row = MODE == Mode::Gather ? fr : row0 + r;
        const uint64_t to_row = MODE == Mode::Gather ? row0 + r : fr;
        const uint4 *src = in + from_row * chunks;
        uint4 *dst = out + to_row * chunks;
        for (uint32_t c0 = 0; c0 < chunks; c0 += 32u * kRowChunkUnroll) {
            uint4 v[kRowChunkUnroll];
#pragma unroll
            for (int u = 0; u < kRowChunkUnroll; ++u) {
                const uint32_t c = c0 + static_cast<uint32_t>(u) * 32u + lane;
                if (c < chunks) v[u] = __ldg(src + c);
            }
#pragma unroll
            for (int u = 0; u < kRowChunkUnroll; ++u) {
                const uint32_t c = c0 + static_cast<uint32_t>(u) * 32u + lane;
                if (c < chunks) dst[c] = v[u];
            }
        }
    }
}

template <class T, Mode MODE>
cudaError_t launch_elem_t(const TileArgs &a, cudaStream_t stream)
{
    const uint32_t per_cta = kDBlock * kDItems;
    const dim3 grid((a.g.n + per_cta - 1) / per_cta), block(kDBlock);
    if (a.g.k & 1u) direct_elem_kernel<T, MODE, true><<<grid, block, 0, stream>>>(a);
    else direct_elem_kernel<T, MODE, false><<<grid, block, 0, stream>>>(a);
    return cudaGetLastError();
}

template <Mode MODE>
cudaError_t launch_rows_t(const TileArgs &a, cudaStream_t stream)
{
    const uint32_t rows_per_cta = (kDBlock / 32) * kRowsPerWarp;
    const dim3 grid((a.g.n + rows_per_cta - 1) / rows_per_cta), block(kDBlock);
    if (a.g.k & 1u) direct_rows_kernel<MODE, true><<<grid, block, 0, stream>>>(a);
    else direct_rows_kernel<MODE, false><<<grid, block, 0, stream>>>(a);
    return cudaGetLastError();
}

template <Mode MODE>
cudaError_t launch_by_width(const TileArgs &a, uint32_t elem_bytes, cudaStream_t stream)
{
    switch (elem_bytes) {
    case 1: return launch_elem_t<unsigned char, MODE>(a, stream);
    case 2: return launch_elem_t<unsigned short, MODE>(a, stream);
    case 4: return launch_elem_t<unsigned int, MODE>(a, stream);
    case 8: return launch_elem_t<unsigned long long, MODE>(a, stream);
    case 16: return launch_elem_t<uint4, MODE>(a, stream);
    default: return elem_bytes % 16u == 0 ? launch_rows_t<MODE>(a, stream) : cudaErrorInvalidValue;
    }
}

template <class T>
cudaError_t launch_range_t(const TileArgs &a, cudaStream_t stream)
{
    const uint64_t per_cta = kDBlock * kDItems;
    const uint64_t blocks = (a.range_end - a.range_first + per_cta - 1) / per_cta;
    if (blocks == 0) return cudaSuccess;
    const dim3 grid(static_cast<unsigned>(blocks)), block(kDBlock);
    if (a.g.k & 1u) direct_range_kernel<T, true><<<grid, block, 0, stream>>>(a);
    else direct_range_kernel<T, false><<<grid, block, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_direct_range(const TileArgs &a, uint32_t elem_bytes, cudaStream_t stream)
{
    if (a.g.domain != a.g.n || a.g.n < 16u || a.g.n > (uint64_t{1} << 31) || a.range_end > a.g.domain ||
        a.range_first > a.range_end)
        return cudaErrorInvalidValue;
    switch (elem_bytes) {
    case 1: return launch_range_t<unsigned char>(a, stream);
    case 2: return launch_range_t<unsigned short>(a, stream);
    case 4: return launch_range_t<unsigned int>(a, stream);
    case 8: return launch_range_t<unsigned long long>(a, stream);
    case 16: return launch_range_t<uint4>(a, stream);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_direct(const TileArgs &a, Mode mode, uint32_t elem_bytes, cudaStream_t stream)
{
    if (a.g.domain != a.g.n || a.g.n < 16u) return cudaErrorInvalidValue;
    switch (mode) {
    case Mode::Gather: return launch_by_width<Mode::Gather>(a, elem_bytes, stream);
    case Mode::Scatter: return launch_by_width<Mode::Scatter>(a, elem_bytes, stream);
    case Mode::Index32: return launch_elem_t<unsigned int, Mode::Index32>(a, stream);
    case Mode::Index64: return launch_elem_t<unsigned long long, Mode::Index64>(a, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace bsh
