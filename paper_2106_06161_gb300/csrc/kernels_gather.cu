// Measurement kernels.  Random gather: out[i] = in[h(i)] for a cheap bijection h
// of [0, 2^k).  It has no cipher rounds, no keep test and no scan, so it
// measures the throughput bound the paper sets for any shuffle (the "Gather"
// column of Tables 1 and 2; Sec. 2.2 argues a shuffle cannot beat a random
// gather).  h is three rounds of (multiply by an odd constant mod 2^k, then
// xor with the value shifted right by k/2), each a bijection of k-bit values.
//
// Window scatter: out[w * 2^m + h_m(i - w * 2^m)] = in[i] for the window
// w = i >> m, with h_m the same bijection on m bits.  Sequential reads and
// random writes confined to 2^m-element windows: the access pattern of the
// staged path's second pass without its bucket bookkeeping, so it measures
// the L2's rate of random writes into a resident window.
#include <cstdint>

#include "bshuffle_internal.h"

namespace bsh {
namespace {

constexpr int kGBlock = 256;
constexpr int kGItems = 8;

__device__ __forceinline__ uint32_t scramble(uint32_t x, uint32_t k, uint32_t mask)
{
    const uint32_t half = k / 2u;
    x = (x * 0x9E3779B1u) & mask;
    x ^= x >> half;
    x = (x * 0x85EBCA77u) & mask;
    x ^= x >> half;
    x = (x * 0xC2B2AE3Du) & mask;
    x ^= x >> half;
    return x;
}

template <class T>
__global__ void __launch_bounds__(kGBlock) random_gather_kernel(const T *__restrict__ in, T *__restrict__ out,
                                                                uint32_t k, uint64_t n)
{
    const uint32_t mask = k >= 32 ? 0xffffffffu : ((1u << k) - 1u);
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * (kGBlock * kGItems) + threadIdx.x;
    T v[kGItems];
#pragma unroll
    for (int j = 0; j < kGItems; ++j) {
        const uint64_t i = base + static_cast<uint64_t>(j) * kGBlock;
        if (i < n) v[j] = __ldg(in + scramble(static_cast<uint32_t>(i), k, mask));
    }
#pragma unroll
    for (int j = 0; j < kGItems; ++j) {
        const uint64_t i = base + static_cast<uint64_t>(j) * kGBlock;
        if (i < n) out[i] = v[j];
    }
}

template <class T>
__global__ void __launch_bounds__(kGBlock) window_scatter_kernel(const T *__restrict__ in, T *__restrict__ out,
                                                                 uint32_t m, uint64_t n)
{
    const uint32_t mask = m >= 32 ? 0xffffffffu : ((1u << m) - 1u);
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * (kGBlock * kGItems) + threadIdx.x;
    T v[kGItems];
#pragma unroll
    for (int j = 0; j < kGItems; ++j) {
        const uint64_t i = base + static_cast<uint64_t>(j) * kGBlock;
        if (i < n) v[j] = __ldcs(in + i);
    }
#pragma unroll
    for (int j = 0; j < kGItems; ++j) {
        const uint64_t i = base + static_cast<uint64_t>(j) * kGBlock;
        if (i < n) {
            const uint64_t window = i >> m;
            out[(window << m) + scramble(static_cast<uint32_t>(i) & mask, m, mask)] = v[j];
        }
    }
}

template <class T>
cudaError_t launch_t(const void *in, void *out, uint32_t k, uint64_t n, cudaStream_t s)
{
    const uint64_t blocks = (n + kGBlock * kGItems - 1) / (kGBlock * kGItems);
    random_gather_kernel<T><<<static_cast<unsigned>(blocks), kGBlock, 0, s>>>(static_cast<const T *>(in),
                                                                              static_cast<T *>(out), k, n);
    return cudaGetLastError();
}

// The staged scatter's occupancy cap: at most this many CTAs per SM, by
// reserving shared memory (more random stores in flight slow the L2 down).
constexpr int kWindowCtasPerSm = 5;
constexpr size_t kWindowSmemReserve = (228u * 1024u) / kWindowCtasPerSm - 1024u;

template <class T>
cudaError_t launch_w(const void *in, void *out, uint32_t m, uint64_t n, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(window_scatter_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kWindowSmemReserve));
    if (e != cudaSuccess) return e;
    const uint64_t blocks = (n + kGBlock * kGItems - 1) / (kGBlock * kGItems);
    window_scatter_kernel<T><<<static_cast<unsigned>(blocks), kGBlock, kWindowSmemReserve, s>>>(
        static_cast<const T *>(in), static_cast<T *>(out), m, n);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_window_scatter(const void *in, void *out, uint32_t k, uint32_t m, uint32_t elem_bytes,
                                  cudaStream_t s)
{
    const uint64_t n = uint64_t{1} << k;
    switch (elem_bytes) {
    case 4: return launch_w<unsigned int>(in, out, m, n, s);
    case 8: return launch_w<unsigned long long>(in, out, m, n, s);
    case 16: return launch_w<uint4>(in, out, m, n, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_random_gather(const void *in, void *out, uint32_t k, uint32_t elem_bytes, cudaStream_t s)
{
    const uint64_t n = uint64_t{1} << k;
    switch (elem_bytes) {
    case 4: return launch_t<unsigned int>(in, out, k, n, s);
    case 8: return launch_t<unsigned long long>(in, out, k, n, s);
    case 16: return launch_t<uint4>(in, out, k, n, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bsh
