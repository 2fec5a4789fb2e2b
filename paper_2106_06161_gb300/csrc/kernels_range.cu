// One shuffle split by domain range (a part of Algorithm 1 per device).
//
// Algorithm 1 (Sec. 4) has one cross-thread dependency, the exclusive scan of
// the keep flags.  Split the domain [0, 2^k) into consecutive ranges: the
// kept indices of range r fill a contiguous run of output slots, starting at
// the number of kept indices in the ranges before it.  So a shuffle splits
// into parts with one exchange of counts: every part counts its range's kept
// indices (count_range_kernel: the cipher and the keep test, no memory
// traffic), the counts are scanned in range order, and every part gathers its
// range's kept elements into its run of slots (the fused single pass
// restricted to the range: the pipelined kernel with RANGE for 4-, 8- and
// 16-byte elements, elem_tile_kernel with RANGE for 1 and 2 bytes).  For n = 2^k nothing
// is dropped: a range's count is its length, and its gather is the scan-free
// direct_range_kernel (kernels_direct.cu).
#include <cstdint>

#include "bshuffle_device.cuh"
#include "bshuffle_internal.h"
#include "elem_kernel.cuh"
#include "pipe_kernel.cuh"

namespace bsh {
namespace {

using dev::kFull;

constexpr int kCountBlock = 256;
constexpr int kCountItems = 8;

struct CountArgs {
    Geometry g;
    uint32_t rounds;
    uint32_t pad0;
    uint64_t first, end;  // domain indices [first, end)
    unsigned long long *count;
    uint32_t keys[kMaxRounds];
};

template <bool ODD>
__global__ void __launch_bounds__(kCountBlock) count_range_kernel(const __grid_constant__ CountArgs a)
{
    const uint64_t base = a.first + uint64_t{blockIdx.x} * (kCountBlock * kCountItems) + threadIdx.x;
    uint32_t left[kCountItems], right[kCountItems];
#pragma unroll
    for (int j = 0; j < kCountItems; ++j) {
        const uint32_t i = static_cast<uint32_t>(base + static_cast<uint64_t>(j * kCountBlock));
        left[j] = i >> a.g.R;
        right[j] = i & a.g.rmask;
    }
    dev::cipher_items<ODD, kCountItems>(left, right, a.keys, a.rounds, a.g);
    uint32_t kept = 0;
#pragma unroll
    for (int j = 0; j < kCountItems; ++j) {
        const uint64_t i = base + static_cast<uint64_t>(j * kCountBlock);
        const uint32_t b = (left[j] << a.g.R) | right[j];
        kept += (i < a.end && b < a.g.n) ? 1u : 0u;
    }
    kept = __reduce_add_sync(kFull, kept);
    if ((threadIdx.x & 31u) == 0 && kept != 0u) atomicAdd(a.count, static_cast<unsigned long long>(kept));
}

__global__ void store_count_kernel(unsigned long long *count, unsigned long long value) { *count = value; }

template <class T>
cudaError_t launch_range_typed(const TileArgs &a, cudaStream_t stream)
{
    constexpr int kBlock = 256, kItems = 8;
    const dim3 grid(a.num_tiles), block(kBlock);
    if (a.g.k & 1u)
        elem::elem_tile_kernel<T, Mode::Gather, true, kBlock, kItems, 0, elem::kVarPhilox, true>
            <<<grid, block, 0, stream>>>(a);
    else
        elem::elem_tile_kernel<T, Mode::Gather, false, kBlock, kItems, 0, elem::kVarPhilox, true>
            <<<grid, block, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_permute_range(const TileArgs &a, uint32_t elem_bytes, cudaStream_t stream)
{
    // tiles as counted by the caller: 2,048 domain indices (the plain
    // kernel's 256 x 8 and the pipelined kernel's 8 warps x 32 x 8)
    if (elem_tile_size(0) != 256u * 8u || pipe_tile_size(elem_bytes, 0) != 256u * 8u) return cudaErrorInvalidValue;
    switch (elem_bytes) {
    case 1: return launch_range_typed<uint8_t>(a, stream);
    case 2: return launch_range_typed<uint16_t>(a, stream);
    case 4: return pipe::launch_shape<uint32_t, Mode::Gather, 8, 8, 3, true, true>(a, stream);
    case 8: return pipe::launch_shape<unsigned long long, Mode::Gather, 8, 8, 3, true, true>(a, stream);
    case 16: return pipe::launch_shape<uint4, Mode::Gather, 8, 8, 3, true, true>(a, stream);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_store_count(unsigned long long *count, uint64_t value, cudaStream_t stream)
{
    store_count_kernel<<<1, 1, 0, stream>>>(count, static_cast<unsigned long long>(value));
    return cudaGetLastError();
}

cudaError_t launch_count_range(const Geometry &g, const uint32_t *keys, uint32_t rounds, uint64_t first,
                               uint64_t end, unsigned long long *count, cudaStream_t stream)
{
    CountArgs a{};
    a.g = g;
    a.rounds = rounds;
    a.first = first;
    a.end = end;
    a.count = count;
    for (uint32_t r = 0; r < rounds && r < kMaxRounds; ++r) a.keys[r] = keys[r];
    const uint64_t per = uint64_t{kCountBlock} * kCountItems;
    const uint64_t blocks = (end - first + per - 1) / per;
    if (blocks == 0) return cudaSuccess;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    if (g.k & 1u)
        count_range_kernel<true><<<static_cast<unsigned>(blocks), kCountBlock, 0, stream>>>(a);
    else
        count_range_kernel<false><<<static_cast<unsigned>(blocks), kCountBlock, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace bsh
