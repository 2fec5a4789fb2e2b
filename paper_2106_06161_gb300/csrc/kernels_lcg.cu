// The fused single-pass gather with the LCG bijection of Sec. 3.1 in place of
// VariablePhilox: the same Algorithm 1 (pad, keep b < n, scan, gather) with
// b = (a i + c) mod 2^k.  The paper evaluates it as a cheaper, statistically
// weaker alternative (Tables 1-2, Sec. 5).
#include <cstdint>

#include "elem_kernel.cuh"

namespace bsh {
namespace {

template <class T>
cudaError_t launch_t(const TileArgs &a, cudaStream_t stream)
{
    const dim3 grid(a.num_tiles), block(256);
    elem::elem_tile_kernel<T, Mode::Gather, false, 256, 8, 0, elem::kLcg><<<grid, block, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gather_lcg(const TileArgs &a, uint32_t elem_bytes, cudaStream_t stream)
{
    switch (elem_bytes) {
    case 1: return launch_t<unsigned char>(a, stream);
    case 2: return launch_t<unsigned short>(a, stream);
    case 4: return launch_t<unsigned int>(a, stream);
    case 8: return launch_t<unsigned long long>(a, stream);
    case 16: return launch_t<uint4>(a, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bsh
