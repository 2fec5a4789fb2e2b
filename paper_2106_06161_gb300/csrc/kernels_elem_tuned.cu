// Tuning configurations of the fused single-pass permute kernel for 4, 8
// and 16-byte elements (the default configuration is in kernels_elem.cu).
#include <cstdint>

#include "elem_kernel.cuh"

namespace bsh {
namespace {

template <class T>
cudaError_t launch_t(const TileArgs &a, int config, cudaStream_t stream)
{
    switch (config) {
    case 1: return elem::launch_config<T, Mode::Gather, 256, 4, 0>(a, stream);
    case 2: return elem::launch_config<T, Mode::Gather, 256, 16, 0>(a, stream);
    case 3: return elem::launch_config<T, Mode::Gather, 512, 8, 0>(a, stream);
    case 4: return elem::launch_config<T, Mode::Gather, 128, 8, 0>(a, stream);
    case 5: return elem::launch_config<T, Mode::Gather, 256, 8, 24>(a, stream);
    case 6: return elem::launch_config<T, Mode::Gather, 512, 4, 0>(a, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_gather_tuned(const TileArgs &a, uint32_t elem_bytes, int config, cudaStream_t stream)
{
    switch (elem_bytes) {
    case 4: return launch_t<unsigned int>(a, config, stream);
    case 8: return launch_t<unsigned long long>(a, config, stream);
    case 16: return launch_t<uint4>(a, config, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bsh
