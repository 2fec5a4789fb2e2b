// The other shapes of the pipelined single pass (pipe_kernel.cuh) for the
// gather of 4-, 8- and 16-byte elements, selected per width by the
// autotuner (configurations 1 .. kNumPipeConfigs - 1 of kPipeConfigs).
#include <cstdint>

#include "bshuffle_internal.h"
#include "pipe_kernel.cuh"

namespace bsh {
namespace {

template <class T>
cudaError_t launch_typed(const TileArgs &a, int config, cudaStream_t stream)
{
    switch (config) {
    case 1: return pipe::launch_shape<T, Mode::Gather, 8, 4, 4, true>(a, stream);
    case 2: return pipe::launch_shape<T, Mode::Gather, 8, 16, 2, true>(a, stream);
    case 3: return pipe::launch_shape<T, Mode::Gather, 4, 8, 5, true>(a, stream);
    case 4: return pipe::launch_shape<T, Mode::Gather, 16, 4, 2, true>(a, stream);
    case 5: return pipe::launch_shape<T, Mode::Gather, 8, 8, 3, false>(a, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_pipe_tuned(const TileArgs &a, uint32_t elem_bytes, int config, cudaStream_t stream)
{
    static_assert(kNumPipeConfigs == 6, "shapes instantiated here");
    switch (elem_bytes) {
    case 4: return launch_typed<unsigned int>(a, config, stream);
    case 8: return launch_typed<unsigned long long>(a, config, stream);
    case 16: return launch_typed<uint4>(a, config, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bsh
