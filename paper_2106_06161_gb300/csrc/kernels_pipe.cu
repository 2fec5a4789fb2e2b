// Pipelined single pass of Algorithm 1 (pipe_kernel.cuh): the default shape
// for every mode and width, the table of shapes the gather of 4-, 8- and
// 16-byte elements can be tuned over, and the selection per width.
//
// Shape 0 is the default: eight compute warps of 8 items and three resident
// CTAs per SM measured fastest on GB300 (more tiles in flight lengthen every
// look-back walk; fewer warps hide less latency).  The other shapes are
// instantiated in kernels_pipe_tuned.cu and serve bshuffle_permute only.
#include <atomic>
#include <cstdint>

#include "bshuffle_internal.h"
#include "pipe_kernel.cuh"

namespace bsh {

const PipeConfig kPipeConfigs[kNumPipeConfigs] = {
    {8, 8, 3, 1}, {8, 4, 4, 1}, {8, 16, 2, 1}, {4, 8, 5, 1}, {16, 4, 2, 1}, {8, 8, 3, 0},
};

namespace {

std::atomic<int> g_pipe_selected[5];  // per width class: 1, 2, 4, 8, 16 bytes

int width_slot(uint32_t elem_bytes)
{
    switch (elem_bytes) {
    case 4: return 2;
    case 8: return 3;
    case 16: return 4;
    default: return -1;
    }
}

template <class T, Mode MODE>
cudaError_t launch_default(const TileArgs &a, cudaStream_t stream)
{
    return pipe::launch_shape<T, MODE, 8, 8, 3, true>(a, stream);
}

}  // namespace

int pipe_config_for(uint32_t elem_bytes, Mode mode)
{
    const int slot = width_slot(elem_bytes);
    if (mode != Mode::Gather || slot < 0) return 0;
    return g_pipe_selected[slot].load();
}

int select_pipe_config(uint32_t elem_bytes, int config)
{
    const int slot = width_slot(elem_bytes);
    if (slot < 0 || config < 0 || config >= kNumPipeConfigs) return -1;
    g_pipe_selected[slot].store(config);
    return 0;
}

int selected_pipe_config(uint32_t elem_bytes)
{
    const int slot = width_slot(elem_bytes);
    return slot < 0 ? 0 : g_pipe_selected[slot].load();
}

uint32_t pipe_tile_size(uint32_t, int config)
{
    const PipeConfig &c = kPipeConfigs[config >= 0 && config < kNumPipeConfigs ? config : 0];
    return static_cast<uint32_t>(c.warps * 32 * c.items);
}

bool pipe_supports(Mode mode, uint32_t elem_bytes)
{
    switch (mode) {
    case Mode::Gather:
    case Mode::Scatter: return elem_bytes == 4 || elem_bytes == 8 || elem_bytes == 16;
    case Mode::Index32:
    case Mode::Index64: return true;
    }
    return false;
}

cudaError_t launch_pipe(const TileArgs &a, Mode mode, uint32_t elem_bytes, int config, cudaStream_t stream)
{
    if (config != 0) {
        if (mode != Mode::Gather) return cudaErrorInvalidValue;
        return launch_pipe_tuned(a, elem_bytes, config, stream);
    }
    switch (mode) {
    case Mode::Index32: return launch_default<unsigned int, Mode::Index32>(a, stream);
    case Mode::Index64: return launch_default<unsigned long long, Mode::Index64>(a, stream);
    case Mode::Gather:
        switch (elem_bytes) {
        case 4: return launch_default<unsigned int, Mode::Gather>(a, stream);
        case 8: return launch_default<unsigned long long, Mode::Gather>(a, stream);
        case 16: return launch_default<uint4, Mode::Gather>(a, stream);
        default: return cudaErrorInvalidValue;
        }
    case Mode::Scatter:
        switch (elem_bytes) {
        case 4: return launch_default<unsigned int, Mode::Scatter>(a, stream);
        case 8: return launch_default<unsigned long long, Mode::Scatter>(a, stream);
        case 16: return launch_default<uint4, Mode::Scatter>(a, stream);
        default: return cudaErrorInvalidValue;
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace bsh
