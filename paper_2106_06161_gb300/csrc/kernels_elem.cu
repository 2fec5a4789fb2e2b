// Instantiations and dispatch of the fused single-pass element kernel
// (elem_kernel.cuh) for every mode and width in its default configuration,
// and the table of tuning configurations (the others are instantiated for
// the permute path in kernels_elem_tuned.cu).
#include <atomic>
#include <cstdint>

#include "elem_kernel.cuh"

namespace bsh {

const ElemConfig kElemConfigs[kNumElemConfigs] = {
    {256, 8, 0}, {256, 4, 0}, {256, 16, 0}, {512, 8, 0}, {128, 8, 0}, {256, 8, 24}, {512, 4, 0},
};

namespace {

std::atomic<int> g_selected[17] = {};  // per element width (index = bytes), 0 = default

template <class T, Mode MODE>
cudaError_t launch_default(const TileArgs &a, cudaStream_t stream)
{
    return elem::launch_config<T, MODE, 256, 8, 0>(a, stream);
}

template <Mode MODE>
cudaError_t launch_by_width(const TileArgs &a, uint32_t elem_bytes, cudaStream_t stream)
{
    switch (elem_bytes) {
    case 1: return launch_default<unsigned char, MODE>(a, stream);
    case 2: return launch_default<unsigned short, MODE>(a, stream);
    case 4: return launch_default<unsigned int, MODE>(a, stream);
    case 8: return launch_default<unsigned long long, MODE>(a, stream);
    case 16: return launch_default<uint4, MODE>(a, stream);
    default: return cudaErrorInvalidValue;
    }
}

bool tunable_width(uint32_t elem_bytes) { return elem_bytes == 4 || elem_bytes == 8 || elem_bytes == 16; }

}  // namespace

int select_elem_config(uint32_t elem_bytes, int config)
{
    if (!tunable_width(elem_bytes) || config < 0 || config >= kNumElemConfigs) return -1;
    g_selected[elem_bytes].store(config);
    return 0;
}

int selected_elem_config(uint32_t elem_bytes)
{
    return tunable_width(elem_bytes) ? g_selected[elem_bytes].load() : 0;
}

int elem_config_for(uint32_t elem_bytes, Mode mode, uint32_t rounds)
{
    if (mode != Mode::Gather || !tunable_width(elem_bytes)) return 0;
    const int c = g_selected[elem_bytes].load();
    const ElemConfig &cfg = kElemConfigs[c];
    return (cfg.rounds == 0 || cfg.rounds == static_cast<int>(rounds)) ? c : 0;
}

uint32_t elem_tile_size(int config) { return static_cast<uint32_t>(kElemConfigs[config].block * kElemConfigs[config].items); }

cudaError_t launch_elem(const TileArgs &a, Mode mode, uint32_t elem_bytes, int config, cudaStream_t stream)
{
    if (config != 0) {
        if (mode != Mode::Gather) return cudaErrorInvalidValue;
        return launch_gather_tuned(a, elem_bytes, config, stream);
    }
    switch (mode) {
    case Mode::Gather: return launch_by_width<Mode::Gather>(a, elem_bytes, stream);
    case Mode::Scatter: return launch_by_width<Mode::Scatter>(a, elem_bytes, stream);
    case Mode::Index32: return launch_default<unsigned int, Mode::Index32>(a, stream);
    case Mode::Index64: return launch_default<unsigned long long, Mode::Index64>(a, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace bsh
