// dressi_tile_bwd.cu -- per-tile kernel, adjoint that re-rasterizes (no stored layer ids).
#include "dressi_tile.cuh"

namespace dressi {
template void launch_tile_mode<1>(const Globals &g, cudaStream_t s);
}  // namespace dressi
