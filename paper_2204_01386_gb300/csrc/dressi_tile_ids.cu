// dressi_tile_ids.cu -- per-tile kernel, adjoint from stored layer ids.
#include "dressi_tile.cuh"

namespace dressi {
template void launch_tile_mode<2>(const Globals &g, cudaStream_t s);
}  // namespace dressi
