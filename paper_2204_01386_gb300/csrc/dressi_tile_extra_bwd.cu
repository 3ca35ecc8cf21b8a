// dressi_tile_extra_bwd.cu -- per-tile kernel, the re-rasterizing adjoint with the light
// gradient and the inverse-UV texel gradient compiled in.
#include "dressi_tile.cuh"

namespace dressi {
template void launch_tile_mode<5>(const Globals &g, cudaStream_t s);
}  // namespace dressi
