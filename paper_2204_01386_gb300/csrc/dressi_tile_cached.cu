// dressi_tile_cached.cu -- per-tile kernel, forward from stored layer ids: re-shading a
// static geometry whose layers an earlier forward kept (textures, colours, light or the
// blend parameters changed).
#include "dressi_tile.cuh"

namespace dressi {
template void launch_tile_mode<3>(const Globals &g, cudaStream_t s);
extern template void launch_tile_mode<7>(const Globals &g, cudaStream_t s);

void launch_tile_shade(const Globals &g, cudaStream_t s)
{
    if (g.shade_mode == 3) launch_tile_mode<7>(g, s);
    else launch_tile_mode<3>(g, s);
    count_launch(1);
}
}  // namespace dressi
