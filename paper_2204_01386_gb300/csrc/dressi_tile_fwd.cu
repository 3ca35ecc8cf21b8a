// dressi_tile_fwd.cu -- per-tile kernel, forward.
#include "dressi_tile.cuh"

namespace dressi {
template void launch_tile_mode<0>(const Globals &g, cudaStream_t s);
extern template void launch_tile_mode<1>(const Globals &g, cudaStream_t s);
extern template void launch_tile_mode<2>(const Globals &g, cudaStream_t s);

void launch_tile(const Globals &g, bool backward, cudaStream_t s)
{
    if (!backward) launch_tile_mode<0>(g, s);
    else if (g.ids_in) launch_tile_mode<2>(g, s);
    else launch_tile_mode<1>(g, s);
    count_launch(1);
}
}  // namespace dressi
