// dressi_tile_fwd.cu -- per-tile kernel, forward.
#include "dressi_tile.cuh"

namespace dressi {
template void launch_tile_mode<0>(const Globals &g, cudaStream_t s);
extern template void launch_tile_mode<1>(const Globals &g, cudaStream_t s);
extern template void launch_tile_mode<2>(const Globals &g, cudaStream_t s);
extern template void launch_tile_mode<4>(const Globals &g, cudaStream_t s);
extern template void launch_tile_mode<5>(const Globals &g, cudaStream_t s);
extern template void launch_tile_mode<6>(const Globals &g, cudaStream_t s);

void launch_tile(const Globals &g, bool backward, cudaStream_t s)
{
    // the adjoint with the light gradient, the inverse UV or the normal map uses the
    // kernels that have them
    const bool extra = (g.glight != nullptr && g.shade_mode >= 2) || g.texgrad_mode == 2 || g.shade_mode == 3;
    if (!backward) g.shade_mode == 3 ? launch_tile_mode<6>(g, s) : launch_tile_mode<0>(g, s);
    else if (g.ids_in) extra ? launch_tile_mode<4>(g, s) : launch_tile_mode<2>(g, s);
    else extra ? launch_tile_mode<5>(g, s) : launch_tile_mode<1>(g, s);
    count_launch(1);
}
}  // namespace dressi
