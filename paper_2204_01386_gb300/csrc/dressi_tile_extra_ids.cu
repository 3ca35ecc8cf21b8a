// dressi_tile_extra_ids.cu -- per-tile kernel, the adjoint from stored layer ids with the
// light gradient and the inverse-UV texel gradient compiled in.
#include "dressi_tile.cuh"

namespace dressi {
template void launch_tile_mode<4>(const Globals &g, cudaStream_t s);
}  // namespace dressi
