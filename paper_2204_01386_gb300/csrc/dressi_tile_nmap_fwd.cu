// dressi_tile_nmap_fwd.cu -- per-tile kernel, the forward with the normal map compiled in.
#include "dressi_tile.cuh"

namespace dressi {
template void launch_tile_mode<6>(const Globals &g, cudaStream_t s);
}  // namespace dressi
