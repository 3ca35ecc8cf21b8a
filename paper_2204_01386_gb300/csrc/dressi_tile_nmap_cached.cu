// dressi_tile_nmap_cached.cu -- per-tile kernel, the forward from stored layer ids with
// the normal map compiled in.
#include "dressi_tile.cuh"

namespace dressi {
template void launch_tile_mode<7>(const Globals &g, cudaStream_t s);
}  // namespace dressi
