// dressi_launch.h -- internal launchers shared by the translation units.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

namespace dressi {
struct Globals;
void count_launch(int n);
void launch_vertex(const Globals &g, int n_views, int max_nv, cudaStream_t s);
void launch_normals(const Globals &g, int n_meshes, int max_nf, int max_nv, cudaStream_t s);
void launch_face(const Globals &g, int n_views, int max_nf, bool count, cudaStream_t s);
void launch_bin(const Globals &g, int n_views, int max_nf, cudaStream_t s);
void launch_tile(const Globals &g, bool backward, cudaStream_t s);
void launch_tile_shade(const Globals &g, cudaStream_t s);
void launch_lpt_order(const Globals &g, cudaStream_t s);
size_t texgather_scratch_bytes(long long slots, long long n_texels, size_t align);
void launch_scan_inplace(int *a, int n, int *partial, cudaStream_t s);
int scan_partials_needed(long long n);
void launch_inv_uv_apply(const Globals &g, long long n_texels, cudaStream_t s);
void launch_tex_gather(const Globals &g, long long slots, long long n_texels, int n_meshes, int max_texels,
                       char *scratch, size_t align, cudaStream_t s);
void launch_vertex_bwd(const Globals &g, int n_views, int max_nv, int n_meshes, int max_nf, bool normals,
                       cudaStream_t s);
void launch_l2(const float *out, const float *tgt, long long n, float *grad, float *loss, cudaStream_t s);
}  // namespace dressi
