/*
 * dressi.h -- C ABI of the GB300 HardSoftRas forward / adjoint library (libdressi.so).
 *
 * HardSoftRas is the soft rasterizer of "Dressi: A Hardware-Agnostic
 * Differentiable Renderer with Reactive Shader Packing and Soft Rasterization"
 * (arXiv 2204.01386), Sec. 3.4.  One call renders (or back-propagates through)
 * a ragged batch of views, each view showing one mesh of a packed scene:
 *
 *   transform and triangle setup      (Sec. 3.4.2; the render-graph listing's
 *                                      vertex transform and face lookup)
 *   per-tile binning of faces grown by r   (Enlarge(), Sec. 3.4.2)
 *   SignedDist, hard test, Shift, K-layer peel  (Alg. 2, Eq. Shift)
 *   perspective-correct interpolation, bilinear texture, shading  (Sec. 3.3.2, 3.3.3)
 *   D_k = sigmoid(dist_k / sigma), edge mask E, colour and silhouette blend
 *                                      (the three blend equations of Sec. 3.4.3)
 *   adjoint of all of the above back to vertex positions, vertex colours and
 *   texels (Sec. 3.4: the gradient dL/dTheta by the chain rule).
 *
 * Conventions shared by every entry point
 *   - Screen space: pixel (x, y) has its centre at (x + 1/2, y + 1/2); the
 *     vertex with clip coordinates c lands at X = (c.x/c.w + 1)/2 * W,
 *     Y = (c.y/c.w + 1)/2 * H (y down), depth c.z/c.w must lie in [0, 1].
 *     Distances handed to sigmoid and Shift are pixel distances / max(W, H)
 *     (the paper's [0, 1] screen units); r, sigma, delta are in those units.
 *   - Ownership: every buffer is owned by the caller.  The library never
 *     allocates device memory; all scratch space lives in the caller's
 *     workspace `ws` (size from dressi_workspace_size).
 *   - Execution: all work is enqueued on `stream` (a cudaStream_t; NULL =
 *     legacy default stream).  No call synchronises the host, so calls can be
 *     captured into a CUDA graph.
 *   - Return codes are synchronous argument checks (DRESSI_*).  Faults found
 *     on the device are OR-ed into `*dev_status` (DRESSI_DEV_* bits); nothing
 *     on the device traps or asserts.
 */
#ifndef DRESSI_H
#define DRESSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* exported from libdressi.so (built with hidden visibility by default) */
#if defined(__GNUC__)
#define DRESSI_API __attribute__((visibility("default")))
#else
#define DRESSI_API
#endif

#define DRESSI_ABI_VERSION 3   /* 2: layer ids carry the soft flag; dressi_forward_from_layers,
                                  dressi_backward_ex; 3: dressi_params.reuse_setup,
                                  dressi_forward_l2 */
#define DRESSI_MAX_K 5          /* the paper keeps K at most five (Sec. 3.4.2) */
#define DRESSI_MAX_VIEWS 65535
#define DRESSI_MAX_MESHES 4096

/* synchronous return codes */
#define DRESSI_OK 0
#define DRESSI_ERR_ARG 1        /* invalid argument (null pointer, bad size, bad mode) */
#define DRESSI_ERR_WORKSPACE 2  /* ws NULL or ws_bytes below dressi_workspace_size() */
#define DRESSI_ERR_LAUNCH 3     /* a CUDA launch failed (cudaGetLastError) */

/* device status bits, OR-ed into *dev_status */
#define DRESSI_DEV_TILE_OVERFLOW 1  /* a tile list exceeded list_cap; that tile fell back to
                                       scanning every face of its view (results stay exact) */
#define DRESSI_DEV_FACE_RANGE 2     /* a face referenced a vertex outside its mesh; face skipped */
#define DRESSI_DEV_NONFINITE 4      /* a vertex transformed to a non-finite position; its faces skipped */

#define DRESSI_TEX_F32 0
#define DRESSI_TEX_F16 1

/* One mesh of the packed scene (host struct). */
typedef struct {
    int32_t n_verts;      /* vertices of this mesh */
    int32_t n_faces;      /* faces of this mesh */
    int64_t vert_off;     /* first vertex in the packed vertex planes */
    int64_t face_off;     /* first face in the packed face array */
    int64_t tex_off;      /* first texel in the packed texture buffer (ignored without texture) */
    int32_t tex_w, tex_h; /* texture size in texels (0 without texture); tex_w * tex_h < 2^31 */
} dressi_mesh;

/* Packed ragged scene.  The struct and `meshes` live in HOST memory; the data
   pointers are DEVICE pointers (caller-owned, read only). */
typedef struct {
    int32_t n_meshes;
    const dressi_mesh *meshes;   /* host array [n_meshes] */
    int64_t n_verts_total;       /* length of one vertex plane */
    const float *pos;            /* [3][n_verts_total] planar x, y, z (object space) */
    const float *col;            /* [3][n_verts_total] planar r, g, b; NULL unless shade_mode 0 */
    const float *uv;             /* [2][n_verts_total] planar u, v; NULL for shade_mode 0 */
    const int32_t *faces;        /* [sum n_faces][3] vertex indices local to the face's mesh */
    const void *tex;             /* [sum texels][4] RGBx texels (row-major per mesh, v = 0 at row 0) */
    int32_t tex_dtype;           /* DRESSI_TEX_F32 or DRESSI_TEX_F16 */
    const void *ntex;            /* shade_mode 3: tangent-space normal map, laid out and typed
                                    like tex (same texel offsets and sizes); NULL otherwise */
} dressi_scene;

/* One view (host struct, passed as a host array). */
typedef struct {
    float mvp[16];      /* row-major 4x4, clip = mvp * (x, y, z, 1) */
    float light[3];     /* unit vector towards a directional light (shade_mode 2) */
    int32_t mesh;       /* index into scene->meshes */
    int32_t width, height;
    int64_t pix_off;    /* first pixel of this view in the packed image buffers; the view
                           occupies pixels [pix_off, pix_off + width*height), row-major */
} dressi_view;

/* Soft-raster parameters (Sec. 3.4.2-3.3.3) and execution choices. */
typedef struct {
    int32_t K;          /* peel layers, 1..DRESSI_MAX_K (Alg. 2) */
    float r;            /* blur radius: faces grow to reach r (Enlarge) */
    float sigma;        /* sigmoid scale of D_k; the paper's default is r / 7 */
    float delta;        /* edge-mask width; window radius rho = max(1, round(delta * max(W, H))) px */
    float gamma;        /* accepted for interface compatibility; unused (the paper drops depth
                           from the colour blend) */
    int32_t edge_mode;  /* 0 edge mask from S^H, 1 E = 1 everywhere (SoftRas-like), 2 E = 0 (hard) */
    int32_t shade_mode; /* 0 vertex colour, 1 unlit texture, 2 texture * max(0, n.l),
                           3 texture * max(0, n'.l) with n' from the normal map ntex: map value
                           t, nt = 2 t - 1 in the face's tangent frame (tangent from the object
                           edges and UV differences, orthogonalised against the interpolated
                           normal n; bitangent h n x T', h the sign of the UV determinant),
                           n' = normalize(nt0 T' + nt1 B' + nt2 n) */
    int32_t texgrad_mode; /* 0 vector red.global atomics, 1 texel-space gather (deterministic),
                             2 inverse UV (Sec. 3.3.2, Alg. 1; approximate: each texel takes the
                             dL/d(albedo) of the last shaded sample that lands on it) */
    int32_t tile;       /* tile edge in pixels: 16 or 32; 0 = 16 */
    int32_t schedule;   /* per-tile kernel: 0 auto (= 1), 1 one CTA per tile, 2 persistent CTAs
                           pulling (view, tile) items longest face list first */
    int64_t list_cap;   /* tile-list capacity in entries; 0 = library default
                           max(4 x faces over all views, 64 x tiles).  Clamped to
                           2^31 - 2.  A tile whose list ends past it falls back to the
                           view's whole mesh and sets DRESSI_DEV_TILE_OVERFLOW */
    float uv_jitter[2]; /* texgrad_mode 2: offset (pixels) of every sample from its pixel
                           centre for the inverse-UV lookup; the paper draws a Sobol point per
                           frame (the caller supplies it; [-0.5, 0.5)^2 keeps it in the pixel) */
    int32_t reuse_setup; /* dressi_backward(_ex) only: 1 = the workspace still holds what the
                            last forward call on it (dressi_forward, dressi_forward_l2, or
                            dressi_forward_from_layers, which builds no tile lists) built for
                            the same scene (positions unchanged), views and params -- vertex
                            transform, face table, normals and, for layer_ids == NULL, the
                            tile lists -- and the backward takes it instead of rebuilding it
                            (with layer_ids == NULL it still re-rasterizes: layers and
                            barycentrics are recomputed, each pixel's K-list starting from the
                            K-th (key, face) that a forward without layer ids kept in the
                            workspace, which culls the candidates that cannot reach the K
                            layers).  0 = rebuild.  The caller guarantees the precondition; a
                            workspace written by another call since gives wrong gradients. */
} dressi_params;

/* Size in bytes of the workspace that dressi_forward / dressi_backward need for
   this scene, view set and parameters (host-only computation; views is a host
   array).  Returns 0 on invalid arguments, among them a packed texel count of
   2^32 - 1 or more with texgrad_mode 1 (the gather sorts 32-bit texel keys). */
DRESSI_API size_t dressi_workspace_size(const dressi_scene *scene, const dressi_view *views, int32_t n_views,
                             const dressi_params *params);

/* Forward pass (Alg. 2 and the blend equations of Sec. 3.4.3).
     out_rgba   DEVICE [n_pix][4] float: colour I_c in rgb, silhouette I_s in alpha,
                at the views' pixel offsets.  Pixels of no view are left untouched.
     layer_ids  DEVICE [K][n_pix] int32 or NULL: per peel layer, the face index (local to
                the view's mesh), with bit 31 set when the fragment is soft (the pixel lies
                outside the hard face, within r of it), and -1 where a layer is empty.
                Decode: face = v & 0x7fffffff, hard = v >= 0.  Pass it to dressi_backward
                to skip re-rasterization; NULL keeps nothing between the passes.
     n_pix      total pixels of the packed image buffers (>= every pix_off + W*H).
     ws         DEVICE workspace of ws_bytes >= dressi_workspace_size(...).
     dev_status DEVICE int32, OR-ed with DRESSI_DEV_* bits (never cleared by the library).
     stream     cudaStream_t. */
DRESSI_API int dressi_forward(const dressi_scene *scene, const dressi_view *views, int32_t n_views,
                   const dressi_params *params, float *out_rgba, int32_t *layer_ids, int64_t n_pix,
                   void *ws, size_t ws_bytes, int32_t *dev_status, void *stream);

/* dressi_forward fused with an L2 image loss L = sum (out_rgba - target)^2 (no counterpart
   in the paper; the loss of a fit to target images): besides out_rgba it writes
   grad_rgba = dL/d(out_rgba) = 2 (out_rgba - target), the input of dressi_backward, and
   adds L to *loss_accum.  grad_rgba equals dressi_forward followed by
   dressi_l2_loss_grad bit for bit; the loss is summed in another order.
     target     DEVICE [n_pix][4] float (16-byte aligned).
     grad_rgba  DEVICE [n_pix][4] float, written for the pixels of the views (the pixels
                of the packed buffers outside every view are left as they are).
     loss_accum DEVICE float or NULL; not cleared.
   All other arguments as for dressi_forward. */
DRESSI_API int dressi_forward_l2(const dressi_scene *scene, const dressi_view *views, int32_t n_views,
                                 const dressi_params *params, const float *target, float *out_rgba,
                                 float *grad_rgba, float *loss_accum, int32_t *layer_ids, int64_t n_pix,
                                 void *ws, size_t ws_bytes, int32_t *dev_status, void *stream);

/* Forward from stored layers: the cached-rasterization counterpart of the reactive cache
   of Sec. 3.3.3 (Stage Packing), which skips passes whose inputs did not change -- here,
   when the geometry and views are static (texture, colour or light optimisation), the
   binning, raster and peel of Sec. 3.4.2 are skipped and only shading and blending
   (Sec. 3.4.3) run on the layers an earlier dressi_forward stored.
     layer_ids  DEVICE [K][n_pix] from dressi_forward with the same positions, faces,
                views, K and r (same encoding; the hard flags give S^H).  Colours,
                textures, shade_mode, the light, sigma, delta and edge_mode may differ;
                the result then equals dressi_forward with the new values bit for bit.
     out_rgba, n_pix, ws, ws_bytes, dev_status, stream as for dressi_forward (the
                workspace size is the same).
   Layer ids that do not match the scene give wrong images but no fault: a face index out
   of its mesh's range makes that layer contribute nothing.
   The adjoint of this call is dressi_backward with the same layer_ids. */
DRESSI_API int dressi_forward_from_layers(const dressi_scene *scene, const dressi_view *views, int32_t n_views,
                                          const dressi_params *params, const int32_t *layer_ids, float *out_rgba,
                                          int64_t n_pix, void *ws, size_t ws_bytes, int32_t *dev_status,
                                          void *stream);

/* Adjoint of dressi_forward for the pixel gradient grad_rgba = dL/d(out_rgba).
     grad_rgba  DEVICE [n_pix][4] float.
     layer_ids  DEVICE [K][n_pix] from dressi_forward with the same inputs, or NULL to
                recompute layers and barycentrics (checkpointing).
     grad_pos   DEVICE [3][n_verts_total] float, OVERWRITTEN with dL/dpos summed over views.
     grad_col   DEVICE [3][n_verts_total] float or NULL, OVERWRITTEN (shade_mode 0).
     grad_tex   DEVICE [sum texels][4] float or NULL, OVERWRITTEN (shade_mode 1, 2); channel 3
                stays zero.  Always FP32, also for an FP16 texture.
   Discrete quantities (layer choice, hard flags, S^H, E, depth keys) carry no gradient. */
DRESSI_API int dressi_backward(const dressi_scene *scene, const dressi_view *views, int32_t n_views,
                    const dressi_params *params, const float *grad_rgba, const int32_t *layer_ids,
                    int64_t n_pix, float *grad_pos, float *grad_col, float *grad_tex,
                    void *ws, size_t ws_bytes, int32_t *dev_status, void *stream);

/* dressi_backward that also returns the gradients of the camera and the light, the
   parameters theta_C and theta_L of Theta (Sec. 3.4.1):
     grad_mvp   DEVICE [n_views][16] float or NULL, OVERWRITTEN with dL/dMVP per view
                (row-major like dressi_view.mvp; row 2, the depth row, stays 0: depth only
                orders the layers, a discrete choice).
     grad_light DEVICE [n_views][3] float or NULL, OVERWRITTEN with dL/dlight per view
                (shade_mode 2, 3; the light is used as given, not renormalised; 0 otherwise).
     grad_ntex  DEVICE [sum texels][4] float or NULL, OVERWRITTEN with the normal-map texel
                gradient (shade_mode 3; texgrad_mode 0: atomics); channel 3 stays zero.
   All other arguments as for dressi_backward, which is this call with both NULL. */
DRESSI_API int dressi_backward_ex(const dressi_scene *scene, const dressi_view *views, int32_t n_views,
                                  const dressi_params *params, const float *grad_rgba, const int32_t *layer_ids,
                                  int64_t n_pix, float *grad_pos, float *grad_col, float *grad_tex,
                                  float *grad_mvp, float *grad_light, float *grad_ntex, void *ws,
                                  size_t ws_bytes, int32_t *dev_status, void *stream);

/* Size of the library's static device scratch array used by
   dressi_forward_static_scratch (bytes; held on every GPU that loads the library). */
#define DRESSI_STATIC_SCRATCH_BYTES (32u << 20)

/* dressi_forward without a caller workspace (the paper has no counterpart: this is
   an interface for callers that cannot allocate device memory, e.g. a plugin whose
   host application owns every device allocation, or a frame loop that must not pay
   cudaMalloc's implicit device synchronisation).  Same arguments and results as
   dressi_forward; the scratch space is a file-scope device array of
   DRESSI_STATIC_SCRATCH_BYTES inside the library instead of `ws`.
     - Scenes whose dressi_workspace_size() exceeds DRESSI_STATIC_SCRATCH_BYTES are
       rejected with DRESSI_ERR_WORKSPACE before anything is enqueued.
     - The first call on a device looks up the array's device address on the current
       device (once per device); make that first call before any stream capture.  The
       address stays cached for the life of the process: after a cudaDeviceReset of that
       device this entry point must not be called again.
     - The library allocates nothing here (no cudaMalloc / cudaFree); the counters the
       pass needs zeroed are cleared on `stream` at every call.
     - All calls on a device share the one array, which keeps the last call's
       contents: calls that overlap on the GPU (different streams, or different host
       threads) race on it and must be serialised by the caller. */
DRESSI_API int dressi_forward_static_scratch(const dressi_scene *scene, const dressi_view *views, int32_t n_views,
                                             const dressi_params *params, float *out_rgba, int32_t *layer_ids,
                                             int64_t n_pix, int32_t *dev_status, void *stream);

/* Autotuner (no counterpart in the paper): times one forward + adjoint pass (the
   adjoint with reuse_setup = 1, as in a training step) for every execution choice (tile edge 16 / 32, schedule 1 / 2) whose workspace fits in
   ws_bytes, keeps the fastest in params->tile / params->schedule, and sets
   params->list_cap to the tile-list entries this scene actually needs plus 25 %
   headroom (so the workspace of later calls can shrink).  The method parameters
   (K, r, sigma, delta, modes) are not changed.  out_rgba, layer_ids, grad_* and ws
   are scratch that this call overwrites (same shapes as for dressi_forward /
   dressi_backward); pass layer_ids (or NULL) as the calls being tuned will, since
   keeping the layer ids or re-rasterizing in the adjoint changes which choice wins.
   This call synchronises the host (it reads timings and the list size back), so it
   must not be captured into a CUDA graph.  *best_ms receives the fastest pass time.
   Returns DRESSI_ERR_WORKSPACE when no choice fits in ws_bytes. */
DRESSI_API int dressi_autotune(const dressi_scene *scene, const dressi_view *views, int32_t n_views,
                               dressi_params *params, float *out_rgba, int32_t *layer_ids, int64_t n_pix,
                               float *grad_pos,
                               float *grad_col, float *grad_tex, void *ws, size_t ws_bytes, int32_t *dev_status,
                               void *stream, float *best_ms);

/* L2 loss helper for training loops: grad[i] = 2 (out[i] - target[i]) over n floats and
   *loss_accum += sum (out - target)^2 (DEVICE float, accumulated atomically). */
DRESSI_API int dressi_l2_loss_grad(const float *out, const float *target, int64_t n, float *grad,
                        float *loss_accum, void *stream);

/* Static description of a synchronous return code (DRESSI_OK .. DRESSI_ERR_LAUNCH). */
DRESSI_API const char *dressi_status_string(int code);

/* Static description of one DRESSI_DEV_* bit of *dev_status. */
DRESSI_API const char *dressi_dev_status_string(int bit);

/* Profiling hook (no counterpart in the paper): when set, each pass records
   `begin` / `end` (cudaEvent_t handles, caller-owned) on its stream right
   before and after its per-tile kernel, so a caller can time that kernel with
   cudaEventElapsedTime.  fwd_* are used by dressi_forward, bwd_* by
   dressi_backward; NULL disables.  Process-wide setting, not thread safe. */
DRESSI_API int dressi_set_profile_events(void *fwd_begin, void *fwd_end, void *bwd_begin, void *bwd_end);

/* Statistics hook (no counterpart in the paper): when dev_counters (DEVICE array of
   4 unsigned 64-bit integers, caller-owned and caller-zeroed) is set, every per-tile
   kernel adds to it: [0] (face, pixel) pairs enumerated, [1] exact SignedDist
   evaluations, [2] of those, candidates (dist >= -r) merged into a K-list, [3] layers
   shaded (forward) or back-propagated (adjoint).  NULL disables.  Process-wide
   setting, not thread safe; the counting costs one atomic per warp and tile. */
DRESSI_API int dressi_set_stats_buffer(void *dev_counters);

/* Inspection hook for texgrad_mode 2 (no counterpart in the paper): when set, each
   dressi_backward(_ex) with texgrad_mode 2 copies the inverse-UV texture -- per texel
   (packed like grad_tex) the number of the sample that wrote it last,
   (view pixel offset + y W + x) K + layer with the views' pixels counted in order, or
   -1 -- into this DEVICE int32 [sum texels] buffer.  NULL disables.  Process-wide
   setting, not thread safe. */
DRESSI_API int dressi_set_inverse_uv_buffer(int32_t *dev_buffer);

/* Inspection hook of the persistent schedule (no counterpart in the paper): when set,
   each pass with schedule 2 that builds tile lists copies the order in which its CTAs
   take the tiles (global tile numbers, views' tiles counted in view order, row-major
   inside a view) into dev_order and each tile's face-list length (indexed by tile)
   into dev_lengths (DEVICE int32 [total tiles] each, either may be NULL).  NULL, NULL
   disables.  Process-wide setting, not thread safe. */
DRESSI_API int dressi_set_tile_order_buffer(int32_t *dev_order, int32_t *dev_lengths);

/* Peaks of the units the per-tile kernels use, measured on the current device (no
   counterpart in the paper: the measured denominators of roofline fractions).
     which 0: FP32 FMA throughput in TFLOP/s (an FMA counts 2): eight independent FMA
              chains in every thread of 2,048 threads per SM on every SM;
     which 1: red.global.add.v4.f32 throughput in GB/s of reduction payload: every lane
              adds a float4 into its own 16 bytes (one warp instruction covers 512
              contiguous bytes), the launch stepping through the buffer;
     which 2: the same with every lane's float4 in a 32-byte sector of its own (lanes 4 KiB
              apart), in GB/s of 32-byte sectors reduced at L2 (the scattered pattern of
              gradient scatters).
   dev_buf  DEVICE scratch, 16-byte aligned, bytes >= 64 MiB (caller-owned; overwritten).
   result   HOST double receiving the figure (the best of five timed launches).
   Synchronises the host (it reads event timings back), so it must not be captured into a
   CUDA graph. */
DRESSI_API int dressi_measure_peak(int32_t which, void *dev_buf, size_t bytes, double *result, void *stream);

/* Number of kernels this library has launched since it was loaded (process-wide). */
DRESSI_API unsigned long long dressi_launch_count(void);

/* DRESSI_ABI_VERSION of the loaded library. */
DRESSI_API int dressi_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DRESSI_H */
