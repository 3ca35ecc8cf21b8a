// dressi_api.cu -- the extern "C" entry points declared in include/dressi.h:
// argument checks, workspace layout, upload of the view / mesh tables into the
// workspace, and the order of the kernel launches of one pass.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "dressi_core.cuh"
#include "dressi_launch.h"

namespace dressi {

constexpr int TILE_DEFAULT = 16;
constexpr int RHO_LIMIT = 8;
constexpr size_t ALIGN = 256;

static size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

static std::atomic<unsigned long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

// optional events recorded around the per-tile kernel (profiling hook)
static cudaEvent_t g_prof[4] = {nullptr, nullptr, nullptr, nullptr};
// optional device work counters of the per-tile kernel (statistics hook)
static unsigned long long *g_stats = nullptr;
static int *g_inv_uv_out = nullptr;
// optional copies of the persistent schedule's tile order and the tiles' face-list lengths
static int *g_order_out = nullptr, *g_lengths_out = nullptr;

// pass: 0 forward, 1 adjoint, 2 forward from stored layer ids (timed as a forward)
static void launch_tile_profiled(const Globals &g, int pass, cudaStream_t s)
{
    const bool bwd = pass == 1;
    cudaEvent_t b = g_prof[bwd ? 2 : 0], e = g_prof[bwd ? 3 : 1];
    if (b) cudaEventRecord(b, s);
    if (pass == 2) launch_tile_shade(g, s);
    else launch_tile(g, bwd, s);
    if (e) cudaEventRecord(e, s);
}

struct Layout {
    size_t views, meshes, vrec, frec, brect, tile_view, tile_count, tile_off, tile_cursor, lists, nrm, adj_off, adj_cur, adj, scan_partial,
        sgrad, ngrad, queue,
        tile_order, lpt_hist, kth, kth_flag, tg_keys, tg_pay0, tg_pay1, tg_scratch, inv_uv, total;
    long long tg_slots;   // texel-gather record slots (0 unless texgrad_mode 1 with a texture)
    long long n_vrec;
    int total_tiles;
    long long list_cap;
};

struct Plan {
    std::vector<ViewK> views;
    std::vector<MeshK> meshes;
    Layout lay;
    int max_nv = 0, max_nf = 0, max_nv_view = 0, max_nf_view = 0, max_texels = 0;
    long long n_texels = 0, n_faces = 0;
};

static bool check_params(const dressi_params *p)
{
    if (!p) return false;
    if (p->K < 1 || p->K > DRESSI_MAX_K) return false;
    if (!(p->r >= 0.f) || !(p->sigma > 0.f) || !(p->delta >= 0.f) || !std::isfinite(p->r) ||
        !std::isfinite(p->sigma) || !std::isfinite(p->delta))
        return false;
    if (p->edge_mode < 0 || p->edge_mode > 2) return false;
    if (p->shade_mode < 0 || p->shade_mode > 3) return false;
    if (p->texgrad_mode < 0 || p->texgrad_mode > 2) return false;
    if (!std::isfinite(p->uv_jitter[0]) || !std::isfinite(p->uv_jitter[1])) return false;
    if (p->tile != 0 && p->tile != 16 && p->tile != 32) return false;
    if (p->schedule < 0 || p->schedule > 2) return false;
    if (p->list_cap < 0) return false;
    if (p->reuse_setup != 0 && p->reuse_setup != 1) return false;
    return true;
}

// Builds the host-side tables and the workspace layout; false on invalid arguments.
static bool make_plan(const dressi_scene *sc, const dressi_view *views, int n_views, const dressi_params *p,
                      long long n_pix, Plan &P)
{
    if (!sc || !views || !check_params(p)) return false;
    if (n_views < 1 || n_views > DRESSI_MAX_VIEWS) return false;
    if (sc->n_meshes < 1 || sc->n_meshes > DRESSI_MAX_MESHES || !sc->meshes) return false;
    if (sc->n_verts_total < 0 || sc->tex_dtype < 0 || sc->tex_dtype > 1) return false;
    const bool textured = p->shade_mode != 0;
    P.meshes.resize(sc->n_meshes);
    for (int m = 0; m < sc->n_meshes; ++m) {
        const dressi_mesh &dm = sc->meshes[m];
        if (dm.n_verts < 0 || dm.n_faces < 0 || dm.vert_off < 0 || dm.face_off < 0) return false;
        if (dm.vert_off + dm.n_verts > sc->n_verts_total) return false;
        MeshK &k = P.meshes[m];
        k.vert_off = dm.vert_off;
        k.face_off = dm.face_off;
        k.tex_off = dm.tex_off;
        k.nV = dm.n_verts;
        k.nF = dm.n_faces;
        k.tex_w = dm.tex_w;
        k.tex_h = dm.tex_h;
        if (textured) {
            if (dm.tex_w <= 0 || dm.tex_h <= 0 || dm.tex_off < 0) return false;
            if ((long long)dm.tex_w * dm.tex_h > 0x7fffffffLL) return false;   // texel counts are int32
            P.n_texels = std::max(P.n_texels, (long long)dm.tex_off + (long long)dm.tex_w * dm.tex_h);
            P.max_texels = std::max(P.max_texels, dm.tex_w * dm.tex_h);
        }
        P.max_nv = std::max(P.max_nv, dm.n_verts);
        P.max_nf = std::max(P.max_nf, dm.n_faces);
        P.n_faces += dm.n_faces;
    }
    if (!sc->pos || !sc->faces) return false;
    if (p->shade_mode == 0 && !sc->col) return false;
    if (textured && (!sc->uv || !sc->tex)) return false;
    if (p->shade_mode == 3 && !sc->ntex) return false;

    P.views.resize(n_views);
    long long vrec = 0, view_faces = 0, view_pixels = 0;
    int tiles = 0;
    const int T = p->tile ? p->tile : TILE_DEFAULT;
    for (int v = 0; v < n_views; ++v) {
        const dressi_view &dv = views[v];
        if (dv.mesh < 0 || dv.mesh >= sc->n_meshes) return false;
        if (dv.width < 1 || dv.height < 1 || dv.width > 32768 || dv.height > 32768) return false;
        if (dv.pix_off < 0 || dv.pix_off + (long long)dv.width * dv.height > n_pix) return false;
        for (int i = 0; i < 16; ++i)
            if (!std::isfinite(dv.mvp[i])) return false;
        ViewK &k = P.views[v];
        std::memcpy(k.mvp, dv.mvp, sizeof(k.mvp));
        std::memcpy(k.light, dv.light, sizeof(k.light));
        k.mesh = dv.mesh;
        k.W = dv.width;
        k.H = dv.height;
        k.tiles_x = (dv.width + T - 1) / T;
        k.tiles_y = (dv.height + T - 1) / T;
        k.tile_base = tiles;
        const double S = (double)std::max(dv.width, dv.height);
        int rho = (int)std::lround((double)p->delta * S);
        if (rho < 1) rho = 1;
        if (p->edge_mode == 0 && rho > RHO_LIMIT) return false;
        k.rho = rho;
        k.r_px = (float)((double)p->r * S);
        k.inv_sigma_px = (float)(1.0 / ((double)p->sigma * S));
        k.half_inv_S = (float)(0.5 / S);
        k.bin_R = std::max(k.r_px, p->edge_mode == 0 ? (float)rho : 0.f) + 1.0f;
        k.pad = 0;
        k.pix_off = dv.pix_off;
        k.vrec_off = vrec;
        k.slot_base = view_pixels;
        k.frec_off = view_faces;
        view_pixels += (long long)dv.width * dv.height;
        const MeshK &mk = P.meshes[dv.mesh];
        vrec += mk.nV;
        view_faces += mk.nF;
        P.max_nv_view = std::max(P.max_nv_view, mk.nV);
        P.max_nf_view = std::max(P.max_nf_view, mk.nF);
        long long nt = (long long)tiles + (long long)k.tiles_x * k.tiles_y;
        if (nt > 0x7fffffff) return false;
        tiles = (int)nt;
    }
    Layout &L = P.lay;
    L.n_vrec = vrec;
    L.total_tiles = tiles;
    L.list_cap = p->list_cap > 0 ? p->list_cap : std::max<long long>(4 * view_faces, 64LL * tiles);
    // below INT_MAX: the saturating tile-count scan marks a total past 2^31 - 1 as INT_MAX,
    // which must read as over capacity
    if (L.list_cap > 0x7ffffffeLL) L.list_cap = 0x7ffffffeLL;
    size_t o = 0;
    L.views = o; o = align_up(o + sizeof(ViewK) * n_views);   // at 0, the mesh table right after it
    L.meshes = o; o = align_up(o + sizeof(MeshK) * sc->n_meshes);
    L.vrec = o; o = align_up(o + sizeof(VRec) * (size_t)std::max<long long>(vrec, 1));
    L.frec = o; o = align_up(o + sizeof(FaceRec) * (size_t)std::max<long long>(view_faces, 1));
    L.brect = o; o = align_up(o + sizeof(unsigned) * (size_t)std::max<long long>(view_faces, 1));
    L.tile_view = o; o = align_up(o + sizeof(int) * (size_t)std::max(tiles, 1));
    L.tile_count = o; o = align_up(o + sizeof(int) * (size_t)tiles);
    L.tile_off = o; o = align_up(o + sizeof(int) * (size_t)(tiles + 1));
    L.tile_cursor = o; o = align_up(o + sizeof(int) * (size_t)tiles);
    L.lists = o; o = align_up(o + sizeof(int) * (size_t)L.list_cap);
    const size_t nv = (size_t)std::max<long long>(sc->n_verts_total, 1);
    L.nrm = o; o = align_up(o + sizeof(float4) * nv);
    L.adj_off = o; o = align_up(o + sizeof(int) * (nv + 1));
    L.adj_cur = o; o = align_up(o + sizeof(int) * nv);
    L.adj = o; o = align_up(o + sizeof(int) * 3 * (size_t)std::max<long long>(P.n_faces, 1));
    L.scan_partial = o;
    o = align_up(o + sizeof(int) * (size_t)scan_partials_needed(std::max<long long>((long long)nv + 1, tiles + 1)));
    L.sgrad = o; o = align_up(o + sizeof(float4) * (size_t)std::max<long long>(vrec, 1));
    L.ngrad = o; o = align_up(o + sizeof(float4) * nv);
    L.queue = o; o = align_up(o + sizeof(int) * 4);
    L.tile_order = o; o = align_up(o + sizeof(int) * (size_t)std::max(tiles, 1));
    L.lpt_hist = o; o = align_up(o + sizeof(int) * LPT_BINS);
    L.kth = o; o = align_up(o + sizeof(unsigned long long) * (size_t)std::max<long long>(view_pixels, 1));
    L.kth_flag = o; o = align_up(o + sizeof(int));
    L.tg_slots = (p->texgrad_mode != 0 && textured) ? view_pixels * p->K : 0;
    // the texel gather sorts 32-bit texel keys with 0xffffffff marking an empty slot: every
    // packed texel index must stay below it
    if (p->texgrad_mode == 1 && textured && P.n_texels >= 0xffffffffLL) return false;
    // the inverse UV stores sample numbers as int32 (atomicMax)
    if (p->texgrad_mode == 2 && L.tg_slots > 0x7fffffffLL) return false;
    L.inv_uv = o; o = align_up(o + sizeof(int) * (size_t)((p->texgrad_mode == 2 && textured) ? std::max<long long>(P.n_texels, 1) : 1));
    const size_t ts = (size_t)std::max<long long>(L.tg_slots, 1);
    L.tg_keys = o; o = align_up(o + sizeof(unsigned) * ts);
    L.tg_pay0 = o; o = align_up(o + sizeof(float4) * ts);
    L.tg_pay1 = o; o = align_up(o + sizeof(float) * ts);
    L.tg_scratch = o;
    o = align_up(o + (L.tg_slots && p->texgrad_mode == 1 ? texgather_scratch_bytes(L.tg_slots, P.n_texels, ALIGN) : 0));
    L.total = o;
    return true;
}

// ---------------------------------------------------------------------------
// table upload: the tables travel as kernel parameters (no host-to-device copy,
// so a whole pass can be captured into a CUDA graph)
// ---------------------------------------------------------------------------
constexpr int BLOB_WORDS = 4000;
struct Blob {
    unsigned int n;
    unsigned int w[BLOB_WORDS];
};

__global__ void k_upload(const __grid_constant__ Blob b, unsigned int *dst)
{
    for (unsigned int i = threadIdx.x; i < b.n; i += blockDim.x) dst[i] = b.w[i];
}

static void upload(const void *src, size_t bytes, void *dst, cudaStream_t s)
{
    const unsigned int *w = static_cast<const unsigned int *>(src);
    size_t words = bytes / 4;
    unsigned int *d = static_cast<unsigned int *>(dst);
    Blob b;
    while (words > 0) {
        const size_t n = std::min<size_t>(words, BLOB_WORDS);
        b.n = (unsigned int)n;
        std::memcpy(b.w, w, n * 4);
        k_upload<<<1, 256, 0, s>>>(b, d);
        count_launch(1);
        w += n;
        d += n;
        words -= n;
    }
}

static Globals make_globals(const dressi_scene *sc, const dressi_params *p, const Plan &P, char *ws,
                            long long n_pix, int *status)
{
    Globals g;
    std::memset(&g, 0, sizeof(g));
    const Layout &L = P.lay;
    g.views = reinterpret_cast<const ViewK *>(ws + L.views);
    g.meshes = reinterpret_cast<const MeshK *>(ws + L.meshes);
    g.n_views = (int)P.views.size();
    g.K = p->K;
    g.edge_mode = p->edge_mode;
    g.shade_mode = p->shade_mode;
    g.tile = p->tile ? p->tile : TILE_DEFAULT;
    g.tile_shift = g.tile == 32 ? 5 : 4;
    g.tex_f16 = sc->tex_dtype == DRESSI_TEX_F16;
    g.texgrad_mode = p->texgrad_mode;
    g.n_verts_total = sc->n_verts_total;
    g.n_pix = n_pix;
    g.list_cap = L.list_cap;
    g.total_tiles = L.total_tiles;
    g.pos = sc->pos;
    g.col = sc->col;
    g.uv = sc->uv;
    g.faces = sc->faces;
    g.tex = sc->tex;
    g.ntex = sc->ntex;
    g.vrec = reinterpret_cast<VRec *>(ws + L.vrec);
    g.frec = reinterpret_cast<FaceRec *>(ws + L.frec);
    g.brect = reinterpret_cast<unsigned *>(ws + L.brect);
    g.tile_view = reinterpret_cast<int *>(ws + L.tile_view);
    g.tile_count = reinterpret_cast<int *>(ws + L.tile_count);
    g.tile_off = reinterpret_cast<int *>(ws + L.tile_off);
    g.tile_cursor = reinterpret_cast<int *>(ws + L.tile_cursor);
    g.lists = reinterpret_cast<int *>(ws + L.lists);
    g.nrm = reinterpret_cast<float4 *>(ws + L.nrm);
    g.adj_off = reinterpret_cast<int *>(ws + L.adj_off);
    g.adj_cur = reinterpret_cast<int *>(ws + L.adj_cur);
    g.adj = reinterpret_cast<int *>(ws + L.adj);
    g.scan_partial = reinterpret_cast<int *>(ws + L.scan_partial);
    g.sgrad = reinterpret_cast<float4 *>(ws + L.sgrad);
    g.ngrad = reinterpret_cast<float4 *>(ws + L.ngrad);
    g.status = status;
    g.persistent = p->schedule == 2;
    g.queue = reinterpret_cast<int *>(ws + L.queue);
    g.tile_order = nullptr;
    g.lpt_hist = reinterpret_cast<int *>(ws + L.lpt_hist);
    g.kth = nullptr;
    g.kth_flag = reinterpret_cast<int *>(ws + L.kth_flag);
    g.stats = g_stats;
    g.tg_keys = reinterpret_cast<unsigned *>(ws + L.tg_keys);
    g.tg_pay0 = reinterpret_cast<float4 *>(ws + L.tg_pay0);
    g.tg_pay1 = reinterpret_cast<float *>(ws + L.tg_pay1);
    g.inv_uv = reinterpret_cast<int *>(ws + L.inv_uv);
    g.uv_jx = p->uv_jitter[0];
    g.uv_jy = p->uv_jitter[1];
    g.n_texels_max_key = P.n_texels;
    return g;
}

// setup shared by both passes: tables, vertex transform, normals, binning
static void run_setup(Globals &g, const Plan &P, char *ws, bool need_bins, cudaStream_t s)
{
    const Layout &L = P.lay;
    // the view and mesh tables, adjacent in the workspace, in one upload
    std::vector<unsigned char> tables(L.meshes + sizeof(MeshK) * P.meshes.size(), 0);
    std::memcpy(tables.data() + L.views, P.views.data(), sizeof(ViewK) * P.views.size());
    std::memcpy(tables.data() + L.meshes, P.meshes.data(), sizeof(MeshK) * P.meshes.size());
    upload(tables.data(), tables.size(), ws + L.views, s);
    // the vertex transform also writes the tile -> view table and, before the face table
    // counts into them, clears the tile counters
    g.zero_bins = need_bins ? 1 : 0;
    launch_vertex(g, (int)P.views.size(), P.max_nv_view, s);
    launch_face(g, (int)P.views.size(), P.max_nf_view, need_bins, s);
    if (g.shade_mode >= 2) {
        const size_t nv = (size_t)std::max<long long>(g.n_verts_total, 1);
        cudaMemsetAsync(ws + L.adj_off, 0, sizeof(int) * (nv + 1), s);
        cudaMemsetAsync(ws + L.adj_cur, 0, sizeof(int) * nv, s);
        launch_normals(g, (int)P.meshes.size(), P.max_nf, P.max_nv, s);
    }
    if (need_bins) launch_bin(g, (int)P.views.size(), P.max_nf_view, s);
}

// a forward that stores no layer ids keeps every pixel's K-th (key, id) in the workspace
// for a re-rasterizing adjoint; the flag says whether the last forward did
static void keep_kth(Globals &g, const Plan &P, char *ws, cudaStream_t s)
{
    const bool keep = g.ids == nullptr;
    g.kth = keep ? reinterpret_cast<unsigned long long *>(ws + P.lay.kth) : nullptr;
    cudaMemsetAsync(ws + P.lay.kth_flag, keep ? 1 : 0, sizeof(int), s);
}

// the per-tile kernel, persistent (longest face list first when the lists exist) or
// one CTA per tile
static void run_tiles(Globals &g, const Plan &P, char *ws, bool bins_built, int pass, cudaStream_t s)
{
    if (g.persistent) {
        cudaMemsetAsync(ws + P.lay.queue, 0, sizeof(int) * 4, s);
        if (bins_built) {
            cudaMemsetAsync(ws + P.lay.lpt_hist, 0, sizeof(int) * LPT_BINS, s);
            g.tile_order = reinterpret_cast<const int *>(ws + P.lay.tile_order);
            launch_lpt_order(g, s);
            const size_t n = sizeof(int) * (size_t)P.lay.total_tiles;
            if (g_order_out) cudaMemcpyAsync(g_order_out, g.tile_order, n, cudaMemcpyDeviceToDevice, s);
            if (g_lengths_out) cudaMemcpyAsync(g_lengths_out, g.tile_count, n, cudaMemcpyDeviceToDevice, s);
        }
    }
    launch_tile_profiled(g, pass, s);
}

// ---------------------------------------------------------------------------
// static scratch for dressi_forward_static_scratch: callers that cannot allocate
// device memory get the workspace from this file-scope device array.  In host code
// the array's name is only a host-side stand-in, so its device address is looked up
// once per device (with that device current) and cached.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_static_scratch[DRESSI_STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
static void *g_static_scratch_addr[MAX_DEVICES] = {};
static std::mutex g_static_scratch_mu;

// device address of g_static_scratch on the current device, or nullptr on failure (the
// CUDA error of a failed lookup is cleared, so it does not surface in the caller's next
// CUDA call).  The address is cached per device ordinal: a cudaDeviceReset in the caller's
// process invalidates it (documented in dressi.h).
static void *static_scratch_address()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_static_scratch_mu);
    if (!g_static_scratch_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return nullptr;
        }
        g_static_scratch_addr[dev] = ptr;
    }
    return g_static_scratch_addr[dev];
}

}  // namespace dressi

using namespace dressi;

extern "C" {

int dressi_abi_version(void) { return DRESSI_ABI_VERSION; }

int dressi_set_profile_events(void *fwd_begin, void *fwd_end, void *bwd_begin, void *bwd_end)
{
    g_prof[0] = static_cast<cudaEvent_t>(fwd_begin);
    g_prof[1] = static_cast<cudaEvent_t>(fwd_end);
    g_prof[2] = static_cast<cudaEvent_t>(bwd_begin);
    g_prof[3] = static_cast<cudaEvent_t>(bwd_end);
    return DRESSI_OK;
}

unsigned long long dressi_launch_count(void) { return g_launches.load(); }

int dressi_set_inverse_uv_buffer(int32_t *dev_buffer)
{
    g_inv_uv_out = dev_buffer;
    return DRESSI_OK;
}

int dressi_set_tile_order_buffer(int32_t *dev_order, int32_t *dev_lengths)
{
    g_order_out = dev_order;
    g_lengths_out = dev_lengths;
    return DRESSI_OK;
}

int dressi_set_stats_buffer(void *dev_counters)
{
    g_stats = static_cast<unsigned long long *>(dev_counters);
    return DRESSI_OK;
}

const char *dressi_status_string(int code)
{
    switch (code) {
    case DRESSI_OK: return "ok";
    case DRESSI_ERR_ARG: return "invalid argument";
    case DRESSI_ERR_WORKSPACE: return "workspace missing or too small";
    case DRESSI_ERR_LAUNCH: return "CUDA launch failed";
    default: return "unknown return code";
    }
}

const char *dressi_dev_status_string(int bit)
{
    switch (bit) {
    case 0: return "ok";
    case DRESSI_DEV_TILE_OVERFLOW: return "tile list over capacity (exact fallback used)";
    case DRESSI_DEV_FACE_RANGE: return "face index out of range (face skipped)";
    case DRESSI_DEV_NONFINITE: return "non-finite vertex input (faces skipped)";
    default: return "unknown device status bit";
    }
}

size_t dressi_workspace_size(const dressi_scene *scene, const dressi_view *views, int32_t n_views,
                             const dressi_params *params)
{
    Plan P;
    if (!make_plan(scene, views, n_views, params, (long long)1 << 62, P)) return 0;
    return P.lay.total;
}

int dressi_forward(const dressi_scene *scene, const dressi_view *views, int32_t n_views,
                   const dressi_params *params, float *out_rgba, int32_t *layer_ids, int64_t n_pix, void *ws,
                   size_t ws_bytes, int32_t *dev_status, void *stream)
{
    Plan P;
    if (!out_rgba || !dev_status || n_pix < 1) return DRESSI_ERR_ARG;
    if (!make_plan(scene, views, n_views, params, n_pix, P)) return DRESSI_ERR_ARG;
    if (!ws || ws_bytes < P.lay.total) return DRESSI_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaGetLastError();
    char *w = static_cast<char *>(ws);
    Globals g = make_globals(scene, params, P, w, n_pix, dev_status);
    g.out = out_rgba;
    g.ids = layer_ids;
    keep_kth(g, P, w, s);
    run_setup(g, P, w, true, s);
    run_tiles(g, P, w, true, 0, s);
    return cudaGetLastError() == cudaSuccess ? DRESSI_OK : DRESSI_ERR_LAUNCH;
}

int dressi_forward_l2(const dressi_scene *scene, const dressi_view *views, int32_t n_views,
                      const dressi_params *params, const float *target, float *out_rgba, float *grad_rgba,
                      float *loss_accum, int32_t *layer_ids, int64_t n_pix, void *ws, size_t ws_bytes,
                      int32_t *dev_status, void *stream)
{
    Plan P;
    if (!target || !out_rgba || !grad_rgba || !dev_status || n_pix < 1) return DRESSI_ERR_ARG;
    if (((reinterpret_cast<uintptr_t>(target) | reinterpret_cast<uintptr_t>(out_rgba) |
          reinterpret_cast<uintptr_t>(grad_rgba)) & 15) != 0)
        return DRESSI_ERR_ARG;
    if (!make_plan(scene, views, n_views, params, n_pix, P)) return DRESSI_ERR_ARG;
    if (!ws || ws_bytes < P.lay.total) return DRESSI_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaGetLastError();
    char *w = static_cast<char *>(ws);
    Globals g = make_globals(scene, params, P, w, n_pix, dev_status);
    g.out = out_rgba;
    g.ids = layer_ids;
    g.l2_target = target;
    g.l2_grad = grad_rgba;
    g.l2_loss = loss_accum;
    keep_kth(g, P, w, s);
    run_setup(g, P, w, true, s);
    run_tiles(g, P, w, true, 0, s);
    return cudaGetLastError() == cudaSuccess ? DRESSI_OK : DRESSI_ERR_LAUNCH;
}

int dressi_forward_static_scratch(const dressi_scene *scene, const dressi_view *views, int32_t n_views,
                                  const dressi_params *params, float *out_rgba, int32_t *layer_ids, int64_t n_pix,
                                  int32_t *dev_status, void *stream)
{
    Plan P;
    if (!out_rgba || !dev_status || n_pix < 1) return DRESSI_ERR_ARG;
    if (!make_plan(scene, views, n_views, params, n_pix, P)) return DRESSI_ERR_ARG;
    if (P.lay.total > (size_t)DRESSI_STATIC_SCRATCH_BYTES) return DRESSI_ERR_WORKSPACE;
    void *ws = static_scratch_address();
    if (!ws) return DRESSI_ERR_LAUNCH;
    return dressi_forward(scene, views, n_views, params, out_rgba, layer_ids, n_pix, ws,
                          (size_t)DRESSI_STATIC_SCRATCH_BYTES, dev_status, stream);
}

int dressi_forward_from_layers(const dressi_scene *scene, const dressi_view *views, int32_t n_views,
                               const dressi_params *params, const int32_t *layer_ids, float *out_rgba, int64_t n_pix,
                               void *ws, size_t ws_bytes, int32_t *dev_status, void *stream)
{
    Plan P;
    if (!layer_ids || !out_rgba || !dev_status || n_pix < 1) return DRESSI_ERR_ARG;
    if (!make_plan(scene, views, n_views, params, n_pix, P)) return DRESSI_ERR_ARG;
    if (!ws || ws_bytes < P.lay.total) return DRESSI_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaGetLastError();
    char *w = static_cast<char *>(ws);
    Globals g = make_globals(scene, params, P, w, n_pix, dev_status);
    g.out = out_rgba;
    g.ids_in = layer_ids;
    cudaMemsetAsync(w + P.lay.kth_flag, 0, sizeof(int), s);   // no K-th keys from this pass
    // vertex records, face table and normals (shading needs them), no binning
    run_setup(g, P, w, false, s);
    run_tiles(g, P, w, false, 2, s);
    return cudaGetLastError() == cudaSuccess ? DRESSI_OK : DRESSI_ERR_LAUNCH;
}

int dressi_backward(const dressi_scene *scene, const dressi_view *views, int32_t n_views,
                    const dressi_params *params, const float *grad_rgba, const int32_t *layer_ids, int64_t n_pix,
                    float *grad_pos, float *grad_col, float *grad_tex, void *ws, size_t ws_bytes,
                    int32_t *dev_status, void *stream)
{
    return dressi_backward_ex(scene, views, n_views, params, grad_rgba, layer_ids, n_pix, grad_pos, grad_col, grad_tex,
                              nullptr, nullptr, nullptr, ws, ws_bytes, dev_status, stream);
}

int dressi_backward_ex(const dressi_scene *scene, const dressi_view *views, int32_t n_views,
                       const dressi_params *params, const float *grad_rgba, const int32_t *layer_ids, int64_t n_pix,
                       float *grad_pos, float *grad_col, float *grad_tex, float *grad_mvp, float *grad_light,
                       float *grad_ntex, void *ws, size_t ws_bytes, int32_t *dev_status, void *stream)
{
    Plan P;
    if (!grad_rgba || !grad_pos || !dev_status || n_pix < 1) return DRESSI_ERR_ARG;
    if (!make_plan(scene, views, n_views, params, n_pix, P)) return DRESSI_ERR_ARG;
    if (!ws || ws_bytes < P.lay.total) return DRESSI_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaGetLastError();
    char *w = static_cast<char *>(ws);
    Globals g = make_globals(scene, params, P, w, n_pix, dev_status);
    g.gin = grad_rgba;
    g.ids_in = layer_ids;
    g.gpos = grad_pos;
    g.gcol = params->shade_mode == 0 ? grad_col : nullptr;
    g.gtex = params->shade_mode != 0 ? grad_tex : nullptr;
    g.gmvp = grad_mvp;
    g.glight = grad_light;
    g.gntex = params->shade_mode == 3 ? grad_ntex : nullptr;
    if (g.gntex && P.n_texels > 0) cudaMemsetAsync(grad_ntex, 0, sizeof(float) * 4 * (size_t)P.n_texels, s);
    if (grad_mvp) cudaMemsetAsync(grad_mvp, 0, sizeof(float) * 16 * (size_t)n_views, s);
    if (grad_light) cudaMemsetAsync(grad_light, 0, sizeof(float) * 3 * (size_t)n_views, s);
    const long long nvt = scene->n_verts_total;
    cudaMemsetAsync(grad_pos, 0, sizeof(float) * 3 * (size_t)nvt, s);
    if (grad_col) cudaMemsetAsync(grad_col, 0, sizeof(float) * 3 * (size_t)nvt, s);
    if (grad_tex && P.n_texels > 0) cudaMemsetAsync(grad_tex, 0, sizeof(float) * 4 * (size_t)P.n_texels, s);
    cudaMemsetAsync(w + P.lay.sgrad, 0, sizeof(float4) * (size_t)std::max<long long>(P.lay.n_vrec, 1), s);
    if (params->shade_mode >= 2)
        cudaMemsetAsync(w + P.lay.ngrad, 0, sizeof(float4) * (size_t)std::max<long long>(nvt, 1), s);
    const bool tex_records = g.gtex && P.lay.tg_slots > 0;
    const bool gather = tex_records && params->texgrad_mode == 1;
    const bool inv_uv = tex_records && params->texgrad_mode == 2;
    if (!tex_records) g.texgrad_mode = 0;
    if (gather) cudaMemsetAsync(w + P.lay.tg_keys, 0xff, sizeof(unsigned) * (size_t)P.lay.tg_slots, s);
    if (inv_uv) cudaMemsetAsync(w + P.lay.inv_uv, 0xff, sizeof(int) * (size_t)P.n_texels, s);
    // re-rasterizing after a forward on this workspace: its K-th keys, if it kept them
    if (params->reuse_setup && !layer_ids) g.kth = reinterpret_cast<unsigned long long *>(w + P.lay.kth);
    if (!params->reuse_setup) run_setup(g, P, w, layer_ids == nullptr, s);
    run_tiles(g, P, w, layer_ids == nullptr, 1, s);
    if (gather)
        launch_tex_gather(g, P.lay.tg_slots, P.n_texels, (int)P.meshes.size(), P.max_texels, w + P.lay.tg_scratch,
                          ALIGN, s);
    if (inv_uv) {
        launch_inv_uv_apply(g, P.n_texels, s);
        if (g_inv_uv_out) cudaMemcpyAsync(g_inv_uv_out, g.inv_uv, sizeof(int) * (size_t)P.n_texels,
                                          cudaMemcpyDeviceToDevice, s);
    }
    launch_vertex_bwd(g, (int)P.views.size(), P.max_nv_view, (int)P.meshes.size(), P.max_nf,
                      params->shade_mode >= 2, s);
    return cudaGetLastError() == cudaSuccess ? DRESSI_OK : DRESSI_ERR_LAUNCH;
}

int dressi_autotune(const dressi_scene *scene, const dressi_view *views, int32_t n_views, dressi_params *params,
                    float *out_rgba, int32_t *layer_ids, int64_t n_pix, float *grad_pos, float *grad_col,
                    float *grad_tex, void *ws, size_t ws_bytes, int32_t *dev_status, void *stream, float *best_ms)
{
    if (!params || !out_rgba || !grad_pos || !dev_status || !ws) return DRESSI_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const dressi_params base = *params;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return DRESSI_ERR_LAUNCH;
    float best = 3.0e38f;
    dressi_params chosen = base;
    int rc = DRESSI_ERR_WORKSPACE;
    const int tiles[2] = {16, 32}, scheds[2] = {1, 2};
    for (int ti = 0; ti < 2; ++ti) {
        for (int si = 0; si < 2; ++si) {
            dressi_params p = base;
            p.tile = tiles[ti];
            p.schedule = scheds[si];
            p.list_cap = 0;
            Plan P;
            if (!make_plan(scene, views, n_views, &p, n_pix, P)) { rc = DRESSI_ERR_ARG; goto done; }
            if (P.lay.total > ws_bytes) continue;
            // the backward takes the forward's setup, as a training step does
            dressi_params pb = p;
            pb.reuse_setup = 1;
            float ms = 0.f;
            for (int rep = 0; rep < 5; ++rep) {   // two runs warm up, the best of the others counts
                cudaEventRecord(e0, s);
                int r1 = dressi_forward(scene, views, n_views, &p, out_rgba, layer_ids, n_pix, ws, ws_bytes,
                                        dev_status, stream);
                int r2 = r1 == DRESSI_OK ? dressi_backward(scene, views, n_views, &pb, out_rgba, layer_ids, n_pix,
                                                           grad_pos, grad_col, grad_tex, ws, ws_bytes, dev_status,
                                                           stream)
                                         : r1;
                cudaEventRecord(e1, s);
                if (r2 != DRESSI_OK) { rc = r2; goto done; }
                if (cudaEventSynchronize(e1) != cudaSuccess) { rc = DRESSI_ERR_LAUNCH; goto done; }
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep == 2 || (rep > 2 && t < ms)) ms = t;
            }
            rc = DRESSI_OK;
            if (ms < best) {
                // keep this choice and size its tile lists from the entries it needed
                // (the exclusive scan's last element, written by the last pass)
                best = ms;
                chosen = p;
                int total = 0;
                if (cudaMemcpy(&total, static_cast<char *>(ws) + P.lay.tile_off + sizeof(int) * P.lay.total_tiles,
                               sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
                    chosen.list_cap = (long long)total + total / 4 + 1024;
            }
        }
    }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == DRESSI_OK) {
        params->tile = chosen.tile;
        params->schedule = chosen.schedule;
        params->list_cap = chosen.list_cap;
        if (best_ms) *best_ms = best;
    }
    return rc;
}

int dressi_l2_loss_grad(const float *out, const float *target, int64_t n, float *grad, float *loss_accum,
                        void *stream)
{
    if (!out || !target || !grad || n < 0) return DRESSI_ERR_ARG;
    cudaGetLastError();
    if (n > 0) launch_l2(out, target, n, grad, loss_accum, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? DRESSI_OK : DRESSI_ERR_LAUNCH;
}

}  // extern "C"
