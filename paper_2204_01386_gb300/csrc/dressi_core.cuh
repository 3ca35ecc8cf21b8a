// dressi_core.cuh -- device-side data layout and the geometric core of HardSoftRas.
//
// Precision plan (GB300, FP32 pixel math):
//   * the vertex transform runs in FP64 with explicitly rounded operations, and
//     each pixel-space corner is kept as an unevaluated float pair hi + lo, so
//     that p - V is accurate to one float ulp of |p - V| (not of |V|): the
//     sigmoid of Sec. 3.4.3 is steep (sigma is a fraction of a pixel), so the
//     distance must be accurate to ~1e-7 px even at 2048^2;
//   * every geometric quantity of an edge is computed from its canonical
//     (lexicographically smaller) endpoint, so two faces sharing an edge or a
//     vertex get bit-identical distances and ties resolve by face id as in an
//     exact evaluation;
//   * the core uses __f*_rn intrinsics only, so the peel, the shading pass and
//     the adjoint (separate kernels and call sites) reproduce identical values.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dressi.h"

namespace dressi {

constexpr int MAXK = DRESSI_MAX_K;
constexpr int CHUNK = 128;   // faces staged in shared memory per round
constexpr int LPT_BINS = 1024;             // face-list lengths bucketed for the longest-first tile order
constexpr unsigned TG_NONE = 0xffffffffu;  // texel-gather record slot without a texture gradient
constexpr int FLAG_LIVE = 1 << 7;
// outside a face, its edge lines' signed distances F closer than this (pixels) count as a
// tie when choosing the edge that holds the closest point (far above their FP32 error)
constexpr float EDGE_TIE_PX = 1e-3f;
constexpr int FLAG_RANGE = 1 << 8;
constexpr int FLAG_ODD = 1 << 9;    // the record's corner order is an odd permutation of the face's

// ---------------------------------------------------------------------------
// tables uploaded into the workspace
// ---------------------------------------------------------------------------
struct ViewK {
    float mvp[16];
    float light[3];
    int mesh;
    int W, H, tiles_x, tiles_y;
    int tile_base;          // first global tile of this view
    int rho;                // edge-mask window radius (pixels)
    float r_px;             // r in pixels
    float inv_sigma_px;     // 1 / (sigma in pixels)
    float half_inv_S;       // 0.5 / max(W, H): soft key slope
    float bin_R;            // bin growth radius in pixels (max(r_px, rho) + guard)
    int pad;
    long long pix_off;
    long long vrec_off;     // first record of this view in the per-view vertex buffer
    long long slot_base;    // first pixel of this view in the texel-gather record slots
    long long frec_off;     // first record of this view in the per-view face table
};

struct MeshK {
    long long vert_off, face_off, tex_off;
    int nV, nF, tex_w, tex_h;
};

// per (view, vertex): pixel-space position as float pairs, depth, 1/w
struct __align__(16) VRec {
    float xh, xl, yh, yl;
    float z, iw;
    int valid;   // w > 1e-6 and depth in [0, 1] and finite
    int pad;
};

// per-face record used by every pixel evaluation.  28 words (112 bytes; word 19 holds
// the flags): staged in shared memory, the records of 8 consecutive faces fall into
// distinct banks for 16-byte loads.  The corners are kept in lexicographic order of their
// screen positions (xh, xl, yh, yl), so that the canonical (lexicographically smaller)
// endpoint of edge i -> i+1 is corner i for edges 0 and 1 and corner 0 for edge 2 (the
// swapped bits of the flags are always 0, 0, 1 for a live face): the evaluations pick no
// endpoints at run time.  FLAG_ODD records whether that order is an odd permutation of the
// face's own corner order (the normal map's tangent-frame handedness needs the latter).
// the geometric part (the first 20 words): all that SignedDist, the hard test and Shift
// read, and what the raster stages in shared memory
struct __align__(16) FaceGeo {
    float xh[3], xl[3], yh[3], yl[3];
    float invL[3];   // 1 / length of edge i (canonical), correctly rounded
    float z[3];
    float invA;      // 1 / |twice the signed area|
    int flags;       // bit 0: orient > 0; bits 1-3: edge i swapped; bits 4-6: edge i owns;
                     // FLAG_LIVE: not culled; FLAG_RANGE: a vertex index is out of range;
                     // FLAG_ODD: corners permuted oddly
};
static_assert(sizeof(FaceGeo) == 80, "FaceGeo is 20 words");

struct __align__(16) FaceRec : FaceGeo {
    int id;          // face index local to the mesh
    int vi[3];       // vertex indices local to the mesh
    float iw[3];     // 1 / w of the corners
    int pad;
};
static_assert(sizeof(FaceRec) == 112, "FaceRec is 28 words");

struct Globals {
    const ViewK *views;
    const MeshK *meshes;
    int n_views;
    int K;
    int edge_mode, shade_mode;
    int tile;            // tile edge in pixels
    int tile_shift;      // log2(tile)
    int tex_f16;
    int texgrad_mode;
    long long n_verts_total;
    long long n_pix;
    long long list_cap;
    int total_tiles;
    int pad0;
    const float *pos, *col, *uv;
    const int *faces;
    const void *tex;
    const void *ntex;     // shade_mode 3: normal map, laid out like tex
    VRec *vrec;
    FaceRec *frec;        // per (view, face): the face's record, written by the setup
    unsigned *brect;      // per (view, face): its binning tile rect, packed (pack_brect)
    int *tile_count, *tile_off, *tile_cursor, *lists;
    int *tile_view;       // [total_tiles] the view owning each tile
    float4 *nrm;          // [n_verts_total] normalized vertex normals, w = |sum|
    int *adj_off;         // [n_verts_total + 1] vertex -> incident faces (CSR offsets)
    int *adj_cur;         // [n_verts_total] fill cursors
    int *adj;             // [3 * faces] incident face ids (mesh-local)
    int *scan_partial;    // scratch of the device-wide scan
    int *status;
    // scheduling of the per-tile kernel
    int persistent;       // 1: persistent CTAs pull tiles from *queue
    int pad1;
    int *queue;           // tile queue head (zeroed before each pass)
    const int *tile_order;  // tiles by descending face-list length, or nullptr
    int *lpt_hist;        // [LPT_BINS] scratch of the ordering sort
    // the forward without stored layer ids keeps each pixel's K-th (key, id) here (per view
    // pixel, at slot_base + pixel; *kth_flag nonzero once it did); the re-rasterizing adjoint
    // that takes the forward's setup starts every K-list with it, so that pairs whose key
    // bound lies above it are culled from the start
    unsigned long long *kth;
    int *kth_flag;
    int zero_bins;        // the vertex transform clears tile_count and tile_cursor
    int pad2;
    // forward
    float *out;
    int *ids;             // [K][n_pix] or nullptr
    const float *l2_target;   // fused L2 loss: [n_pix][4] target, or nullptr
    float *l2_grad;       // [n_pix][4] 2 (out - target)
    float *l2_loss;       // sum of (out - target)^2 added here, or nullptr
    // backward
    const float *gin;
    const int *ids_in;    // [K][n_pix] or nullptr (recompute)
    float4 *sgrad;        // per (view, vertex): dX, dY, d(1/w)
    float4 *ngrad;        // [n_verts_total] gradient of the normalized vertex normals
    float *gpos, *gcol, *gtex;
    float *gmvp;          // [n_views][16] dL/dMVP or nullptr
    float *gntex;         // shade_mode 3: [sum texels][4] normal-map texel gradient or nullptr
    int *inv_uv;          // texgrad_mode 2: [sum texels] last sample written per texel (-1 none)
    float uv_jx, uv_jy;   // texgrad_mode 2: sample offset from the pixel centre
    float *glight;        // [n_views][3] dL/dlight or nullptr
    // texel-space gather of the texture gradient (texgrad_mode 1): one record per
    // (pixel, layer) at slot (slot_base + pixel) * K + layer
    unsigned long long *stats;  // optional work counters (see dressi_set_stats_buffer) or nullptr
    unsigned *tg_keys;
    float4 *tg_pay0;      // dL/dA (RGB), fx
    float *tg_pay1;       // fy
    long long n_texels_max_key;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool lex_less(float axh, float axl, float ayh, float ayl,
                                         float bxh, float bxl, float byh, float byl)
{
    if (axh != bxh) return axh < bxh;
    if (axl != bxl) return axl < bxl;
    if (ayh != byh) return ayh < byh;
    return ayl < byl;
}

__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Builds the record of face f of mesh m as seen in the view whose vertex
// records start at vr.  Returns false (live bit clear) for culled faces.
__device__ __forceinline__ bool face_load(const Globals &g, const MeshK &m, const VRec *vr, int f,
                                          FaceRec &R)
{
    R.id = f;
    R.flags = 0;
    if ((unsigned)f >= (unsigned)m.nF) {
        R.flags = FLAG_RANGE;
        return false;
    }
    const int *fv = g.faces + 3 * (m.face_off + f);
    int v0 = __ldg(fv), v1 = __ldg(fv + 1), v2 = __ldg(fv + 2);
    if ((unsigned)v0 >= (unsigned)m.nV || (unsigned)v1 >= (unsigned)m.nV || (unsigned)v2 >= (unsigned)m.nV) {
        R.flags = FLAG_RANGE;
        return false;
    }
    R.vi[0] = v0; R.vi[1] = v1; R.vi[2] = v2;
    // two 16-byte loads per corner, kept in scalars (an array of records would live in local memory)
    bool live = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float4 *rec = reinterpret_cast<const float4 *>(vr + R.vi[i]);
        const float4 p = rec[0], q = rec[1];
        R.xh[i] = p.x; R.xl[i] = p.y; R.yh[i] = p.z; R.yl[i] = p.w;
        R.z[i] = q.x; R.iw[i] = q.y;
        live = live && (__float_as_int(q.z) != 0);
    }
    // corners in lexicographic order (a three-element sorting network), counting the swaps
    bool odd = false;
    auto order = [&](int a, int b) {
        if (lex_less(R.xh[b], R.xl[b], R.yh[b], R.yl[b], R.xh[a], R.xl[a], R.yh[a], R.yl[a])) {
            float t;
            t = R.xh[a]; R.xh[a] = R.xh[b]; R.xh[b] = t;
            t = R.xl[a]; R.xl[a] = R.xl[b]; R.xl[b] = t;
            t = R.yh[a]; R.yh[a] = R.yh[b]; R.yh[b] = t;
            t = R.yl[a]; R.yl[a] = R.yl[b]; R.yl[b] = t;
            t = R.z[a]; R.z[a] = R.z[b]; R.z[b] = t;
            t = R.iw[a]; R.iw[a] = R.iw[b]; R.iw[b] = t;
            const int v = R.vi[a]; R.vi[a] = R.vi[b]; R.vi[b] = v;
            odd = !odd;
        }
    };
    order(0, 1);
    order(1, 2);
    order(0, 1);
    // twice the signed area from accurate corner differences
    const float ux = fadd(fsub(R.xh[1], R.xh[0]), fsub(R.xl[1], R.xl[0]));
    const float uy = fadd(fsub(R.yh[1], R.yh[0]), fsub(R.yl[1], R.yl[0]));
    const float wx = fadd(fsub(R.xh[2], R.xh[0]), fsub(R.xl[2], R.xl[0]));
    const float wy = fadd(fsub(R.yh[2], R.yh[0]), fsub(R.yl[2], R.yl[0]));
    const float A2 = ffma(ux, wy, -fmul(uy, wx));
    if (!(A2 != 0.f) || !isfinite(A2)) live = false;
    const bool orient = A2 > 0.f;
    int flags = orient ? 1 : 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int ia = i, ib = (i + 1) % 3;
        const bool sw = lex_less(R.xh[ib], R.xl[ib], R.yh[ib], R.yl[ib], R.xh[ia], R.xl[ia], R.yh[ia], R.yl[ia]);
        // canonical edge P -> Q
        const float Pxh = sw ? R.xh[ib] : R.xh[ia], Pxl = sw ? R.xl[ib] : R.xl[ia];
        const float Pyh = sw ? R.yh[ib] : R.yh[ia], Pyl = sw ? R.yl[ib] : R.yl[ia];
        const float Qxh = sw ? R.xh[ia] : R.xh[ib], Qxl = sw ? R.xl[ia] : R.xl[ib];
        const float Qyh = sw ? R.yh[ia] : R.yh[ib], Qyl = sw ? R.yl[ia] : R.yl[ib];
        const float ex = fadd(fsub(Qxh, Pxh), fsub(Qxl, Pxl));
        const float ey = fadd(fsub(Qyh, Pyh), fsub(Qyl, Pyl));
        const float L = __fsqrt_rn(ffma(ex, ex, fmul(ey, ey)));
        R.invL[i] = __fdiv_rn(1.f, L);
        // oriented edge ia -> ib
        const float eox = sw ? -ex : ex, eoy = sw ? -ey : ey;
        const bool owns = orient ? (eoy < 0.f || (eoy == 0.f && eox > 0.f)) : (eoy > 0.f || (eoy == 0.f && eox < 0.f));
        flags |= (sw ? 1 : 0) << (1 + i);
        flags |= (owns ? 1 : 0) << (4 + i);
    }
    R.invA = __fdiv_rn(1.f, fabsf(A2));
    if (live) flags |= FLAG_LIVE;
    if (odd) flags |= FLAG_ODD;
    R.flags = flags;
    return live;
}

// the (view, face) record of the face table (face_load's result, written once per call
// by the setup); false for a face out of range or culled, as face_load
__device__ __forceinline__ bool face_get(const Globals &g, const ViewK &V, const MeshK &m, int f, FaceRec &R)
{
    if ((unsigned)f >= (unsigned)m.nF) {
        R.id = f;
        R.flags = FLAG_RANGE;
        return false;
    }
    const float4 *src = reinterpret_cast<const float4 *>(g.frec + V.frec_off + f);
    float w[28];
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        const float4 q = __ldg(src + i);
        w[4 * i] = q.x; w[4 * i + 1] = q.y; w[4 * i + 2] = q.z; w[4 * i + 3] = q.w;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        R.xh[i] = w[i]; R.xl[i] = w[3 + i]; R.yh[i] = w[6 + i]; R.yl[i] = w[9 + i];
        R.invL[i] = w[12 + i]; R.z[i] = w[15 + i];
        R.vi[i] = __float_as_int(w[21 + i]); R.iw[i] = w[24 + i];
    }
    R.invA = w[18];
    R.flags = __float_as_int(w[19]);
    R.id = __float_as_int(w[20]);
    return (R.flags & FLAG_LIVE) != 0;
}

// a hint that the line holding address a will be read soon: fetch it into L2
__device__ __forceinline__ void prefetch_l2(const void *a)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// the geometric part of face_get into shared memory: five 16-byte copies
__device__ __forceinline__ bool face_stage(const Globals &g, const ViewK &V, const MeshK &m, int f, FaceGeo &dst)
{
    if ((unsigned)f >= (unsigned)m.nF) {
        dst.flags = FLAG_RANGE;
        return false;
    }
    const float4 *src = reinterpret_cast<const float4 *>(g.frec + V.frec_off + f);
    float4 *d = reinterpret_cast<float4 *>(&dst);
    int flags = 0;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float4 q = __ldg(src + i);
        d[i] = q;
        if (i == 4) flags = __float_as_int(q.w);   // word 19
    }
    return (flags & FLAG_LIVE) != 0;
}

// the record of face f with its geometric part taken from a staged copy: the rest (id,
// vertex indices, 1/w) from the face table
__device__ __forceinline__ void face_complete(const Globals &g, const ViewK &V, int f, const FaceGeo &geo, FaceRec &R)
{
    static_cast<FaceGeo &>(R) = geo;
    const float4 *src = reinterpret_cast<const float4 *>(g.frec + V.frec_off + f);
    const float4 a = __ldg(src + 5), b = __ldg(src + 6);
    R.id = __float_as_int(a.x);
    R.vi[0] = __float_as_int(a.y); R.vi[1] = __float_as_int(a.z); R.vi[2] = __float_as_int(a.w);
    R.iw[0] = b.x; R.iw[1] = b.y; R.iw[2] = b.z;
}

// Result of evaluating one face at one pixel centre.
struct Frag {
    float dist;      // signed pixel distance (positive inside the hard face)
    float key;       // Shift() key
    float Fn[3];     // oriented edge numerators: lam_{(i+2)%3} = Fn[i] * invA
    float t;         // soft fragment on edge `feat`: closest point = P + t (Q - P), canonical P, Q
    int hard;
    int feat;        // 0..2: edge i interior; 3..5: corner (feat - 3)
};

// SignedDist, candidate rule, hard test (top-left fill rule) and Shift (Eq. Shift) of
// face R at pixel centre (px, py).  Returns false when the face is not a candidate
// (farther than r_px outside).  Pure function of (R, px, py, r_px, half_inv_S).
// Every array index below is a compile-time constant (canonical endpoints are
// chosen by selects), so nothing spills to local memory.  An edge distance is the
// canonical cross product times the record's 1/L and a corner distance the square
// root at the shared corner, so the faces around a shared edge or corner compute
// bit-identical distances to it.
// With LAMBDA false the closest point's parameter o.t is left at 0: the peel needs the
// key alone, shading and the adjoint re-evaluate the kept layers with LAMBDA.
template <bool LAMBDA = true>
__device__ __forceinline__ bool eval_face(const FaceGeo &R, float px, float py, float r_px, float half_inv_S,
                                          Frag &o)
{
    float dx[3], dy[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dx[i] = fsub(fsub(px, R.xh[i]), R.xl[i]);
        dy[i] = fsub(fsub(py, R.yh[i]), R.yl[i]);
    }
    const bool orient = R.flags & 1;
    // canonical endpoint offsets p - P and p - Q of every edge
    float pX[3], pY[3], qX[3], qY[3], c[3], F[3];
    bool early_out = false;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const bool sw = i == 2;   // corners in lexicographic order
        const int ia = i, ib = (i + 1) % 3;
        pX[i] = sw ? dx[ib] : dx[ia]; pY[i] = sw ? dy[ib] : dy[ia];
        qX[i] = sw ? dx[ia] : dx[ib]; qY[i] = sw ? dy[ia] : dy[ib];
        // cross(Q - P, p - P) == cross(p - P, p - Q)
        c[i] = ffma(pX[i], qY[i], -fmul(pY[i], qX[i]));
        const float fn = (orient != sw) ? c[i] : -c[i];
        o.Fn[i] = fn;
        F[i] = fmul(fn, R.invL[i]);
        early_out |= F[i] < -r_px;
    }
    if (early_out) return false;
    bool inside = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const bool owns = (R.flags >> (4 + i)) & 1;
        inside &= (o.Fn[i] > 0.f) || (o.Fn[i] == 0.f && owns);
    }
    float dist, bt = 0.f;
    int feat;
    // the edge whose line the pixel is farthest outside of (smallest F), and the gap to
    // the next smallest
    int emin = 0;
    float fmin1 = F[0];
    if (F[1] < fmin1) { emin = 1; fmin1 = F[1]; }
    if (F[2] < fmin1) { emin = 2; fmin1 = F[2]; }
    if (inside) {
        feat = emin;
        dist = fmin1;
    } else {
        // Outside, the closest point of the triangle lies on the edge with the smallest F
        // (its interior, or one of its endpoints).  That edge alone is measured unless
        // the two smallest F are within EDGE_TIE_PX of each other (slivers, where rounding
        // could swap them): then every edge is, and the closest taken.
        const float fmid = emin == 0 ? fminf(F[1], F[2]) : (emin == 1 ? fminf(F[0], F[2]) : fminf(F[0], F[1]));
        const bool single = fsub(fmid, fmin1) > EDGE_TIE_PX;
        // squared distances compared without branches; one square root for a corner
        float best2 = 3.4e38f, bsel = -1.f, btn = 0.f, btd = 1.f;
        feat = 0;
        if (single) {
            const int i = emin;
            const float Pxi = i == 0 ? pX[0] : (i == 1 ? pX[1] : pX[2]);
            const float Pyi = i == 0 ? pY[0] : (i == 1 ? pY[1] : pY[2]);
            const float Qxi = i == 0 ? qX[0] : (i == 1 ? qX[1] : qX[2]);
            const float Qyi = i == 0 ? qY[0] : (i == 1 ? qY[1] : qY[2]);
            const float ci = i == 0 ? c[0] : (i == 1 ? c[1] : c[2]);
            const float iLi = i == 0 ? R.invL[0] : (i == 1 ? R.invL[1] : R.invL[2]);
            const bool sw = i == 2;   // corners in lexicographic order
            const int ia = i, ib = i == 2 ? 0 : i + 1;
            const float ex = fsub(Pxi, Qxi), ey = fsub(Pyi, Qyi);   // V_Q - V_P
            const float tP = ffma(Pxi, ex, fmul(Pyi, ey));
            const float tQ = ffma(Qxi, ex, fmul(Qyi, ey));
            const bool atP = tP <= 0.f, atQ = !atP && tQ >= 0.f;
            const float cx = atQ ? Qxi : Pxi, cy = atQ ? Qyi : Pyi;
            best2 = ffma(cx, cx, fmul(cy, cy));
            feat = atP ? 3 + (sw ? ib : ia) : atQ ? 3 + (sw ? ia : ib) : i;
            bsel = (atP || atQ) ? -1.f : fmul(fabsf(ci), iLi);
            btn = tP;
            btd = ffma(ex, ex, fmul(ey, ey));
        } else {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const bool sw = i == 2;   // corners in lexicographic order
                const int ia = i, ib = (i + 1) % 3;
                const float ex = fsub(pX[i], qX[i]), ey = fsub(pY[i], qY[i]);   // V_Q - V_P
                const float tP = ffma(pX[i], ex, fmul(pY[i], ey));
                const float tQ = ffma(qX[i], ex, fmul(qY[i], ey));
                const float dP2 = ffma(pX[i], pX[i], fmul(pY[i], pY[i]));
                const float dQ2 = ffma(qX[i], qX[i], fmul(qY[i], qY[i]));
                const float se = fmul(fabsf(c[i]), R.invL[i]);
                const bool atP = tP <= 0.f, atQ = !atP && tQ >= 0.f;
                const float s2 = atP ? dP2 : atQ ? dQ2 : fmul(se, se);
                const int ft = atP ? 3 + (sw ? ib : ia) : atQ ? 3 + (sw ? ia : ib) : i;
                if (s2 < best2) {
                    best2 = s2; feat = ft; bsel = (atP || atQ) ? -1.f : se;
                    btn = tP; btd = ffma(ex, ex, fmul(ey, ey));
                }
            }
        }
        // edge interior: the closest point's parameter along the edge
        if (LAMBDA && feat < 3) bt = __fdiv_rn(btn, btd);
        dist = -(bsel >= 0.f ? bsel : __fsqrt_rn(best2));
    }
    if (!(dist >= -r_px)) return false;
    o.dist = dist;
    o.hard = inside;
    o.feat = feat;
    o.t = bt;
    if (inside) {
        // z(p) = sum lam_j z_j,  lam_{(i+2)%3} = Fn[i] / |A2|
        float zs = ffma(o.Fn[1], R.z[0], ffma(o.Fn[2], R.z[1], fmul(o.Fn[0], R.z[2])));
        o.key = fmul(0.5f, fmul(zs, R.invA));
    } else {
        o.key = ffma(-dist, half_inv_S, 0.5f);
    }
    return true;
}

// Screen-space barycentrics of a fragment: area ratios inside the hard face; for a
// soft fragment those of its closest point of the hard face (a corner, or the point
// at parameter t along the canonical edge P -> Q).
__device__ __forceinline__ void frag_lambda(const FaceGeo &R, const Frag &fr, float lam[3])
{
    if (fr.hard) {
        lam[0] = fmul(fr.Fn[1], R.invA);
        lam[1] = fmul(fr.Fn[2], R.invA);
        lam[2] = fmul(fr.Fn[0], R.invA);
        return;
    }
    if (fr.feat >= 3) {
#pragma unroll
        for (int j = 0; j < 3; ++j) lam[j] = (j == fr.feat - 3) ? 1.f : 0.f;
        return;
    }
    const int i = fr.feat;
    const bool sw = i == 2;   // corners in lexicographic order
    const int P = sw ? (i + 1) % 3 : i, Q = sw ? i : (i + 1) % 3;
#pragma unroll
    for (int j = 0; j < 3; ++j) lam[j] = (j == P) ? fsub(1.f, fr.t) : ((j == Q) ? fr.t : 0.f);
}

// Hard test only (for S^H of halo pixels): true if p lies in the closed face under
// the fill rule.
__device__ __forceinline__ bool hard_test(const FaceGeo &R, float px, float py)
{
    float dx[3], dy[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dx[i] = fsub(fsub(px, R.xh[i]), R.xl[i]);
        dy[i] = fsub(fsub(py, R.yh[i]), R.yl[i]);
    }
    const bool orient = R.flags & 1;
    bool inside = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const bool sw = i == 2;   // corners in lexicographic order
        const int ia = i, ib = (i + 1) % 3;
        const float pX = sw ? dx[ib] : dx[ia], pY = sw ? dy[ib] : dy[ia];
        const float qX = sw ? dx[ia] : dx[ib], qY = sw ? dy[ia] : dy[ib];
        const float c = ffma(pX, qY, -fmul(pY, qX));
        const float fn = (orient != sw) ? c : -c;
        const bool owns = (R.flags >> (4 + i)) & 1;
        inside &= (fn > 0.f) || (fn == 0.f && owns);
    }
    return inside;
}

// 1 / (1 + exp(-x)) from e = exp(-|x|) <= 1 (no overflow): 1 / (1 + e) for x >= 0, e / (1 + e)
// below; the exponential and the division are the fast hardware forms (a few ulp)
__device__ __forceinline__ float sigmoidf_stable(float x)
{
    const float e = __expf(-fabsf(x));
    const float s = __fdividef(1.f, 1.f + e);
    return x >= 0.f ? s : e * s;
}

}  // namespace dressi
