// dressi_tile.cuh -- the per-tile hot kernel of HardSoftRas, forward and adjoint
// (included by one translation unit per mode: dressi_tile_fwd.cu, _bwd.cu, _ids.cu,
// _cached.cu, _extra_ids.cu, _extra_bwd.cu, _nmap_fwd.cu, _nmap_cached.cu).
//
// One CTA owns one TT x TT pixel tile of one view (TT = 16 or 32; 256 threads).  Per CTA:
//   1. the tile's face list is staged in shared memory, CH faces at a time, from the
//      per-(view, face) record table (the 80-byte geometric part of each record), with
//      tile-local edge equations for a cheap conservative pretest; the next round's
//      records are prefetched into L2;
//   2. every (face, 4-pixel row segment) item of the faces' r-grown bounding boxes is
//      enumerated (item -> face through a per-32-item table); warps take 32 items at a
//      time, the pixels passing the pretest and the key lower bound go to the warp's own
//      queue, and the queue gets the exact SignedDist, hard test and Shift key with full
//      warps; each pixel keeps its K smallest (key, id) pairs in shared memory (depth
//      peeling of Alg. 2 as a per-pixel K-selection, the rows of K-lists rotated so that
//      neighbouring pixels use different banks; the re-rasterizing adjoint starts from
//      the forward's K-th pair when the forward kept it);
//   3. the hard stencil S^H of a ring of rho pixels around the tile is built from the
//      same staged faces (hard test only), so the edge mask E of every tile pixel is
//      known without a second pass over the image;
//   4. forward: each warp re-evaluates and shades (perspective-correct interpolation,
//      bilinear texture, Lambert or normal map) the layers its pixels blend as one list,
//      and each pixel blends them (D_k = sigmoid(dist/sigma), colour and silhouette
//      equations of Sec. 3.4.3), optionally with the L2 loss; adjoint: the same values are
//      rebuilt, by warp lists (re-rasterizing) or a CTA-wide layer queue (stored ids), and
//      dL/dI is pushed back to the screen-space corners, vertex colours, vertex normals,
//      texels, the camera and the light.
// With layer ids stored by the forward (modes 2, 3, 4, 7), steps 1-3 are skipped: S^H of
// the tile and its ring is the stored front layer's hard flag.
#pragma once
#include "dressi_core.cuh"
#include "dressi_launch.h"

#include <algorithm>
#include <atomic>
#include <mutex>

namespace dressi {

constexpr int NT = 256;                // threads per CTA
constexpr int TT_MAX = 32;             // tile edges: 16 (one pixel per thread) or 32 (four)
constexpr int RHO_MAX = 8;             // largest supported edge-mask radius
constexpr int HS_MAX = TT_MAX + 2 * RHO_MAX;
constexpr float APPROX_EPS = 1e-3f;    // pixel slack of the tile-local (approximate) edge equations
constexpr int CH = 128;                // faces staged per round (one per thread)
constexpr int HASH = 256;              // face id -> staged slot, open addressing (2 CH: at most half full)
constexpr unsigned long long EMPTY = ~0ULL;
constexpr int WQ = 160;                // a warp's queue of pretested pairs (31 waiting + 32 items x 4)
constexpr int QN = NT / 32 * WQ;       // the CTA's warp queues
constexpr int NBLK = 1024;             // pair blocks of 32 with a table entry (32,768 items)

// conservative tile-local data of a staged face: edge equations in pixels relative to
// the tile origin (FP32, a few 1e-6 px of error) and the smallest corner depth.  12 words:
// the records of 8 consecutive faces fall into distinct banks for 16-byte loads.
struct Pre {
    float nx[3], ny[3], c[3];    // F_i(p) ~ nx p.x + ny p.y + c, inward unit normal
    float zmin;
    float pad[2];
};
static_assert(sizeof(Pre) == 48, "Pre is 12 words");

// the face's bounding box in tile-local pixels, grown by r
struct Box {
    float bx0, bx1, by0, by1;
};

__device__ __forceinline__ void make_pre(const FaceGeo &R, bool live, float tx0, float ty0, float r_px, Pre &P, Box &B)
{
    if (!live) {
        B.bx0 = 3.0e38f; B.bx1 = -3.0e38f; B.by0 = 3.0e38f; B.by1 = -3.0e38f;
#pragma unroll
        for (int i = 0; i < 3; ++i) { P.nx[i] = 0.f; P.ny[i] = 0.f; P.c[i] = -3.0e38f; }
        P.zmin = 3.0e38f;
        return;
    }
    const bool orient = R.flags & 1;
    float vx[3], vy[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        vx[i] = (R.xh[i] - tx0) + R.xl[i];
        vy[i] = (R.yh[i] - ty0) + R.yl[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int ib = (i + 1) % 3;
        const float ex = vx[ib] - vx[i], ey = vy[ib] - vy[i];
        float nx = orient ? -ey : ey, ny = orient ? ex : -ex;
        // 1 / |edge| of the record (same edge, accurate corners): within a few ulp of
        // this edge's own length, far inside the pretest's slack
        const float s = isfinite(R.invL[i]) ? R.invL[i] : 0.f;
        nx *= s; ny *= s;
        P.nx[i] = nx; P.ny[i] = ny;
        P.c[i] = -(nx * vx[i] + ny * vy[i]);
    }
    B.bx0 = fminf(vx[0], fminf(vx[1], vx[2])) - r_px;
    B.bx1 = fmaxf(vx[0], fmaxf(vx[1], vx[2])) + r_px;
    B.by0 = fminf(vy[0], fminf(vy[1], vy[2])) - r_px;
    B.by1 = fmaxf(vy[0], fmaxf(vy[1], vy[2])) + r_px;
    P.zmin = fminf(R.z[0], fminf(R.z[1], R.z[2]));
}

// smallest approximate edge value of the face at one tile-local pixel centre
__device__ __forceinline__ float approx_fmin(const Pre &P, float lx, float ly)
{
    const float f0 = fmaf(P.nx[0], lx, fmaf(P.ny[0], ly, P.c[0]));
    const float f1 = fmaf(P.nx[1], lx, fmaf(P.ny[1], ly, P.c[1]));
    const float f2 = fmaf(P.nx[2], lx, fmaf(P.ny[2], ly, P.c[2]));
    return fminf(f0, fminf(f1, f2));
}

// ---------------------------------------------------------------------------
// per-layer shading (Sec. 3.3.2 texture sampling, Sec. 3.4.3 shading)
// ---------------------------------------------------------------------------
struct Shade {
    int vi[3];
    float iw[3];
    int odd;              // the record's corner order is an odd permutation of the face's
    float lam[3], b[3], Q;
    float C[3];
    float D;
    // texture
    int ix[2], iy[2];
    float fx, fy;
    float A[3];
    float Xt[3], Yt[3];   // texel-space corner coordinates relative to corner 0
    // Lambert
    float n[3], mlen, ndl;
    float np[3];          // the shading normal: n, or the normal-mapped n' (shade_mode 3)
};

__device__ __forceinline__ float4 load_texel(const Globals &g, long long idx)
{
    if (g.tex_f16) {
        uint2 raw = __ldg(reinterpret_cast<const uint2 *>(g.tex) + idx);
        __half2 a = *reinterpret_cast<__half2 *>(&raw.x), b = *reinterpret_cast<__half2 *>(&raw.y);
        float2 fa = __half22float2(a), fb = __half22float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
    return __ldg(reinterpret_cast<const float4 *>(g.tex) + idx);
}

__device__ __forceinline__ float4 load_ntexel(const Globals &g, long long idx)
{
    if (g.tex_f16) {
        uint2 raw = __ldg(reinterpret_cast<const uint2 *>(g.ntex) + idx);
        __half2 a = *reinterpret_cast<__half2 *>(&raw.x), b = *reinterpret_cast<__half2 *>(&raw.y);
        float2 fa = __half22float2(a), fb = __half22float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
    return __ldg(reinterpret_cast<const float4 *>(g.ntex) + idx);
}

__device__ __forceinline__ int wrapi(int i, int n)
{
    int m = i % n;
    return m < 0 ? m + n : m;
}

// texel coordinate x = (sum b_i u_i) W - 1/2 without losing the fraction at large W:
// corners as exact float pairs u_i W = hi_i + lo_i, offsets from corner 0 carry
// the barycentric mix, the floor is split off exactly.
__device__ __forceinline__ void texcoord(const float b[3], const float u[3], float Wt, int &i0, float &f, float rel[3])
{
    float hi[3], lo[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        hi[i] = fmul(u[i], Wt);
        lo[i] = ffma(u[i], Wt, -hi[i]);
    }
    rel[0] = 0.f;
    rel[1] = fadd(fsub(hi[1], hi[0]), fsub(lo[1], lo[0]));
    rel[2] = fadd(fsub(hi[2], hi[0]), fsub(lo[2], lo[0]));
    const float delta = ffma(b[1], rel[1], ffma(b[2], rel[2], lo[0]));
    const float A = fsub(hi[0], 0.5f);
    const float fA = floorf(A);
    const float t = fadd(fsub(A, fA), delta);
    const float ft = floorf(t);
    f = fsub(t, ft);
    i0 = (int)fA + (int)ft;
}

// normal map (shade_mode 3): the face's tangent frame and the mapped normal at the
// layer's sample.  Tf = (e1 dv2 - e2 dv1) / det from the object-space edges and UV
// differences, T' = normalize(Tf - n (n . Tf)), B' = h n x T' (h the sign of det); the
// map value t decodes to nt = 2 t - 1 and n' = m' / |m'|, m' = nt0 T' + nt1 B' + nt2 n.
// The adjoint rebuilds this from the same inputs.
struct NMap {
    float Tf[3], Tp[3], Bp[3], nt[3], np[3];
    float tl, mpl, h, idet, dv1, dv2, nT;
    float t00[3], t10[3], t01[3], t11[3];   // the four map texels (for the UV gradient)
};

__device__ __forceinline__ void nmap_eval(const Globals &g, const MeshK &M, const Shade &S, const float u[3],
                                          const float v[3], NMap &N)
{
    const long long nvt = g.n_verts_total;
    float P[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) P[i][c] = __ldg(g.pos + c * nvt + M.vert_off + S.vi[i]);
    const float du1 = fsub(u[1], u[0]), du2 = fsub(u[2], u[0]);
    N.dv1 = fsub(v[1], v[0]);
    N.dv2 = fsub(v[2], v[0]);
    const float det = fsub(fmul(du1, N.dv2), fmul(du2, N.dv1));
    N.idet = det != 0.f ? __fdiv_rn(1.f, det) : 0.f;
    // the handedness of the face's own corner order (the record's is that or its mirror)
    N.h = ((det < 0.f) != (S.odd != 0)) ? -1.f : 1.f;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        N.Tf[c] = fmul(fsub(fmul(fsub(P[1][c], P[0][c]), N.dv2), fmul(fsub(P[2][c], P[0][c]), N.dv1)), N.idet);
    N.nT = ffma(S.n[2], N.Tf[2], ffma(S.n[1], N.Tf[1], fmul(S.n[0], N.Tf[0])));
    float tau[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) tau[c] = ffma(-S.n[c], N.nT, N.Tf[c]);
    N.tl = __fsqrt_rn(ffma(tau[2], tau[2], ffma(tau[1], tau[1], fmul(tau[0], tau[0]))));
    const float itl = N.tl > 0.f ? __fdiv_rn(1.f, N.tl) : 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) N.Tp[c] = fmul(tau[c], itl);
    N.Bp[0] = fmul(N.h, fsub(fmul(S.n[1], N.Tp[2]), fmul(S.n[2], N.Tp[1])));
    N.Bp[1] = fmul(N.h, fsub(fmul(S.n[2], N.Tp[0]), fmul(S.n[0], N.Tp[2])));
    N.Bp[2] = fmul(N.h, fsub(fmul(S.n[0], N.Tp[1]), fmul(S.n[1], N.Tp[0])));
    const long long tb = M.tex_off;
    const float4 a00 = load_ntexel(g, tb + (long long)S.iy[0] * M.tex_w + S.ix[0]);
    const float4 a10 = load_ntexel(g, tb + (long long)S.iy[0] * M.tex_w + S.ix[1]);
    const float4 a01 = load_ntexel(g, tb + (long long)S.iy[1] * M.tex_w + S.ix[0]);
    const float4 a11 = load_ntexel(g, tb + (long long)S.iy[1] * M.tex_w + S.ix[1]);
    N.t00[0] = a00.x; N.t00[1] = a00.y; N.t00[2] = a00.z;
    N.t10[0] = a10.x; N.t10[1] = a10.y; N.t10[2] = a10.z;
    N.t01[0] = a01.x; N.t01[1] = a01.y; N.t01[2] = a01.z;
    N.t11[0] = a11.x; N.t11[1] = a11.y; N.t11[2] = a11.z;
    const float gx = fsub(1.f, S.fx), gy = fsub(1.f, S.fy);
    const float w00 = fmul(gx, gy), w10 = fmul(S.fx, gy), w01 = fmul(gx, S.fy), w11 = fmul(S.fx, S.fy);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float t = ffma(w11, N.t11[c], ffma(w01, N.t01[c], ffma(w10, N.t10[c], fmul(w00, N.t00[c]))));
        N.nt[c] = ffma(2.f, t, -1.f);
    }
    float mp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) mp[c] = ffma(N.nt[2], S.n[c], ffma(N.nt[1], N.Bp[c], fmul(N.nt[0], N.Tp[c])));
    N.mpl = __fsqrt_rn(ffma(mp[2], mp[2], ffma(mp[1], mp[1], fmul(mp[0], mp[0]))));
    const float iml = N.mpl > 0.f ? __fdiv_rn(1.f, N.mpl) : 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) N.np[c] = fmul(mp[c], iml);
}

// b, C, D and the sampling state of one layer from S.vi, S.iw, S.lam and dist.  Every
// operation is rounded as written (no contraction left to the compiler), so the kernels
// that shade a layer -- forward, forward from stored layers, adjoint -- agree bit for bit.
// The reciprocals of the barycentric sum and of the normal's length, and the sigmoid's
// exponential and division, are the fast hardware approximations (a few ulp, far inside the
// 1e-5 image tolerance): this function runs for every shaded layer in every pass.
// X: the kernel has the normal map compiled in (the kernels without it stay lean)
template <bool X>
__device__ __forceinline__ void shade(const Globals &g, const ViewK &V, const MeshK &M, float dist, Shade &S)
{
    float q[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) q[i] = fmul(S.lam[i], S.iw[i]);
    S.Q = fadd(fadd(q[0], q[1]), q[2]);
    const float iQ = __fdividef(1.f, S.Q);   // 2 ulp
#pragma unroll
    for (int i = 0; i < 3; ++i) S.b[i] = fmul(q[i], iQ);
    S.D = sigmoidf_stable(fmul(dist, V.inv_sigma_px));
    const long long nvt = g.n_verts_total;
    if (g.shade_mode == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float a = 0.f;
#pragma unroll
            for (int i = 0; i < 3; ++i) a = ffma(S.b[i], __ldg(g.col + c * nvt + M.vert_off + S.vi[i]), a);
            S.C[c] = a;
        }
        return;
    }
    float u[3], v[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        u[i] = __ldg(g.uv + M.vert_off + S.vi[i]);
        v[i] = __ldg(g.uv + nvt + M.vert_off + S.vi[i]);
    }
    int x0, y0;
    texcoord(S.b, u, (float)M.tex_w, x0, S.fx, S.Xt);
    texcoord(S.b, v, (float)M.tex_h, y0, S.fy, S.Yt);
    S.ix[0] = wrapi(x0, M.tex_w); S.ix[1] = wrapi(x0 + 1, M.tex_w);
    S.iy[0] = wrapi(y0, M.tex_h); S.iy[1] = wrapi(y0 + 1, M.tex_h);
    const long long tb = M.tex_off;
    const float4 t00 = load_texel(g, tb + (long long)S.iy[0] * M.tex_w + S.ix[0]);
    const float4 t10 = load_texel(g, tb + (long long)S.iy[0] * M.tex_w + S.ix[1]);
    const float4 t01 = load_texel(g, tb + (long long)S.iy[1] * M.tex_w + S.ix[0]);
    const float4 t11 = load_texel(g, tb + (long long)S.iy[1] * M.tex_w + S.ix[1]);
    const float gx = fsub(1.f, S.fx), gy = fsub(1.f, S.fy);
    const float w00 = fmul(gx, gy), w10 = fmul(S.fx, gy), w01 = fmul(gx, S.fy), w11 = fmul(S.fx, S.fy);
    S.A[0] = ffma(w11, t11.x, ffma(w01, t01.x, ffma(w10, t10.x, fmul(w00, t00.x))));
    S.A[1] = ffma(w11, t11.y, ffma(w01, t01.y, ffma(w10, t10.y, fmul(w00, t00.y))));
    S.A[2] = ffma(w11, t11.z, ffma(w01, t01.z, ffma(w10, t10.z, fmul(w00, t00.z))));
    if (g.shade_mode == 1) {
        S.C[0] = S.A[0]; S.C[1] = S.A[1]; S.C[2] = S.A[2];
        return;
    }
    float m[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float4 nv = g.nrm[M.vert_off + S.vi[i]];
        m[0] = ffma(S.b[i], nv.x, m[0]);
        m[1] = ffma(S.b[i], nv.y, m[1]);
        m[2] = ffma(S.b[i], nv.z, m[2]);
    }
    const float m2 = ffma(m[0], m[0], ffma(m[1], m[1], fmul(m[2], m[2])));
    const float il = m2 > 0.f ? rsqrtf(m2) : 0.f;   // 2 ulp
    S.mlen = fmul(m2, il);
    S.n[0] = fmul(m[0], il); S.n[1] = fmul(m[1], il); S.n[2] = fmul(m[2], il);
    S.np[0] = S.n[0]; S.np[1] = S.n[1]; S.np[2] = S.n[2];
    if (X && g.shade_mode == 3) {
        NMap N;
        nmap_eval(g, M, S, u, v, N);
        S.np[0] = N.np[0]; S.np[1] = N.np[1]; S.np[2] = N.np[2];
    }
    S.ndl = ffma(S.np[2], V.light[2], ffma(S.np[1], V.light[1], fmul(S.np[0], V.light[0])));
    const float sl = fmaxf(S.ndl, 0.f);
    S.C[0] = fmul(S.A[0], sl); S.C[1] = fmul(S.A[1], sl); S.C[2] = fmul(S.A[2], sl);
}

// a layer rebuilt from its face id (adjoint): record, fragment, shading
struct Layer {
    FaceRec R;
    Frag fr;
    Shade S;
};

template <bool X>
__device__ __forceinline__ bool layer_build(const Globals &g, const ViewK &V, const MeshK &M, int id,
                                            float px, float py, Layer &L)
{
    if (!face_get(g, V, M, id, L.R)) return false;
    if (!eval_face(L.R, px, py, V.r_px, V.half_inv_S, L.fr)) return false;
    frag_lambda(L.R, L.fr, L.S.lam);
#pragma unroll
    for (int i = 0; i < 3; ++i) { L.S.vi[i] = L.R.vi[i]; L.S.iw[i] = L.R.iw[i]; }
    L.S.odd = (L.R.flags & FLAG_ODD) != 0;
    shade<X>(g, V, M, L.fr.dist, L.S);
    return true;
}

// ---------------------------------------------------------------------------
// adjoint of one layer: gC = dL/dC_k, gD = dL/dD_k
// ---------------------------------------------------------------------------
// gl: this thread's dL/dlight accumulator, or nullptr.  Returns true when it stored
// the sample's dL/d(albedo) in its record slot (texgrad_mode 2, the inverse UV).  EXTRA
// compiles the light gradient and the inverse UV in (the adjoint without them is leaner).
template <bool EXTRA>
__device__ __forceinline__ bool layer_adjoint(const Globals &g, const ViewK &V, const MeshK &M, const Layer &L,
                                              float px, float py, const float gC[3], float gD, long long slot,
                                              float *gl)
{
    bool stored = false;
    const long long nvt = g.n_verts_total;
    const FaceRec &R = L.R;
    const Shade &S = L.S;
    float dx[3], dy[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dx[i] = (px - R.xh[i]) - R.xl[i];
        dy[i] = (py - R.yh[i]) - R.yl[i];
    }
    float gX[3] = {0.f, 0.f, 0.f}, gY[3] = {0.f, 0.f, 0.f}, gW[3] = {0.f, 0.f, 0.f};
    const float o = (R.flags & 1) ? 1.f : -1.f;

    // sigmoid -> signed distance -> corners (closest feature)
    const float gdist = gD * S.D * (1.f - S.D) * V.inv_sigma_px;
    if (gdist != 0.f) {
        const int ft = L.fr.feat;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int b = (a + 1) % 3;
            if (ft == a) {
                // F = o cross(V_b - V_a, p - V_a) / |V_b - V_a|
                const float ex = dx[a] - dx[b], ey = dy[a] - dy[b];
                const float il = 1.f / sqrtf(ex * ex + ey * ey);
                const float c = ex * dy[a] - ey * dx[a];
                const float il3 = il * il * il;
                const float gex = o * (dy[a] * il - c * ex * il3);
                const float gey = o * (-dx[a] * il - c * ey * il3);
                const float gdx = o * (-ey * il), gdy = o * (ex * il);
                gX[b] += gdist * gex; gY[b] += gdist * gey;
                gX[a] += gdist * (-gex - gdx); gY[a] += gdist * (-gey - gdy);
            }
            if (ft == 3 + a) {
                // dist = -|p - V_a|
                const float l = sqrtf(dx[a] * dx[a] + dy[a] * dy[a]);
                if (l > 0.f) {
                    gX[a] += gdist * dx[a] / l;
                    gY[a] += gdist * dy[a] / l;
                }
            }
        }
    }

    // shading -> barycentrics and attributes
    float gb[3] = {0.f, 0.f, 0.f};
    const bool anyC = gC[0] != 0.f || gC[1] != 0.f || gC[2] != 0.f;
    if (anyC) {
        if (g.shade_mode == 0) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const long long gi = M.vert_off + S.vi[i];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (g.gcol) atomicAdd(g.gcol + c * nvt + gi, S.b[i] * gC[c]);
                    gb[i] = fmaf(gC[c], __ldg(g.col + c * nvt + gi), gb[i]);
                }
            }
        } else {
            float gA[3];
            float gxn = 0.f, gyn = 0.f;   // the normal map's texel-space UV gradient
            if (g.shade_mode == 1) {
                gA[0] = gC[0]; gA[1] = gC[1]; gA[2] = gC[2];
            } else {
                const float sl = fmaxf(S.ndl, 0.f);
                gA[0] = gC[0] * sl; gA[1] = gC[1] * sl; gA[2] = gC[2] * sl;
                if (S.ndl > 0.f && S.mlen > 0.f) {
                    const float gs = gC[0] * S.A[0] + gC[1] * S.A[1] + gC[2] * S.A[2];
                    if (EXTRA && gl) {
                        // C = A max(0, n.l): dL/dl = (gC . A) n (n' with a normal map)
                        gl[0] = fmaf(gs, S.np[0], gl[0]);
                        gl[1] = fmaf(gs, S.np[1], gl[1]);
                        gl[2] = fmaf(gs, S.np[2], gl[2]);
                    }
                    float gn[3] = {gs * V.light[0], gs * V.light[1], gs * V.light[2]};
                    if (EXTRA && g.shade_mode == 3) {
                        // normal map: dL/dn' = gs l back through n' = m' / |m'|, the map
                        // sample and the tangent frame, to dL/dn of the smooth normal
                        const long long nvt = g.n_verts_total;
                        float u[3], v[3];
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            u[i] = __ldg(g.uv + M.vert_off + S.vi[i]);
                            v[i] = __ldg(g.uv + nvt + M.vert_off + S.vi[i]);
                        }
                        NMap N;
                        nmap_eval(g, M, S, u, v, N);
                        const float d = N.np[0] * gn[0] + N.np[1] * gn[1] + N.np[2] * gn[2];
                        const float iml = 1.f / N.mpl;
                        float gmp[3], gTp[3], gBp[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) gmp[c] = (gn[c] - N.np[c] * d) * iml;
                        const float gt[3] = {2.f * (gmp[0] * N.Tp[0] + gmp[1] * N.Tp[1] + gmp[2] * N.Tp[2]),
                                             2.f * (gmp[0] * N.Bp[0] + gmp[1] * N.Bp[1] + gmp[2] * N.Bp[2]),
                                             2.f * (gmp[0] * S.n[0] + gmp[1] * S.n[1] + gmp[2] * S.n[2])};
                        // map texels (bilinear weights) and the map's texel-space UV gradient
                        const float ox = 1.f - S.fx, oy = 1.f - S.fy;
                        if (g.gntex) {
                            float4 *gt4 = reinterpret_cast<float4 *>(g.gntex);
                            const long long tb = M.tex_off;
                            const float w[4] = {ox * oy, S.fx * oy, ox * S.fy, S.fx * S.fy};
                            const long long ix[4] = {tb + (long long)S.iy[0] * M.tex_w + S.ix[0],
                                                     tb + (long long)S.iy[0] * M.tex_w + S.ix[1],
                                                     tb + (long long)S.iy[1] * M.tex_w + S.ix[0],
                                                     tb + (long long)S.iy[1] * M.tex_w + S.ix[1]};
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                atomicAdd(gt4 + ix[q], make_float4(w[q] * gt[0], w[q] * gt[1], w[q] * gt[2], 0.f));
                        }
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            gxn += gt[c] * (oy * (N.t10[c] - N.t00[c]) + S.fy * (N.t11[c] - N.t01[c]));
                            gyn += gt[c] * (ox * (N.t01[c] - N.t00[c]) + S.fx * (N.t11[c] - N.t10[c]));
                        }
                        // m' = nt0 T' + nt1 B' + nt2 n
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            gTp[c] = N.nt[0] * gmp[c];
                            gBp[c] = N.nt[1] * gmp[c];
                            gn[c] = N.nt[2] * gmp[c];
                        }
                        // B' = h n x T': dL/dn += h T' x gB', dL/dT' += h gB' x n
                        gn[0] += N.h * (N.Tp[1] * gBp[2] - N.Tp[2] * gBp[1]);
                        gn[1] += N.h * (N.Tp[2] * gBp[0] - N.Tp[0] * gBp[2]);
                        gn[2] += N.h * (N.Tp[0] * gBp[1] - N.Tp[1] * gBp[0]);
                        gTp[0] += N.h * (gBp[1] * S.n[2] - gBp[2] * S.n[1]);
                        gTp[1] += N.h * (gBp[2] * S.n[0] - gBp[0] * S.n[2]);
                        gTp[2] += N.h * (gBp[0] * S.n[1] - gBp[1] * S.n[0]);
                        // T' = tau / |tau|, tau = Tf - n (n . Tf)
                        const float dT = N.Tp[0] * gTp[0] + N.Tp[1] * gTp[1] + N.Tp[2] * gTp[2];
                        const float itl = N.tl > 0.f ? 1.f / N.tl : 0.f;
                        float gtau[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) gtau[c] = (gTp[c] - N.Tp[c] * dT) * itl;
                        const float ng = S.n[0] * gtau[0] + S.n[1] * gtau[1] + S.n[2] * gtau[2];
                        // Tf = (e1 dv2 - e2 dv1) / det: object-space corners
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const float gTf = gtau[c] - S.n[c] * ng;
                            gn[c] += -N.nT * gtau[c] - N.Tf[c] * ng;
                            const float ge1 = gTf * N.dv2 * N.idet, ge2 = -gTf * N.dv1 * N.idet;
                            atomicAdd(g.gpos + c * nvt + M.vert_off + S.vi[1], ge1);
                            atomicAdd(g.gpos + c * nvt + M.vert_off + S.vi[2], ge2);
                            atomicAdd(g.gpos + c * nvt + M.vert_off + S.vi[0], -(ge1 + ge2));
                        }
                    }
                    const float nd = S.n[0] * gn[0] + S.n[1] * gn[1] + S.n[2] * gn[2];
                    const float il = 1.f / S.mlen;
                    const float gm[3] = {(gn[0] - S.n[0] * nd) * il, (gn[1] - S.n[1] * nd) * il,
                                         (gn[2] - S.n[2] * nd) * il};
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const long long gi = M.vert_off + S.vi[i];
                        const float4 nv = g.nrm[gi];
                        atomicAdd(g.ngrad + gi, make_float4(S.b[i] * gm[0], S.b[i] * gm[1], S.b[i] * gm[2], 0.f));
                        gb[i] += gm[0] * nv.x + gm[1] * nv.y + gm[2] * nv.z;
                    }
                }
            }
            // bilinear texture adjoint
            const long long tb = M.tex_off;
            const long long i00 = tb + (long long)S.iy[0] * M.tex_w + S.ix[0];
            const long long i10 = tb + (long long)S.iy[0] * M.tex_w + S.ix[1];
            const long long i01 = tb + (long long)S.iy[1] * M.tex_w + S.ix[0];
            const long long i11 = tb + (long long)S.iy[1] * M.tex_w + S.ix[1];
            const float w00 = (1.f - S.fx) * (1.f - S.fy), w10 = S.fx * (1.f - S.fy), w01 = (1.f - S.fx) * S.fy,
                        w11 = S.fx * S.fy;
            if (g.gtex && g.texgrad_mode == 1) {
                // deterministic mode: one record at this (pixel, layer)'s own slot
                g.tg_keys[slot] = (unsigned)i00;
                g.tg_pay0[slot] = make_float4(gA[0], gA[1], gA[2], S.fx);
                g.tg_pay1[slot] = S.fy;
            } else if (EXTRA && g.gtex && g.texgrad_mode == 2) {
                // inverse UV: the sample's dL/dA waits in its slot for the texel lookup
                g.tg_pay0[slot] = make_float4(gA[0], gA[1], gA[2], 0.f);
                stored = true;
            } else if (g.gtex) {
                float4 *gt = reinterpret_cast<float4 *>(g.gtex);
                atomicAdd(gt + i00, make_float4(w00 * gA[0], w00 * gA[1], w00 * gA[2], 0.f));
                atomicAdd(gt + i10, make_float4(w10 * gA[0], w10 * gA[1], w10 * gA[2], 0.f));
                atomicAdd(gt + i01, make_float4(w01 * gA[0], w01 * gA[1], w01 * gA[2], 0.f));
                atomicAdd(gt + i11, make_float4(w11 * gA[0], w11 * gA[1], w11 * gA[2], 0.f));
            }
            const float4 t00 = load_texel(g, i00), t10 = load_texel(g, i10), t01 = load_texel(g, i01),
                         t11 = load_texel(g, i11);
            const float gx = gA[0] * ((1.f - S.fy) * (t10.x - t00.x) + S.fy * (t11.x - t01.x)) +
                             gA[1] * ((1.f - S.fy) * (t10.y - t00.y) + S.fy * (t11.y - t01.y)) +
                             gA[2] * ((1.f - S.fy) * (t10.z - t00.z) + S.fy * (t11.z - t01.z));
            const float gy = gA[0] * ((1.f - S.fx) * (t01.x - t00.x) + S.fx * (t11.x - t10.x)) +
                             gA[1] * ((1.f - S.fx) * (t01.y - t00.y) + S.fx * (t11.y - t10.y)) +
                             gA[2] * ((1.f - S.fx) * (t01.z - t00.z) + S.fx * (t11.z - t10.z));
            // x = sum b_i X_i - 1/2; adding a constant to every gb_i is invisible to the
            // perspective step below (sum b = 1), so corner offsets from corner 0 are used
            // (the normal map, sampled at the same texel coordinates, adds gxn, gyn)
#pragma unroll
            for (int i = 0; i < 3; ++i) gb[i] += (gx + gxn) * S.Xt[i] + (gy + gyn) * S.Yt[i];
        }
        // perspective-correct barycentrics: b_i = q_i / Q, q_i = lam_i / w_i
        const float bdot = S.b[0] * gb[0] + S.b[1] * gb[1] + S.b[2] * gb[2];
        const float iQ = 1.f / S.Q;
        float glam[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float gq = (gb[i] - bdot) * iQ;
            glam[i] = gq * S.iw[i];
            gW[i] += gq * S.lam[i];
        }
        if (L.fr.hard) {
            // lam_i = cross(V_B - V_A, p - V_A) / A2,  A = i+1, B = i+2
            const float iA2 = o * R.invA;
            float gA2 = 0.f;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int A = (i + 1) % 3, B = (i + 2) % 3;
                const float gn = glam[i] * iA2;
                gA2 -= glam[i] * S.lam[i] * iA2;
                const float ex = dx[A] - dx[B], ey = dy[A] - dy[B];
                const float gex = dy[A], gey = -dx[A], gdx = -ey, gdy = ex;
                gX[B] += gn * gex; gY[B] += gn * gey;
                gX[A] += gn * (-gex - gdx); gY[A] += gn * (-gey - gdy);
            }
            const float ux = dx[0] - dx[1], uy = dy[0] - dy[1];   // V1 - V0
            const float wx = dx[0] - dx[2], wy = dy[0] - dy[2];   // V2 - V0
            gX[1] += gA2 * wy; gY[1] -= gA2 * wx;
            gX[2] -= gA2 * uy; gY[2] += gA2 * ux;
            gX[0] += gA2 * (uy - wy); gY[0] += gA2 * (wx - ux);
        } else {
            // lam_P = 1 - s, lam_Q = s, s = (p - P).(Q - P) / |Q - P|^2 on the closest edge
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (L.fr.feat != i) continue;
                const bool sw = i == 2;   // corners in lexicographic order
                const int ia = i, ib = (i + 1) % 3;
                const float dPx = sw ? dx[ib] : dx[ia], dPy = sw ? dy[ib] : dy[ia];
                const float dQx = sw ? dx[ia] : dx[ib], dQy = sw ? dy[ia] : dy[ib];
                const float gP = sw ? glam[ib] : glam[ia], gQ = sw ? glam[ia] : glam[ib];
                const float ex = dPx - dQx, ey = dPy - dQy;            // Q - P
                const float iee = 1.f / (ex * ex + ey * ey), s = L.fr.t;
                const float gs = gQ - gP;
                const float gex = (dPx - 2.f * s * ex) * iee, gey = (dPy - 2.f * s * ey) * iee;
                const float gdx = ex * iee, gdy = ey * iee;
                const float gPx = gs * (-gex - gdx), gPy = gs * (-gey - gdy), gQx = gs * gex, gQy = gs * gey;
                if (sw) {
                    gX[ib] += gPx; gY[ib] += gPy; gX[ia] += gQx; gY[ia] += gQy;
                } else {
                    gX[ia] += gPx; gY[ia] += gPy; gX[ib] += gQx; gY[ib] += gQy;
                }
            }
        }
    }
    float4 *sg = g.sgrad + V.vrec_off;
#pragma unroll
    for (int i = 0; i < 3; ++i)
        if (gX[i] != 0.f || gY[i] != 0.f || gW[i] != 0.f) atomicAdd(sg + S.vi[i], make_float4(gX[i], gY[i], gW[i], 0.f));
    return stored;
}

// inverse UV (Sec. 3.3.2, Alg. 1): the sample of face id at the (jittered) screen
// position (qx, qy) claims the texel holding its UV there; the largest sample number
// wins, as the last writer of a sequential pass over the samples would.  A face that
// is no candidate at the jittered position writes nothing.
__device__ __forceinline__ void inv_uv_write(const Globals &g, const ViewK &V, const MeshK &M, int id, float qx,
                                             float qy, int rec)
{
    FaceRec R;
    Frag fr;
    if (!face_get(g, V, M, id, R) || !eval_face(R, qx, qy, V.r_px, V.half_inv_S, fr)) return;
    float lam[3];
    frag_lambda(R, fr, lam);
    float q[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) q[i] = fmul(lam[i], R.iw[i]);
    const float iQ = __fdiv_rn(1.f, fadd(fadd(q[0], q[1]), q[2]));
    const long long nvt = g.n_verts_total;
    float u = 0.f, v = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float b = fmul(q[i], iQ);
        u = ffma(b, __ldg(g.uv + M.vert_off + R.vi[i]), u);
        v = ffma(b, __ldg(g.uv + nvt + M.vert_off + R.vi[i]), v);
    }
    const float x = fmul(u, (float)M.tex_w), y = fmul(v, (float)M.tex_h);
    if (!(fabsf(x) < 1e9f && fabsf(y) < 1e9f)) return;
    const int tx = wrapi((int)floorf(x), M.tex_w), ty = wrapi((int)floorf(y), M.tex_h);
    atomicMax(g.inv_uv + M.tex_off + (long long)ty * M.tex_w + tx, rec);
}

// ---------------------------------------------------------------------------
// the tile kernel
//
// Raster phase, per staged chunk of faces: every face contributes the (face,
// pixel) pairs of its r-grown bbox inside the tile, and the (face, pixel) pairs
// of its bbox inside the rho-ring around the tile; the pairs are spread evenly
// over all threads.  A pair that survives the approximate test is evaluated
// exactly and merged into the pixel's K-list in shared memory: each slot holds a
// 64-bit (Shift key, face id) and takes atomicMin; the displaced larger value
// moves on to the next slot.  Every value passes slot 0, the values leaving slot
// k are all values but slot k's minimum, so the slots end up holding the K
// smallest pairs in order, whatever the interleaving.
// ---------------------------------------------------------------------------
struct Smem {
    // every mode
    int view, totals[2], next;
    int item_ctr;        // raster: the next (face, row segment) item of the chunk a warp takes
    int qn[2];           // the stored-ids adjoint: its layer ring's items queued / taken
    unsigned long long m0[HS_MAX], m1[HS_MAX];   // per halo row: columns with S^H = 0 / 1
    unsigned char sh[HS_MAX * HS_MAX];
    // the raster (forward and re-rasterizing adjoint) only: the modes from stored layer
    // ids are launched with the shared memory up to F (the stored-ids adjoint adds its
    // layer queues there, adj_smem_bytes), leaving the rest of the SM's unified L1 / shared storage
    // to the L1 cache
    FaceGeo F[CH];       // the staged chunk's faces (geometric part)
    int fid[CH];         // their face ids
    Pre P[CH];
    int rect[CH];        // tile pairs: x0 | y0 << 8 | w << 16 | h << 24 (tile-local, x0/y0 >= 0)
    int hrect[CH];       // ring pairs: (x0 + 16) | (y0 + 16) << 8 | w << 16 | h << 24
    int start[CH];       // exclusive prefix of tile segments (4-pixel row pieces of the rects)
    int hstart[CH];      // exclusive prefix of ring pairs
    unsigned rdiv[CH];   // rounded-up 2^32 / (segments per rect row), 0 for one (rect_xy)
    unsigned hdiv[CH];   // the same for the ring rect's width
    int2 hash[HASH];     // (face id, slot) of the last staged chunk
    int wsum[2][NT / 32];
};

__device__ __forceinline__ unsigned long long pack_frag(float key, int id)
{
    const unsigned int kb = __float_as_uint(key) & 0x7fffffffu;   // keys are >= 0; folds -0 into +0
    return ((unsigned long long)kb << 32) | (unsigned int)id;
}

// The K-list slots of tile pixel (x, y) start at kbuf + kslot(x, y) K.  Each row is rotated
// by 5 y columns: with K = 3 (24-byte slot groups) the 8-byte bank pair of a pixel's group
// is then 3 x + 15 y mod 16, so both access patterns of the raster spread over the banks --
// the pretest's lanes (one 4-pixel row segment each, the segments of a face's rows) at two
// lanes per bank pair, the exact evaluations (8 x 4 pixel patches) at three at most; within
// a row the map is a permutation.
__device__ __forceinline__ int kswz(int y) { return 5 * y; }
template <int TT>
__device__ __forceinline__ int kslot(int x, int y) { return y * TT + ((x + kswz(y)) & (TT - 1)); }

template <int K>
__device__ __forceinline__ void kbuf_insert(unsigned long long *slots, unsigned long long v)
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const unsigned long long old = atomicMin(slots + k, v);
        if (old == EMPTY) return;
        v = old > v ? old : v;
    }
}

__device__ __forceinline__ int find_slot(const Smem &S, int id)
{
    unsigned h = ((unsigned)id * 2654435761u) & (HASH - 1);
    for (int probe = 0; probe < HASH; ++probe) {
        const int2 e = S.hash[h];
        if (e.x == id) return e.y;
        if (e.x < 0) return -1;
        h = (h + 1) & (HASH - 1);
    }
    return -1;
}

// largest f < n with start[f] <= i
__device__ __forceinline__ int search_start(const int *start, int n, int i)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// face of pair i = base + lane (base a multiple of 32): the face holding the block's
// first pair from the block table (a search past the table), then a short walk (a face
// holds tens of pairs, so a warp spans one or two faces)
__device__ __forceinline__ int pair_face(const int *start, const unsigned char *blk, int n, int base, int i)
{
    int f = (base >> 5) < NBLK ? (int)blk[base >> 5] : search_start(start, n, base);
    while (f + 1 < n && start[f + 1] <= i) ++f;
    return f;
}

// block table of a pair prefix: blk[b] = the face holding pair 32 b
__device__ __forceinline__ void fill_blocks(unsigned char *blk, int f, int start, int cnt)
{
    if (cnt <= 0) return;
    const int be = min((start + cnt - 1) >> 5, NBLK - 1);
    for (int b = (start + 31) >> 5; b <= be; ++b) blk[b] = (unsigned char)f;
}

// the multiplier of rect_xy for rects of width w >= 1: ceil(2^32 / w), 0 for w = 1
__device__ __forceinline__ unsigned rect_div(int w)
{
    return w > 1 ? 0xffffffffu / (unsigned)w + 1u : 0u;
}

// (x, y) of pair q in a rect of width w, m = rect_div(w): q / w as the high word of q m,
// exact for q < 2^32 / w (here q and w are below 2^12)
__device__ __forceinline__ void rect_xy(int q, int w, unsigned m, int &x, int &y)
{
    const int qy = m ? (int)__umulhi((unsigned)q, m) : q;
    x = q - qy * w;
    y = qy;
}

// hard or soft, from the key a fragment was kept with: hard keys are 0.5 z <= 1/2 and
// soft keys 0.5 + 0.5 |d| / S >= 1/2, so only a key of exactly 1/2 needs the face again
__device__ __forceinline__ bool kept_hard(const Globals &g, const ViewK &V, const MeshK &M,
                                          unsigned long long v, float px, float py)
{
    const float key = __uint_as_float((unsigned int)(v >> 32));
    if (key != 0.5f) return key < 0.5f;
    FaceRec R;
    Frag fr;
    return face_get(g, V, M, (int)(unsigned int)(v & 0xffffffffu), R) &&
           eval_face<false>(R, px, py, V.r_px, V.half_inv_S, fr) && fr.hard;
}

// edge mask (Sec. 3.4.3) of tile pixel (lx, ly): the window of radius rho sees both
// S^H = 0 and 1 (S.m0 / S.m1 hold the columns of each halo row with either value)
__device__ __forceinline__ bool edge_mask(const Globals &g, const Smem &S, int lx, int ly, int rho)
{
    if (g.edge_mode != 0) return g.edge_mode == 1;
    unsigned long long a0 = 0ull, a1 = 0ull;
    for (int wy = 0; wy <= 2 * rho; ++wy) { a0 |= S.m0[ly + wy]; a1 |= S.m1[ly + wy]; }
    const unsigned long long wm = (2ull << (2 * rho)) - 1ull;   // columns lx .. lx + 2 rho
    return ((a0 >> lx) & wm) && ((a1 >> lx) & wm);
}

// the adjoint of the edge-mask blend (Sec. 3.4.3) at one pixel: the colour
// sum_k D_k C_k / sum_k D_k and the silhouette 1 - prod_k (1 - D_k), from the nl layers'
// D_k and C_k and the incoming dL/d(RGBA) gi4; adds into gCk / gDk (zero on entry)
template <int K>
__device__ __forceinline__ void blend_weights(const float (&Dk)[K], const float (&Ck)[K][3], int nl, float4 gi4,
                                              float (&gCk)[K][3], float (&gDk)[K])
{
    const float gc[3] = {gi4.x, gi4.y, gi4.z};
    float Ds = 0.f, Ie[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < K; ++k) {
        Ds += Dk[k];
        Ie[0] = fmaf(Dk[k], Ck[k][0], Ie[0]);
        Ie[1] = fmaf(Dk[k], Ck[k][1], Ie[1]);
        Ie[2] = fmaf(Dk[k], Ck[k][2], Ie[2]);
    }
    if (Ds > 0.f) {
        const float iD = 1.f / Ds;
        Ie[0] *= iD; Ie[1] *= iD; Ie[2] *= iD;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            gCk[k][0] = Dk[k] * iD * gc[0];
            gCk[k][1] = Dk[k] * iD * gc[1];
            gCk[k][2] = Dk[k] * iD * gc[2];
            gDk[k] = (gc[0] * (Ck[k][0] - Ie[0]) + gc[1] * (Ck[k][1] - Ie[1]) + gc[2] * (Ck[k][2] - Ie[2])) * iD;
        }
    }
    // silhouette 1 - prod_k (1 - D_k)
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float others = 1.f;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (j != k && j < nl) others *= 1.f - Dk[j];
        if (k < nl) gDk[k] += gi4.w * others;
    }
}

// dL/dC_k and dL/dD_k of the K layers of one pixel (the adjoint of the blend, Sec.
// 3.4.3): E and SH as the forward decided them; returns false when nothing flows back
// (no layer, or a zero incoming gradient unless every sample is wanted)
template <int K, bool EXTRA>
__device__ __forceinline__ bool pixel_weights(const Globals &g, const ViewK &V, const MeshK &M, long long pix,
                                              float px, float py, const int (&ids)[K], int nl, bool E, bool SH,
                                              bool inv, float (&gCk)[K][3], float (&gDk)[K])
{
#pragma unroll
    for (int k = 0; k < K; ++k) { gDk[k] = 0.f; gCk[k][0] = gCk[k][1] = gCk[k][2] = 0.f; }
    if (nl == 0) return false;
    const float4 gi4 = __ldg(reinterpret_cast<const float4 *>(g.gin) + pix);
    const float gc[3] = {gi4.x, gi4.y, gi4.z};
    if (!inv && gc[0] == 0.f && gc[1] == 0.f && gc[2] == 0.f && gi4.w == 0.f) return false;
    if (E) {
        // pass 1: D_k and C_k of every layer
        float Dk[K], Ck[K][3];
#pragma unroll
        for (int k = 0; k < K; ++k) { Dk[k] = 0.f; Ck[k][0] = Ck[k][1] = Ck[k][2] = 0.f; }
        // rolled loop: one inlined copy of the layer code keeps the kernel small
#pragma unroll 1
        for (int k = 0; k < nl; ++k) {
            Layer L;
            if (layer_build<EXTRA>(g, V, M, ids[k], px, py, L)) {
                Dk[k] = L.S.D;
                Ck[k][0] = L.S.C[0]; Ck[k][1] = L.S.C[1]; Ck[k][2] = L.S.C[2];
            }
        }
        blend_weights<K>(Dk, Ck, nl, gi4, gCk, gDk);
    } else if (SH) {
        gCk[0][0] = gc[0]; gCk[0][1] = gc[1]; gCk[0][2] = gc[2];
    }
    return true;
}

// The adjoint of one pixel whose K layer ids are known, by pixel: the adjoints with
// the extras (light gradient, inverse UV, normal map); S.sh holds the tile's S^H with its
// ring.
template <int K, int TT, bool EXTRA>
__device__ __forceinline__ unsigned adjoint_pixel(const Globals &g, const Smem &S, const ViewK &V, const MeshK &M,
                                                  int X0, int Y0, int lx, int ly, int rho, const int (&ids)[K],
                                                  float *gl)
{
    const int X = X0 + lx, Y = Y0 + ly;   // view-local pixel coordinates
    const float px = (float)X + 0.5f, py = (float)Y + 0.5f;
    const int hs = TT + 2 * rho;
    const long long pix = V.pix_off + (long long)Y * V.W + X;
    int nl = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) nl += (ids[k] != 0x7fffffff) ? 1 : 0;
    const bool SH = S.sh[(ly + rho) * hs + (lx + rho)] == 1;
    const bool E = edge_mask(g, S, lx, ly, rho);

    unsigned layers = 0;
    const bool inv = EXTRA && g.texgrad_mode == 2;
    float gCk[K][3], gDk[K];
    if (!pixel_weights<K, EXTRA>(g, V, M, pix, px, py, ids, nl, E, SH, inv, gCk, gDk)) return 0;
    // the adjoint of each layer with a gradient
    unsigned stored = 0u;
#pragma unroll 1
    for (int k = 0; k < nl; ++k) {
        const float gCl[3] = {gCk[k][0], gCk[k][1], gCk[k][2]};
        const float gDl = gDk[k];
        const bool any = gDl != 0.f || gCl[0] != 0.f || gCl[1] != 0.f || gCl[2] != 0.f;
        Layer L;
        const long long slot = (V.slot_base + (long long)Y * V.W + X) * K + k;
        if (any && layer_build<EXTRA>(g, V, M, ids[k], px, py, L)) {
            ++layers;
            if (layer_adjoint<EXTRA>(g, V, M, L, px, py, gCl, gDl, slot, gl)) stored |= 1u << k;
        }
    }
    if (inv) {
        // every shaded sample (the layers the forward blends) claims its texel; a sample
        // without a texture gradient offers dL/dA = 0
#pragma unroll 1
        for (int k = 0; k < nl; ++k) {
            if (!(E || k == 0)) continue;
            const long long slot = (V.slot_base + (long long)Y * V.W + X) * K + k;
            if (!((stored >> k) & 1u)) g.tg_pay0[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
            inv_uv_write(g, V, M, ids[k], fadd(px, g.uv_jx), fadd(py, g.uv_jy), (int)slot);
        }
    }
    return layers;
}

// S^H, edge mask, shading and blend of one round of pixels (one per thread; lanes
// outside the image take part with no layer).  A warp shades the layers its pixels
// blend -- all of a pixel's layers inside the edge mask, else the front one where
// S^H = 1 -- as one list, 32 at a time, so pixels with three layers, one or none
// share full warps; each pixel then takes its layers' colours and coverages back by
// shuffles and blends them in layer order.
template <int K, int TT, bool EXTRA>
__device__ __forceinline__ unsigned finish_forward(const Globals &g, const Smem &S, const ViewK &V, const MeshK &M,
                                                   int X0, int Y0, int p, int rho, bool in, const int (&ids)[K],
                                                   unsigned hardbits, bool single_chunk, float &l2acc)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int lx = p % TT, ly = p / TT;
    const int hs = TT + 2 * rho;
    int nl = 0;
    bool SH = false, E = false;
    long long pix = 0;
    if (in) {
        pix = V.pix_off + (long long)(Y0 + ly) * V.W + (X0 + lx);
#pragma unroll
        for (int k = 0; k < K; ++k) nl += (ids[k] != 0x7fffffff) ? 1 : 0;
        SH = S.sh[(ly + rho) * hs + (lx + rho)] == 1;
        E = edge_mask(g, S, lx, ly, rho);
        if (g.ids) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                // stored layer: the face index, with bit 31 set for a soft fragment
                const unsigned soft = ((hardbits >> k) & 1u) ? 0u : 0x80000000u;
                g.ids[(long long)k * g.n_pix + pix] = (k < nl) ? (int)((unsigned)ids[k] | soft) : -1;
            }
        }
    }
    // the layers blended (outside the edge mask only the front one is seen), and their
    // place in the warp's list
    const int cnt = E ? nl : (SH && nl > 0 ? 1 : 0);
    int off = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, off, o);
        if (lane >= o) off += y;
    }
    const int tot = __shfl_sync(FULL, off, 31);
    off -= cnt;

    float Cs[3] = {0.f, 0.f, 0.f}, C1[3] = {0.f, 0.f, 0.f};
    float Ds = 0.f, prod = 1.f;
    unsigned layers = 0;
    for (int w = 0; w * 32 < tot; ++w) {
        const int i = w * 32 + lane;
        // the pixel (lane) whose layers include list entry i: the last one starting at or before it
        int o = 0;
#pragma unroll
        for (int st = 16; st > 0; st >>= 1)
            if (__shfl_sync(FULL, off, o + st) <= i) o += st;
        const int k = i - __shfl_sync(FULL, off, o);
        int id = 0x7fffffff;
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            const int v = __shfl_sync(FULL, ids[kk], o);
            if (kk == k) id = v;
        }
        float C[3] = {0.f, 0.f, 0.f}, D = 0.f;
        int live = 0;
        if (i < tot) {
            // re-evaluate the layer at its pixel (from shared memory when the whole tile
            // list was staged at once): distance and barycentrics, then the shading
            const int po = p - lane + o;
            const float px = (float)(X0 + po % TT) + 0.5f, py = (float)(Y0 + po / TT) + 0.5f;
            const int slot = single_chunk ? find_slot(S, id) : -1;
            FaceRec R;
            bool ok;
            if (slot >= 0) {
                face_complete(g, V, id, S.F[slot], R);
                ok = (R.flags & FLAG_LIVE) != 0;
            } else {
                ok = face_get(g, V, M, id, R);
            }
            Frag fr;
            if (ok && eval_face(R, px, py, V.r_px, V.half_inv_S, fr)) {
                Shade Sh;
                frag_lambda(R, fr, Sh.lam);
#pragma unroll
                for (int q = 0; q < 3; ++q) { Sh.vi[q] = R.vi[q]; Sh.iw[q] = R.iw[q]; }
                Sh.odd = (R.flags & FLAG_ODD) != 0;
                shade<EXTRA>(g, V, M, fr.dist, Sh);
                C[0] = Sh.C[0]; C[1] = Sh.C[1]; C[2] = Sh.C[2];
                D = Sh.D;
                live = 1;
                ++layers;
            }
        }
        // this pixel's layers among the entries of this pass, in layer order
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            const int src = off + kk - w * 32;
            const int sl = src & 31;
            const float c0 = __shfl_sync(FULL, C[0], sl), c1 = __shfl_sync(FULL, C[1], sl),
                        c2 = __shfl_sync(FULL, C[2], sl), d = __shfl_sync(FULL, D, sl);
            const int lv = __shfl_sync(FULL, live, sl);
            if (kk < cnt && src >= 0 && src < 32 && lv) {
                Cs[0] = ffma(d, c0, Cs[0]);
                Cs[1] = ffma(d, c1, Cs[1]);
                Cs[2] = ffma(d, c2, Cs[2]);
                Ds = fadd(Ds, d);
                prod = fmul(prod, fsub(1.f, d));
                if (kk == 0) { C1[0] = c0; C1[1] = c1; C1[2] = c2; }
            }
        }
    }
    if (in) {
        float4 o;
        if (E) {
            const float iD = Ds > 0.f ? __fdiv_rn(1.f, Ds) : 0.f;
            o = make_float4(fmul(Cs[0], iD), fmul(Cs[1], iD), fmul(Cs[2], iD), fsub(1.f, prod));
        } else {
            o = SH ? make_float4(C1[0], C1[1], C1[2], 1.f) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        reinterpret_cast<float4 *>(g.out)[pix] = o;
        if (g.l2_target) {
            // the L2 loss's gradient 2 (out - target) and its sum of squares
            const float4 t = __ldg(reinterpret_cast<const float4 *>(g.l2_target) + pix);
            const float dx = o.x - t.x, dy = o.y - t.y, dz = o.z - t.z, dw = o.w - t.w;
            reinterpret_cast<float4 *>(g.l2_grad)[pix] = make_float4(2.f * dx, 2.f * dy, 2.f * dz, 2.f * dw);
            l2acc += dx * dx + dy * dy + dz * dz + dw * dw;
        }
    }
    return layers;
}

// The re-rasterizing adjoint of one round of pixels (one per thread; lanes outside the
// image take part with no layer), warp-collective like the forward's shading: a warp
// rebuilds the layers its edge-masked pixels blend (for D_k, C_k) as one list, each
// pixel forms dL/dC_k, dL/dD_k (blend_weights), and the warp then rebuilds and
// back-propagates the layers with a gradient as a second list.
template <int K, int TT>
__device__ __forceinline__ unsigned adjoint_warp(const Globals &g, const Smem &S, const ViewK &V, const MeshK &M,
                                                 int X0, int Y0, int p, int rho, bool in, const int (&ids)[K])
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int lx = p % TT, ly = p / TT;
    const int hs = TT + 2 * rho;
    int nl = 0;
    bool E = false, SH = false, active = false;
    float4 gi4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (in) {
#pragma unroll
        for (int k = 0; k < K; ++k) nl += (ids[k] != 0x7fffffff) ? 1 : 0;
        if (nl > 0) {
            gi4 = __ldg(reinterpret_cast<const float4 *>(g.gin) + V.pix_off + (long long)(Y0 + ly) * V.W + (X0 + lx));
            active = gi4.x != 0.f || gi4.y != 0.f || gi4.z != 0.f || gi4.w != 0.f;
            if (active) {
                SH = S.sh[(ly + rho) * hs + (lx + rho)] == 1;
                E = edge_mask(g, S, lx, ly, rho);
            }
        }
    }
    // list entry i of a warp list with per-lane counts cnt (exclusive offsets off):
    // the owning lane
    auto owner = [&](int off, int i) {
        int o = 0;
#pragma unroll
        for (int st = 16; st > 0; st >>= 1)
            if (__shfl_sync(FULL, off, o + st) <= i) o += st;
        return o;
    };
    auto scan = [&](int cnt, int &tot) {
        int off = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, off, o);
            if (lane >= o) off += y;
        }
        tot = __shfl_sync(FULL, off, 31);
        return off - cnt;
    };

    // pass 1: D_k and C_k of every layer of an edge-masked pixel
    float Dk[K], Ck[K][3];
#pragma unroll
    for (int k = 0; k < K; ++k) { Dk[k] = 0.f; Ck[k][0] = Ck[k][1] = Ck[k][2] = 0.f; }
    {
        const int cnt = (active && E) ? nl : 0;
        int tot;
        const int off = scan(cnt, tot);
        for (int w = 0; w * 32 < tot; ++w) {
            const int i = w * 32 + lane;
            const int o = owner(off, i);
            const int k = i - __shfl_sync(FULL, off, o);
            int id = 0x7fffffff;
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                const int v = __shfl_sync(FULL, ids[kk], o);
                if (kk == k) id = v;
            }
            float C[3] = {0.f, 0.f, 0.f}, D = 0.f;
            if (i < tot) {
                const int po = p - lane + o;
                Layer L;
                if (layer_build<false>(g, V, M, id, (float)(X0 + po % TT) + 0.5f, (float)(Y0 + po / TT) + 0.5f, L)) {
                    C[0] = L.S.C[0]; C[1] = L.S.C[1]; C[2] = L.S.C[2];
                    D = L.S.D;
                }
            }
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                const int src = off + kk - w * 32;
                const int sl = src & 31;
                const float c0 = __shfl_sync(FULL, C[0], sl), c1 = __shfl_sync(FULL, C[1], sl),
                            c2 = __shfl_sync(FULL, C[2], sl), d = __shfl_sync(FULL, D, sl);
                if (kk < cnt && src >= 0 && src < 32) {
                    Dk[kk] = d;
                    Ck[kk][0] = c0; Ck[kk][1] = c1; Ck[kk][2] = c2;
                }
            }
        }
    }
    // the blend's adjoint per pixel
    float gCk[K][3], gDk[K];
#pragma unroll
    for (int k = 0; k < K; ++k) { gDk[k] = 0.f; gCk[k][0] = gCk[k][1] = gCk[k][2] = 0.f; }
    if (active) {
        if (E) blend_weights<K>(Dk, Ck, nl, gi4, gCk, gDk);
        else if (SH) { gCk[0][0] = gi4.x; gCk[0][1] = gi4.y; gCk[0][2] = gi4.z; }
    }
    unsigned want = 0u;
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (k < nl && (gDk[k] != 0.f || gCk[k][0] != 0.f || gCk[k][1] != 0.f || gCk[k][2] != 0.f)) want |= 1u << k;

    // pass 2: the adjoints of the layers with a gradient
    unsigned layers = 0;
    {
        int tot;
        const int off = scan(__popc(want), tot);
        for (int w = 0; w * 32 < tot; ++w) {
            const int i = w * 32 + lane;
            const int o = owner(off, i);
            const int j = i - __shfl_sync(FULL, off, o);   // the owner's j-th layer with a gradient
            const unsigned wm = __shfl_sync(FULL, want, o);
            int k = 0;
#pragma unroll
            for (int kk = 0, seen = 0; kk < K; ++kk)
                if ((wm >> kk) & 1u) {
                    if (seen == j) k = kk;
                    ++seen;
                }
            int id = 0x7fffffff;
            float gC[3] = {0.f, 0.f, 0.f}, gD = 0.f;
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                const int v = __shfl_sync(FULL, ids[kk], o);
                const float a0 = __shfl_sync(FULL, gCk[kk][0], o), a1 = __shfl_sync(FULL, gCk[kk][1], o),
                            a2 = __shfl_sync(FULL, gCk[kk][2], o), b = __shfl_sync(FULL, gDk[kk], o);
                if (kk == k) { id = v; gC[0] = a0; gC[1] = a1; gC[2] = a2; gD = b; }
            }
            if (i < tot) {
                const int po = p - lane + o;
                const int Xo = X0 + po % TT, Yo = Y0 + po / TT;
                const float px = (float)Xo + 0.5f, py = (float)Yo + 0.5f;
                const long long slot = (V.slot_base + (long long)Yo * V.W + Xo) * K + k;
                Layer L;
                if (layer_build<false>(g, V, M, id, px, py, L)) {
                    ++layers;
                    layer_adjoint<false>(g, V, M, L, px, py, gC, gD, slot, nullptr);
                }
            }
        }
    }
    return layers;
}

// The adjoint from stored layer ids, by layer rather than by pixel.  A layer rebuilt
// from its face id (record, distance, barycentrics, shading) is the costliest step, and
// by pixel it would run with the lanes of background, single-layer and gradient-free
// pixels idle.  Each round of NT pixels (one per thread) instead
//   1. queues, for an edge-masked pixel, each of its layers for the blend (D_k, C_k);
//      a pixel outside the mask queues its front layer's adjoint directly
//      (dL/dC = dL/dRGB when S^H = 1);
//   2. rebuilds the queued layers with all threads into a (pixel, layer) table;
//   3. forms each edge-masked pixel's dL/dC_k, dL/dD_k from the table (blend_weights)
//      and queues its layers with a gradient;
//   4. rebuilds and back-propagates the queued adjoints, whole multiples of NT at a
//      time (the rest waits for the next round; the last round takes all).
// Steps 2 and 3 are skipped in a round without edge-masked pixels.  The adjoint ring
// holds fewer than NT leftovers plus one round's K NT items.
template <int K>
__host__ __device__ constexpr int adj_ring() { return NT * (K + 1); }
__host__ __device__ constexpr size_t adj_ring_off() { return (offsetof(Smem, F) + 15) / 16 * 16; }
template <int K>
__host__ __device__ constexpr size_t adj_smem_bytes()
{
    // adjoint ring (dL/dC, dL/dD | face id, pixel and layer), blend table, blend queue
    return adj_ring_off() + (sizeof(float4) + sizeof(int2)) * adj_ring<K>() + sizeof(float4) * NT * K +
           sizeof(unsigned short) * NT * K;
}

template <int K, int TT>
__device__ __forceinline__ unsigned adjoint_queued(const Globals &g, Smem &S, const ViewK &V, const MeshK &M,
                                                   int X0, int Y0, int rho, int wlim, int hlim)
{
    constexpr int PPT = TT * TT / NT;
    constexpr int QC = adj_ring<K>();
    float4 *qg = reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(&S) + adj_ring_off());
    int2 *qi = reinterpret_cast<int2 *>(qg + QC);        // (face id, pixel | layer << 10)
    float4 *dc = reinterpret_cast<float4 *>(qi + QC);    // [thread][layer]: (C_k, D_k)
    unsigned short *bq = reinterpret_cast<unsigned short *>(dc + NT * K);   // thread | layer << 8
    const int tid = threadIdx.x, lane = tid & 31;
    const int hs = TT + 2 * rho;
    unsigned layers = 0;
    // S.qn[0]: adjoint items queued, S.qn[1]: taken (both zero at the tile's start);
    // S.totals[0]: blend items of the round
    if (tid == 0) S.totals[0] = 0;
    __syncthreads();

    // warp-aggregated reservation of c slots on counter *ctr: returns this lane's first slot
    auto reserve = [&](int *ctr, int c) {
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int base = 0;
        if (lane == 31 && incl > 0) base = atomicAdd(ctr, incl);
        return __shfl_sync(0xffffffffu, base, 31) + incl - c;
    };
    auto push_adj = [&](int base, int id, int p, int k, float c0, float c1, float c2, float d) {
        const int q = base % QC;
        qg[q] = make_float4(c0, c1, c2, d);
        qi[q] = make_int2(id, p | (k << 10));
    };

    for (int j = 0; j < PPT; ++j) {
        const int p = tid + j * NT;
        const int lx = p % TT, ly = p / TT;
        const int X = X0 + lx, Y = Y0 + ly;
        const long long pix = V.pix_off + (long long)Y * V.W + X;
        const bool in = lx < wlim && ly < hlim;
        // step 1
        int nl = 0, id0 = 0;
        bool E = false, front = false;
        float4 gi4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (in) {
            // the layer ids and dL/dI together: one load latency instead of two in a row
            int idk[K];
#pragma unroll
            for (int k = 0; k < K; ++k) idk[k] = __ldg(g.ids_in + (long long)k * g.n_pix + pix);
            gi4 = __ldg(reinterpret_cast<const float4 *>(g.gin) + pix);
#pragma unroll
            for (int k = 0; k < K; ++k) nl += idk[k] != -1 ? 1 : 0;
            if (nl > 0 && (gi4.x != 0.f || gi4.y != 0.f || gi4.z != 0.f || gi4.w != 0.f)) {
                E = edge_mask(g, S, lx, ly, rho);
                // outside the mask the pixel is its front layer's colour where S^H = 1
                front = !E && S.sh[(ly + rho) * hs + (lx + rho)] == 1 &&
                        (gi4.x != 0.f || gi4.y != 0.f || gi4.z != 0.f);
                id0 = idk[0] & 0x7fffffff;
            }
        }
        {
            const int b = reserve(&S.totals[0], E ? nl : 0);
            for (int k = 0; k < (E ? nl : 0); ++k) bq[b + k] = (unsigned short)(tid | (k << 8));
            const int a = reserve(&S.qn[0], front ? 1 : 0);
            if (front) push_adj(a, id0, p, 0, gi4.x, gi4.y, gi4.z, 0.f);
        }
        __syncthreads();
        const int nb = S.totals[0];
        if (nb > 0) {
            // step 2: the blend table
            for (int i = tid; i < nb; i += NT) {
                const int it = bq[i];
                const int o = it & 255, k = it >> 8;
                const int po = o + j * NT;
                const int Xo = X0 + po % TT, Yo = Y0 + po / TT;
                const long long pixo = V.pix_off + (long long)Yo * V.W + Xo;
                const int id = __ldg(g.ids_in + (long long)k * g.n_pix + pixo) & 0x7fffffff;
                Layer L;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (layer_build<false>(g, V, M, id, (float)Xo + 0.5f, (float)Yo + 0.5f, L))
                    v = make_float4(L.S.C[0], L.S.C[1], L.S.C[2], L.S.D);
                dc[o * K + k] = v;
            }
            __syncthreads();
            // every thread has read the blend count; the next round's reservations
            // come after this round's last barrier
            if (tid == 0) S.totals[0] = 0;
            // step 3
            float gCk[K][3], gDk[K];
            unsigned want = 0u;
            int ids[K];
            if (E) {
                float Dk[K], Ck[K][3];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    gDk[k] = 0.f; gCk[k][0] = gCk[k][1] = gCk[k][2] = 0.f;
                    const float4 v = k < nl ? dc[tid * K + k] : make_float4(0.f, 0.f, 0.f, 0.f);
                    Ck[k][0] = v.x; Ck[k][1] = v.y; Ck[k][2] = v.z; Dk[k] = v.w;
                }
                blend_weights<K>(Dk, Ck, nl, gi4, gCk, gDk);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    ids[k] = k < nl ? __ldg(g.ids_in + (long long)k * g.n_pix + pix) & 0x7fffffff : 0;
                    if (k < nl && (gDk[k] != 0.f || gCk[k][0] != 0.f || gCk[k][1] != 0.f || gCk[k][2] != 0.f))
                        want |= 1u << k;
                }
            }
            int a = reserve(&S.qn[0], __popc(want));
#pragma unroll
            for (int k = 0; k < K; ++k)
                if ((want >> k) & 1u) push_adj(a++, ids[k], p, k, gCk[k][0], gCk[k][1], gCk[k][2], gDk[k]);
            __syncthreads();
        }
        // step 4
        const int head = S.qn[1], n = S.qn[0] - head;
        const int m = (j == PPT - 1) ? n : n / NT * NT;
        for (int i = tid; i < m; i += NT) {
            const int q = (head + i) % QC;
            const float4 gg = qg[q];
            const int2 it = qi[q];
            const int pp = it.y & 1023, k = it.y >> 10;
            const int Xq = X0 + pp % TT, Yq = Y0 + pp / TT;
            const float px = (float)Xq + 0.5f, py = (float)Yq + 0.5f;
            const float gCl[3] = {gg.x, gg.y, gg.z};
            const long long slot = (V.slot_base + (long long)Yq * V.W + Xq) * K + k;
            Layer L;
            if (layer_build<false>(g, V, M, it.x, px, py, L)) {
                ++layers;
                layer_adjoint<false>(g, V, M, L, px, py, gCl, gg.w, slot, nullptr);
            }
        }
        __syncthreads();   // the items taken are free and every thread has read the counters
        if (tid == 0) S.qn[1] = head + m;
    }
    return layers;
}

// The pretest and exact evaluation of one staged chunk's (face, 4-pixel row segment) items
// (total of them).  Warps take 32 items at a time from the chunk's shared counter, so no
// CTA barrier is needed until the chunk is done.  Each lane tests its item's (up to) four
// pixel centres -- inside the face's grown bbox by construction of the rect -- with the
// approximate edge equations stepped along x and a lower bound of the Shift key against
// the pixel's current K-th key; the pairs that pass go to the warp's own queue (a ring of
// WQ entries in shared memory), and whenever it holds 32 of them the warp evaluates them
// exactly with all lanes and merges the candidates into the pixels' K-lists (other warps
// merge into the same lists concurrently: the atomicMin cascade is order independent).
// A queue entry is x | y << 5 | face << 10 with the top 14 bits of the key lower bound
// above (truncated: still a lower bound).
template <int K, int TT>
__device__ __forceinline__ void raster_items(Smem &S, unsigned long long *kbuf, unsigned *wq,
                                             const unsigned char *blk, const ViewK &V, int X0, int Y0, int nch,
                                             int total, bool count, unsigned &n_pairs, unsigned &n_exact,
                                             unsigned &n_cand)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int head = 0, qn = 0;   // the warp's queue: qn entries from wq[head] on (warp-uniform)
    // exact evaluation of the n <= 32 entries at the queue's head, one per lane
    auto evaluate = [&](int n) {
        if (lane < n) {
            int q = head + lane;
            if (q >= WQ) q -= WQ;
            const unsigned ent = wq[q];
            const int x = ent & 31, y = (ent >> 5) & 31, f = (ent >> 10) & 0xff;
            unsigned long long *slots = kbuf + kslot<TT>(x, y) * K;
            const unsigned long long last = *reinterpret_cast<volatile unsigned long long *>(slots + K - 1);
            if (!(__uint_as_float(ent & 0xfffc0000u) > __uint_as_float((unsigned int)(last >> 32)))) {
                Frag fr;
                ++n_exact;
                if (eval_face<false>(S.F[f], (float)(X0 + x) + 0.5f, (float)(Y0 + y) + 0.5f, V.r_px, V.half_inv_S,
                                     fr)) {
                    ++n_cand;
                    kbuf_insert<K>(slots, pack_frag(fr.key, S.fid[f]));
                }
            }
        }
        head += n;
        if (head >= WQ) head -= WQ;
        qn -= n;
        __syncwarp();   // the entries read are free for the next pushes
    };
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&S.item_ctr, 32);
        base = __shfl_sync(FULL, base, 0);
        if (base >= total) break;
        const int i = base + lane;
        unsigned pm = 0u;   // pass bits of the segment's pixels
        float kl[4] = {0.f, 0.f, 0.f, 0.f};
        int f = 0, x = 0, y = 0;
        if (i < total) {
            f = pair_face(S.start, blk, nch, base, i);
            const int rc = S.rect[f];
            const int w = (rc >> 16) & 0xff;
            int qx, qy;
            rect_xy(i - S.start[f], (w + 3) >> 2, S.rdiv[f], qx, qy);
            x = (rc & 0xff) + 4 * qx;
            y = ((rc >> 8) & 0xff) + qy;
            const int np = min(4, (rc & 0xff) + w - x);
            if (count) n_pairs += np;
            const Pre &P = S.P[f];
            const float fx = (float)x + 0.5f, fy = (float)y + 0.5f;
            float e0 = fmaf(P.nx[0], fx, fmaf(P.ny[0], fy, P.c[0]));
            float e1 = fmaf(P.nx[1], fx, fmaf(P.ny[1], fy, P.c[1]));
            float e2 = fmaf(P.nx[2], fx, fmaf(P.ny[2], fy, P.c[2]));
            const float klb_in = 0.5f * P.zmin * (1.f - 1e-6f);
            // the K-th slots change under other warps' merges; any value read is an upper
            // bound of the final one, so a pair culled against it stays culled
            const volatile unsigned long long *last = kbuf + K - 1;
            const int row = y * TT, sw = kswz(y);
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                // F(p) ~ the smallest edge value: outside, the distance is at least -F;
                // inside, the depth is at least the smallest corner depth
                const float fmin = fminf(e0, fminf(e1, e2));
                if (d < np && fmin >= -V.r_px - APPROX_EPS) {
                    const float klb = fmin > APPROX_EPS    ? klb_in
                                      : fmin < -APPROX_EPS ? fmaf(-fmin - APPROX_EPS, V.half_inv_S, 0.5f)
                                                           : 0.f;
                    if (!(klb > __uint_as_float((unsigned int)(last[(row + ((x + d + sw) & (TT - 1))) * K] >> 32)))) {
                        pm |= 1u << d;
                        kl[d] = klb;
                    }
                }
                e0 += P.nx[0];
                e1 += P.nx[1];
                e2 += P.nx[2];
            }
        }
        // warp-wide prefix of the pass counts: the lanes' places behind the queue's tail
        const int c = __popc(pm);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const int wtot = __shfl_sync(FULL, incl, 31);
        if (wtot) {
            int q = head + qn + incl - c;
            if (q >= WQ) q -= WQ;
            const unsigned ebase = ((unsigned)f << 10) | ((unsigned)y << 5) | (unsigned)x;
#pragma unroll
            for (int d = 0; d < 4; ++d)
                if ((pm >> d) & 1u) {
                    wq[q] = (__float_as_uint(kl[d]) & 0xfffc0000u) | (ebase + d);
                    if (++q == WQ) q = 0;
                }
            qn += wtot;
            __syncwarp();   // the pushed entries are visible to every lane
            while (qn >= 32) evaluate(32);
        }
    }
    if (qn > 0) evaluate(qn);
}

// everything one CTA does for global tile t.  MODE: 0 forward, 1 adjoint that
// re-rasterizes, 2 adjoint from stored layer ids, 3 forward from stored layer ids
// (re-shading a static geometry: no binning, raster or peel); 4, 5, 6, 7 = 2, 1, 0, 3
// with the normal map, the light gradient and the inverse UV compiled in
template <int K, int MODE, int TT>
__device__ __forceinline__ void tile_body(const Globals &g, Smem &S, unsigned long long *kbuf, const int t)
{
    constexpr int PPT = TT * TT / NT;   // pixels per thread in the per-pixel phases
    // after the K-lists: the candidate queue and the two pair-block tables
    unsigned *qbuf = reinterpret_cast<unsigned *>(kbuf + TT * TT * K);
    unsigned char *blk = reinterpret_cast<unsigned char *>(qbuf + QN);
    unsigned char *hblk = blk + NBLK;
    // the adjoints with extras: each thread's share of dL/dlight, after the part of the
    // shared memory the kernel uses (the header alone when it reads stored layers)
    float(*gl_slots)[3] = reinterpret_cast<float(*)[3]>(
        MODE == 4 ? reinterpret_cast<unsigned char *>(&S) + offsetof(Smem, F) : hblk + NBLK);
    if (threadIdx.x == 0) {
        S.view = g.tile_view[t];
        S.qn[0] = 0;
        S.qn[1] = 0;
    }
    __syncthreads();
    const ViewK &V = g.views[S.view];
    const MeshK &M = g.meshes[V.mesh];
    const int lt = t - V.tile_base;
    const int X0 = (lt % V.tiles_x) * TT, Y0 = (lt / V.tiles_x) * TT;
    const int tid = threadIdx.x;
    const int rho = (g.edge_mode == 0) ? min(V.rho, RHO_MAX) : 0;
    const int hs = TT + 2 * rho;
    const int wlim = min(TT, V.W - X0), hlim = min(TT, V.H - Y0);   // tile part inside the image

    for (int i = tid; i < hs * hs; i += NT) {
        const int hx = X0 - rho + i % hs, hy = Y0 - rho + i / hs;
        S.sh[i] = (hx >= 0 && hy >= 0 && hx < V.W && hy < V.H) ? 0 : 2;
    }
    constexpr bool EXTRA = MODE >= 4;
    constexpr bool BWD = MODE == 1 || MODE == 2 || MODE == 4 || MODE == 5;
    constexpr bool from_ids = MODE == 2 || MODE == 3 || MODE == 4 || MODE == 7;
    const bool light_grad = EXTRA && g.glight != nullptr && g.shade_mode >= 2;
    float *glacc = light_grad ? gl_slots[tid] : nullptr;
    if (light_grad) glacc[0] = glacc[1] = glacc[2] = 0.f;
    bool single_chunk = false;
    bool empty = false;   // a forward over a tile that no face reaches
    unsigned n_pairs = 0, n_exact = 0, n_cand = 0, n_layers = 0;
    float l2acc = 0.f;   // the fused L2 loss: this thread's sum of squares
    if (!from_ids) {
        const long long lb = g.tile_off[t], le = g.tile_off[t + 1];
        const bool fallback = le > g.list_cap;
        const int n = fallback ? M.nF : (int)(le - lb);
        if (fallback && tid == 0) atomicOr(g.status, DRESSI_DEV_TILE_OVERFLOW);
        // an adjoint over a tile no face reaches has nothing to propagate
        if (BWD && n == 0) return;
        // a forward over such a tile has no layer and S^H = 0 in the tile and its ring (no
        // face comes within the binning radius), so E = 0 or no layer to blend: background
        empty = n == 0;
        if (!empty)   // 16-byte stores (TT^2 K is even; kbuf is 16-byte aligned)
            for (int i = tid; i < TT * TT * K / 2; i += NT)
                reinterpret_cast<ulonglong2 *>(kbuf)[i] = make_ulonglong2(EMPTY, EMPTY);
        if (BWD && g.kth && *g.kth_flag) {
            // the forward's K-th (key, id) of every pixel as a first entry of its K-list: it
            // is the K-th smallest of the pixel's candidates, so it stays in the last slot and
            // every pair whose key bound exceeds it is culled; its own pair finds it there
            __syncthreads();   // after the clearing stores
            for (int p = tid; p < TT * TT; p += NT) {
                const int lx = p % TT, ly = p / TT;
                if (lx < wlim && ly < hlim)
                    kbuf[kslot<TT>(lx, ly) * K + K - 1] = g.kth[V.slot_base + (long long)(Y0 + ly) * V.W + (X0 + lx)];
            }
        }
        single_chunk = n <= CH;
        // the id -> slot hash serves the forward's shading of a tile staged in one chunk
        const bool use_hash = !BWD && single_chunk;
        for (int c0 = 0; c0 < n; c0 += CH) {
            const int nch = min(CH, n - c0);
            // the next chunk's face ids, loaded under this chunk's staging: their records
            // are prefetched into L2 once this chunk is staged
            const int nnext = min(CH, n - c0 - CH);
            int fnext = -1;
            if (tid < nnext) fnext = fallback ? c0 + CH + tid : g.lists[lb + c0 + CH + tid];
            __syncthreads();   // previous chunk consumed
            if (use_hash) {
                for (int i = tid; i < HASH; i += NT) S.hash[i] = make_int2(-1, -1);
                __syncthreads();
            }
            int cnt = 0, hcnt = 0;
            if (tid < nch) {
                const int f = fallback ? c0 + tid : g.lists[lb + c0 + tid];
                FaceGeo &R = S.F[tid];
                S.fid[tid] = f;
                const bool live = face_stage(g, V, M, f, R);
                Box B;
                make_pre(R, live, (float)X0, (float)Y0, V.r_px, S.P[tid], B);
                if (live) {
                    // pixel centres lx + 1/2 inside [bx0, bx1] (grown by r), clipped to the tile and image
                    const int x0 = max(0, (int)ceilf(B.bx0 - 0.5f - APPROX_EPS));
                    const int x1 = min(wlim - 1, (int)floorf(B.bx1 - 0.5f + APPROX_EPS));
                    const int y0 = max(0, (int)ceilf(B.by0 - 0.5f - APPROX_EPS));
                    const int y1 = min(hlim - 1, (int)floorf(B.by1 - 0.5f + APPROX_EPS));
                    const int w = x1 - x0 + 1, h = y1 - y0 + 1;
                    if (w > 0 && h > 0) {
                        cnt = ((w + 3) >> 2) * h;   // segments of up to 4 pixels per row
                        S.rect[tid] = x0 | (y0 << 8) | (w << 16) | (h << 24);
                        S.rdiv[tid] = rect_div((w + 3) >> 2);
                    }
                    if (rho > 0) {
                        // hard bbox (without r) against the ring [-rho, TT + rho), clipped to the image
                        const float r = V.r_px;
                        const int hx0 = max(max(-rho, -X0), (int)ceilf(B.bx0 + r - 0.5f - APPROX_EPS));
                        const int hx1 = min(min(TT + rho, V.W - X0) - 1, (int)floorf(B.bx1 - r - 0.5f + APPROX_EPS));
                        const int hy0 = max(max(-rho, -Y0), (int)ceilf(B.by0 + r - 0.5f - APPROX_EPS));
                        const int hy1 = min(min(TT + rho, V.H - Y0) - 1, (int)floorf(B.by1 - r - 0.5f + APPROX_EPS));
                        // only faces reaching outside the tile interior have ring pixels; a box
                        // that leaves the tile across one side only is cut to its part outside
                        const bool ring = hx0 < 0 || hy0 < 0 || hx1 >= TT || hy1 >= TT;
                        int rx0 = hx0, rx1 = hx1, ry0 = hy0, ry1 = hy1;
                        if (hx0 >= 0 && hx1 < TT) {
                            if (hy1 < TT) ry1 = min(hy1, -1);
                            else if (hy0 >= 0) ry0 = max(hy0, TT);
                        } else if (hy0 >= 0 && hy1 < TT) {
                            if (hx1 < TT) rx1 = min(hx1, -1);
                            else if (hx0 >= 0) rx0 = max(hx0, TT);
                        }
                        const int hw = rx1 - rx0 + 1, hh = ry1 - ry0 + 1;
                        if (hw > 0 && hh > 0 && ring) {
                            hcnt = hw * hh;
                            S.hrect[tid] = (rx0 + 16) | ((ry0 + 16) << 8) | (hw << 16) | (hh << 24);
                            S.hdiv[tid] = rect_div(hw);
                        }
                    }
                    // id -> slot for the shading phase
                    if (use_hash) {
                        unsigned hsh = ((unsigned)f * 2654435761u) & (HASH - 1);
                        for (int probe = 0; probe < HASH; ++probe) {
                            const int prev = atomicCAS(&S.hash[hsh].x, -1, f);
                            if (prev == -1 || prev == f) { S.hash[hsh].y = tid; break; }
                            hsh = (hsh + 1) & (HASH - 1);
                        }
                    }
                }
            }
            if ((unsigned)fnext < (unsigned)M.nF) {
                // both 128-byte lines a 112-byte record can touch
                const char *a = reinterpret_cast<const char *>(g.frec + V.frec_off + fnext);
                prefetch_l2(a);
                prefetch_l2(a + sizeof(FaceRec) - 1);
            }
            // exclusive prefix of the two pair counts over the chunk
            {
                const int lane = tid & 31, wp = tid >> 5;
                int a = cnt, b = hcnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int ya = __shfl_up_sync(0xffffffffu, a, o), yb = __shfl_up_sync(0xffffffffu, b, o);
                    if (lane >= o) { a += ya; b += yb; }
                }
                if (lane == 31) { S.wsum[0][wp] = a; S.wsum[1][wp] = b; }
                __syncthreads();
                int oa = 0, ob = 0, ta = 0, tb = 0;
#pragma unroll
                for (int w = 0; w < NT / 32; ++w) {
                    const int va = S.wsum[0][w], vb = S.wsum[1][w];
                    if (w < wp) { oa += va; ob += vb; }
                    ta += va; tb += vb;
                }
                if (tid < CH) {
                    S.start[tid] = oa + a - cnt;
                    S.hstart[tid] = ob + b - hcnt;
                    fill_blocks(blk, tid, oa + a - cnt, cnt);
                    fill_blocks(hblk, tid, ob + b - hcnt, hcnt);
                }
                if (tid == 0) { S.totals[0] = ta; S.totals[1] = tb; S.item_ctr = 0; }
            }
            __syncthreads();
            const int total = S.totals[0], htotal = S.totals[1];
            raster_items<K, TT>(S, kbuf, qbuf + (tid >> 5) * WQ, blk, V, X0, Y0, nch, total, g.stats != nullptr,
                                n_pairs, n_exact, n_cand);
            // (face, pixel) pairs of the ring: hard test only
            for (int i = tid; i < htotal; i += NT) {
                const int f = pair_face(S.hstart, hblk, nch, i - (tid & 31), i);
                const int rc = S.hrect[f];
                int x, y;
                rect_xy(i - S.hstart[f], (rc >> 16) & 0xff, S.hdiv[f], x, y);
                x += (rc & 0xff) - 16;
                y += ((rc >> 8) & 0xff) - 16;
                if (x >= 0 && x < TT && y >= 0 && y < TT) continue;   // interior: decided by the peel
                const int si = (y + rho) * hs + (x + rho);
                if (S.sh[si] != 0) continue;
                const Pre &P = S.P[f];
                const float fx = (float)x + 0.5f, fy = (float)y + 0.5f;
                const float fmin = approx_fmin(P, fx, fy);
                if (fmin < -APPROX_EPS) continue;
                // clearly inside (margin far above the FP32 error of either test) or
                // decided by the exact fill-rule test
                if (fmin > APPROX_EPS || hard_test(S.F[f], (float)(X0 + x) + 0.5f, (float)(Y0 + y) + 0.5f))
                    S.sh[si] = 1;
            }
        }
        __syncthreads();
        // S^H of the tile's own pixels from the front slot
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const int p = tid + j * NT;
            const int lx = p % TT, ly = p / TT;
            if (empty || lx >= wlim || ly >= hlim) continue;
            const int ks = kslot<TT>(lx, ly) * K;
            if (!BWD && g.kth) g.kth[V.slot_base + (long long)(Y0 + ly) * V.W + (X0 + lx)] = kbuf[ks + K - 1];
            const unsigned long long v = kbuf[ks];
            const bool sh = v != EMPTY && kept_hard(g, V, M, v, (float)(X0 + lx) + 0.5f, (float)(Y0 + ly) + 0.5f);
            S.sh[(ly + rho) * hs + (lx + rho)] = sh ? 1 : 0;
        }
    } else {
        // layers stored by the forward: S^H of the tile and of its ring is the hard flag
        // of every pixel's stored front layer (a non-negative id: hard; bit 31: soft)
        bool any = false;   // some pixel of the tile itself holds a layer
        // every load of the thread's share is issued before the first result is used
        constexpr int HI = (HS_MAX * HS_MAX + NT - 1) / NT;
        int fl[HI];
        unsigned loaded = 0u;   // bit u: entry u is inside the halo and the image
#pragma unroll
        for (int u = 0; u < HI; ++u) {
            const int i = tid + u * NT;
            fl[u] = -1;
            if (i < hs * hs && S.sh[i] != 2) {
                const int hx = i % hs - rho, hy = i / hs - rho;
                fl[u] = __ldg(g.ids_in + V.pix_off + (long long)(Y0 + hy) * V.W + (X0 + hx));
                loaded |= 1u << u;
            }
        }
#pragma unroll
        for (int u = 0; u < HI; ++u) {
            if (!((loaded >> u) & 1u)) continue;
            const int i = tid + u * NT;
            const int hx = i % hs - rho, hy = i / hs - rho;
            S.sh[i] = fl[u] >= 0 ? 1 : 0;
            any |= fl[u] != -1 && hx >= 0 && hy >= 0 && hx < TT && hy < TT;
        }
        // an adjoint over a tile whose pixels hold no layer has nothing to propagate; a
        // forward over it writes the background
        const bool some = __syncthreads_or(any);
        if (BWD && !some) return;
        empty = !some;
    }
    __syncthreads();
    if (g.edge_mode == 0 && !empty) {
        // per halo row, the columns holding S^H = 0 and S^H = 1 (hs <= 48 fits 64 bits)
        const int lane = tid & 31;
        for (int row = tid >> 5; row < hs; row += NT / 32) {
            unsigned long long b0 = 0ull, b1 = 0ull;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int col = half * 32 + lane;
                const unsigned char v = col < hs ? S.sh[row * hs + col] : (unsigned char)2;
                b0 |= (unsigned long long)__ballot_sync(0xffffffffu, v == 0) << (32 * half);
                b1 |= (unsigned long long)__ballot_sync(0xffffffffu, v == 1) << (32 * half);
            }
            if (lane == 0) { S.m0[row] = b0; S.m1[row] = b1; }
        }
        __syncthreads();
    }

    if constexpr (MODE == 2) {
        n_layers = adjoint_queued<K, TT>(g, S, V, M, X0, Y0, rho, wlim, hlim);
    } else if (empty) {
        // background: no layer, RGBA 0 (the loss's gradient 2 (0 - target))
        for (int j = 0; j < PPT; ++j) {
            const int p = tid + j * NT;
            const int lx = p % TT, ly = p / TT;
            if (lx >= wlim || ly >= hlim) continue;
            const long long pix = V.pix_off + (long long)(Y0 + ly) * V.W + (X0 + lx);
            if (g.ids)
#pragma unroll
                for (int k = 0; k < K; ++k) g.ids[(long long)k * g.n_pix + pix] = -1;
            const float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
            reinterpret_cast<float4 *>(g.out)[pix] = o;
            if (g.l2_target) {
                const float4 tg = __ldg(reinterpret_cast<const float4 *>(g.l2_target) + pix);
                const float dx = o.x - tg.x, dy = o.y - tg.y, dz = o.z - tg.z, dw = o.w - tg.w;
                reinterpret_cast<float4 *>(g.l2_grad)[pix] = make_float4(2.f * dx, 2.f * dy, 2.f * dz, 2.f * dw);
                l2acc += dx * dx + dy * dy + dz * dz + dw * dw;
            }
        }
    } else for (int j = 0; j < PPT; ++j) {
        const int p = tid + j * NT;
        const int lx = p % TT, ly = p / TT;
        const bool in = lx < wlim && ly < hlim;
        // the forward's shading and the re-rasterizing adjoint are warp-collective: every
        // lane takes part
        if (BWD && MODE != 1 && !in) continue;
        int ids[K];
        unsigned hardbits = 0u;
#pragma unroll
        for (int k = 0; k < K; ++k) ids[k] = 0x7fffffff;
        if (!in) {
        } else if (!from_ids) {
            const int ks = kslot<TT>(lx, ly) * K;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const unsigned long long v = kbuf[ks + k];
                ids[k] = (v == EMPTY) ? 0x7fffffff : (int)(unsigned int)(v & 0xffffffffu);
            }
            if (!BWD && g.ids) {
                // hard flags of the stored layers; the front one is S^H itself
                hardbits = S.sh[(ly + rho) * hs + (lx + rho)] == 1 ? 1u : 0u;
#pragma unroll
                for (int k = 1; k < K; ++k) {
                    const unsigned long long v = kbuf[ks + k];
                    if (v != EMPTY && kept_hard(g, V, M, v, (float)(X0 + lx) + 0.5f, (float)(Y0 + ly) + 0.5f))
                        hardbits |= 1u << k;
                }
            }
        } else {
            const long long pix = V.pix_off + (long long)(Y0 + ly) * V.W + (X0 + lx);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int id = __ldg(g.ids_in + (long long)k * g.n_pix + pix);
                ids[k] = id == -1 ? 0x7fffffff : (id & 0x7fffffff);
            }
        }
        if constexpr (MODE == 1)
            n_layers += adjoint_warp<K, TT>(g, S, V, M, X0, Y0, p, rho, in, ids);
        else if constexpr (BWD)
            n_layers += adjoint_pixel<K, TT, EXTRA>(g, S, V, M, X0, Y0, lx, ly, rho, ids, glacc);
        else
            n_layers += finish_forward<K, TT, EXTRA>(g, S, V, M, X0, Y0, p, rho, in, ids, hardbits, single_chunk, l2acc);
    }
    if (!BWD && g.l2_loss) {
        // this tile's share of the fused L2 loss: warp sums, one atomic per warp
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l2acc += __shfl_xor_sync(0xffffffffu, l2acc, o);
        if ((tid & 31) == 0 && l2acc != 0.f) atomicAdd(g.l2_loss, l2acc);
    }
    if (light_grad) {
        // this tile's dL/dlight: warp sums, one atomic per warp and component
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float v = glacc[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((tid & 31) == 0 && v != 0.f) atomicAdd(g.glight + 3 * (long long)S.view + c, v);
        }
    }
    if (g.stats) {
        // work counters: pairs enumerated, exact evaluations, candidates kept, layers shaded
        unsigned long long c[4] = {n_pairs, n_exact, n_cand, n_layers};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c[q] += __shfl_xor_sync(0xffffffffu, c[q], o);
            if ((threadIdx.x & 31) == 0) atomicAdd(g.stats + q, c[q]);
        }
    }
}

// one CTA per tile.  CTAs per SM (measured best): four for the forward (64 registers),
// for the layer-queued adjoint from stored ids (64, a few spills: more warps beat the
// registers for its gathers; five, at 48 registers, spill too much) and for the adjoint
// that re-rasterizes, which holds both the raster and the adjoint state (64 registers and
// spills, but four CTAs beat three at 80 registers by 4 % on the 2048^2 views); three for
// the instantiations with the normal map, the light gradient and the inverse UV.
template <int MODE, int TT>
constexpr int tile_min_ctas()
{
    return (MODE == 4 || MODE >= 6) ? 3 : 4;
}

template <int K, int MODE, int TT>
__global__ void __launch_bounds__(NT, tile_min_ctas<MODE, TT>()) k_tile(Globals g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    unsigned long long *kbuf = reinterpret_cast<unsigned long long *>(smem_raw + sizeof(Smem));
    tile_body<K, MODE, TT>(g, S, kbuf, blockIdx.x);
}

// persistent: as many CTAs as fit on the GPU pull tiles from one queue, in the
// order of g.tile_order (longest face list first) when it is given
template <int K, int MODE, int TT>
__global__ void __launch_bounds__(NT, tile_min_ctas<MODE, TT>()) k_tile_persistent(Globals g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    unsigned long long *kbuf = reinterpret_cast<unsigned long long *>(smem_raw + sizeof(Smem));
    for (;;) {
        if (threadIdx.x == 0) S.next = atomicAdd(g.queue, 1);
        __syncthreads();
        const int q = S.next;
        if (q >= g.total_tiles) break;
        const int t = g.tile_order ? g.tile_order[q] : q;
        tile_body<K, MODE, TT>(g, S, kbuf, t);
        __syncthreads();   // the tile's shared memory is free again
    }
}

template <int K, int MODE, int TT>
constexpr size_t tile_smem_bytes()
{
    // from stored ids: the first part of Smem; otherwise Smem, the K-lists, the
    // candidate queue, the two pair-block tables; the adjoints with extras add the
    // per-thread dL/dlight slots
    return (MODE == 2   ? adj_smem_bytes<K>()
            : MODE == 3 || MODE == 4 || MODE == 7
                ? offsetof(Smem, F)
                : sizeof(Smem) + sizeof(unsigned long long) * TT * TT * K + sizeof(unsigned) * QN + 2 * NBLK) +
           (MODE == 4 || MODE == 5 ? sizeof(float) * 3 * NT : 0);
}
// four forward CTAs of the default configuration (K = 3, 16 px tiles) per SM: 228 KB of
// shared memory per SM, 1 KB of it reserved per CTA
static_assert(4 * (tile_smem_bytes<3, 0, 16>() + 1024) <= 228 * 1024, "K = 3 forward tiles no longer fit four CTAs per SM");
static_assert(4 * (tile_smem_bytes<3, 0, 32>() + 1024) <= 228 * 1024, "K = 3, 32 px forward tiles no longer fit four CTAs per SM");
static_assert(4 * (tile_smem_bytes<3, 2, 32>() + 1024) <= 228 * 1024,
              "K = 3 adjoint from stored ids no longer fits four CTAs per SM");

constexpr int LAUNCH_MAX_DEVICES = 64;

template <int K, int MODE, int TT>
static void launch_kk(const Globals &g, cudaStream_t s)
{
    // per device (the caller's current one): the shared-memory attribute above 48 KB is a
    // property of the function in each device's context, and the persistent grid follows
    // that device's SM count and occupancy.  Devices past LAUNCH_MAX_DEVICES are configured
    // on every launch.
    static std::atomic<bool> ready[LAUNCH_MAX_DEVICES];
    static int per_sm_of[LAUNCH_MAX_DEVICES], sms_of[LAUNCH_MAX_DEVICES];
    static std::mutex mu;
    const size_t smem = tile_smem_bytes<K, MODE, TT>();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    const bool cached = dev >= 0 && dev < LAUNCH_MAX_DEVICES;
    int per_sm = 1, sms = 1;
    if (cached && ready[dev].load(std::memory_order_acquire)) {
        per_sm = per_sm_of[dev];
        sms = sms_of[dev];
    } else {
        std::lock_guard<std::mutex> lock(mu);
        cudaFuncSetAttribute(k_tile<K, MODE, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_tile_persistent<K, MODE, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev < 0 ? 0 : dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_persistent<K, MODE, TT>, NT, smem);
        if (per_sm < 1) per_sm = 1;
        if (sms < 1) sms = 1;
        if (cached) {
            per_sm_of[dev] = per_sm;
            sms_of[dev] = sms;
            ready[dev].store(true, std::memory_order_release);
        }
    }
    if (g.persistent) {
        const int grid = std::min(g.total_tiles, per_sm * sms);
        k_tile_persistent<K, MODE, TT><<<grid, NT, smem, s>>>(g);
    } else {
        k_tile<K, MODE, TT><<<g.total_tiles, NT, smem, s>>>(g);
    }
}

template <int MODE, int TT>
static void launch_k(const Globals &g, cudaStream_t s)
{
    switch (g.K) {
    case 1: launch_kk<1, MODE, TT>(g, s); break;
    case 2: launch_kk<2, MODE, TT>(g, s); break;
    case 3: launch_kk<3, MODE, TT>(g, s); break;
    case 4: launch_kk<4, MODE, TT>(g, s); break;
    default: launch_kk<5, MODE, TT>(g, s); break;
    }
}

// the per-tile kernel of one mode (0 forward, 1 adjoint re-rasterizing, 2 adjoint from
// stored layer ids, 3 forward from stored layer ids, 4 / 5 / 6 / 7: 2 / 1 / 0 / 3 with the
// normal map, the light gradient and the inverse UV); instantiated by that mode's
// translation unit
template <int MODE>
void launch_tile_mode(const Globals &g, cudaStream_t s)
{
    if (g.tile == 32) launch_k<MODE, 32>(g, s);
    else launch_k<MODE, 16>(g, s);
}

}  // namespace dressi
