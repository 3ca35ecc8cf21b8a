// dressi_setup.cu -- per-vertex and per-face stages: double-float vertex transform,
// vertex normals, tile binning (count / scan / fill) and the per-vertex end of
// the adjoint (screen -> clip -> object space, normals -> positions).
#include "dressi_core.cuh"
#include "dressi_launch.h"

namespace dressi {

// ---------------------------------------------------------------------------
// vertex transform (render-graph listing: homogeneous position, MVP, face lookup)
// clip = MVP (p, 1), X = (x/w + 1)/2 W, Y = (y/w + 1)/2 H, depth z/w, evaluated in
// double-float arithmetic (an unevaluated sum hi + lo of two FP32 numbers, ~2^-45
// relative accuracy) built from the error-free transformations two-sum (Knuth) and
// two-product with FMA (as in Ogita, Rump and Oishi, "Accurate sum and dot product",
// 2005).  The screen position comes out as the float pair the records keep; products
// of FP32 inputs are exact, so integer geometry with w = 1 stays exact.  GB300's FP64
// rate is low, FP32 is not.
// ---------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ DF quick_two_sum(float a, float b)   // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ DF df_add(DF x, DF y)
{
    const DF s = two_sum(x.hi, y.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ DF df_mul(DF x, DF y)
{
    const DF p = two_prod(x.hi, y.hi);
    return quick_two_sum(p.hi, __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo)));
}

__device__ __forceinline__ DF df_mul_f(DF x, float b)
{
    const DF p = two_prod(x.hi, b);
    return quick_two_sum(p.hi, __fmaf_rn(x.lo, b, p.lo));
}

// 1 / w: the rounded reciprocal and one Newton correction from the exact residual
__device__ __forceinline__ DF df_recip(DF w)
{
    const float r = __frcp_rn(w.hi);
    const float e = __fmaf_rn(-w.lo, r, __fmaf_rn(-w.hi, r, 1.f));   // 1 - w r (w.hi r exact in the FMA)
    return quick_two_sum(r, __fmul_rn(e, r));
}

__global__ void k_vertex(Globals g)
{
    const ViewK &V = g.views[blockIdx.y];
    const MeshK &M = g.meshes[V.mesh];
    VRec *out = g.vrec + V.vrec_off;
    const long long nvt = g.n_verts_total;
    bool bad = false;
    // this view's tiles: the tile -> view table, and cleared bin counters when the face table
    // will count into them
    const int nt = V.tiles_x * V.tiles_y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += gridDim.x * blockDim.x) {
        g.tile_view[V.tile_base + i] = blockIdx.y;
        if (g.zero_bins) {
            g.tile_count[V.tile_base + i] = 0;
            g.tile_cursor[V.tile_base + i] = 0;
        }
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M.nV; i += gridDim.x * blockDim.x) {
        const long long gi = M.vert_off + i;
        const float p0 = __ldg(g.pos + gi), p1 = __ldg(g.pos + nvt + gi), p2 = __ldg(g.pos + 2 * nvt + gi);
        DF c[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float *m = V.mvp + 4 * r;
            c[r] = df_add(df_add(df_add(two_prod(m[0], p0), two_prod(m[1], p1)), two_prod(m[2], p2)), DF{m[3], 0.f});
        }
        const DF iw = df_recip(c[3]);
        const DF X = df_mul_f(df_add(df_mul(c[0], iw), DF{1.f, 0.f}), 0.5f * (float)V.W);
        const DF Y = df_mul_f(df_add(df_mul(c[1], iw), DF{1.f, 0.f}), 0.5f * (float)V.H);
        const DF Z = df_mul(c[2], iw);
        VRec r;
        r.xh = X.hi;
        r.xl = X.lo;
        r.yh = Y.hi;
        r.yl = Y.lo;
        r.z = Z.hi;
        r.iw = iw.hi;
        const bool fin = isfinite(X.hi) && isfinite(Y.hi) && isfinite(Z.hi) && isfinite(X.lo) && isfinite(Y.lo);
        // the signs of w - 1e-6, Z and 1 - Z from the pairs (hi carries the sign unless it is 0)
        const bool w_pos = c[3].hi > 1e-6f || (c[3].hi == 1e-6f && c[3].lo > 0.f);
        const bool z_ge0 = Z.hi > 0.f || (Z.hi == 0.f && Z.lo >= 0.f);
        const bool z_le1 = Z.hi < 1.f || (Z.hi == 1.f && Z.lo <= 0.f);
        r.valid = w_pos && z_ge0 && z_le1 && fin && fabsf(X.hi) < 1e30f && fabsf(Y.hi) < 1e30f;
        r.pad = 0;
        if (!(isfinite(p0) && isfinite(p1) && isfinite(p2))) bad = true;
        out[i] = r;
    }
    if (bad) atomicOr(g.status, DRESSI_DEV_NONFINITE);
}

// ---------------------------------------------------------------------------
// area-weighted vertex normals (listing BuildNormalCompute): m_v = sum of
// (P1 - P0) x (P2 - P0) over the faces holding v, n_v = m_v / |m_v|.
// The sum runs over a vertex -> face adjacency in increasing face order, so the
// normals (and everything shaded with them) are bitwise reproducible.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool face_vertices(const Globals &g, const MeshK &M, int f, int v[3])
{
    const int *fv = g.faces + 3 * (M.face_off + f);
    v[0] = __ldg(fv); v[1] = __ldg(fv + 1); v[2] = __ldg(fv + 2);
    return (unsigned)v[0] < (unsigned)M.nV && (unsigned)v[1] < (unsigned)M.nV && (unsigned)v[2] < (unsigned)M.nV;
}

template <int PASS>
__global__ void k_adjacency(Globals g)
{
    const MeshK &M = g.meshes[blockIdx.y];
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < M.nF; f += gridDim.x * blockDim.x) {
        int v[3];
        if (!face_vertices(g, M, f, v)) continue;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const long long gv = M.vert_off + v[j];
            if (PASS == 0) atomicAdd(g.adj_off + gv, 1);
            else g.adj[g.adj_off[gv] + atomicAdd(g.adj_cur + gv, 1)] = f;
        }
    }
}

__global__ void k_normal_csr(Globals g)
{
    const MeshK &M = g.meshes[blockIdx.y];
    const long long nvt = g.n_verts_total;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M.nV; i += gridDim.x * blockDim.x) {
        const long long gv = M.vert_off + i;
        const int b = g.adj_off[gv], e = g.adj_off[gv + 1];
        float m0 = 0.f, m1 = 0.f, m2 = 0.f;
        // incident faces in increasing id order (the lists are short: pick the next
        // larger id each round)
        int last = -1;
        for (int round = b; round < e; ++round) {
            int f = 0x7fffffff;
            for (int q = b; q < e; ++q) {
                const int c = g.adj[q];
                if (c > last && c < f) f = c;
            }
            if (f == 0x7fffffff) break;
            last = f;
            int v[3];
            face_vertices(g, M, f, v);
            float P[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int c = 0; c < 3; ++c) P[j][c] = __ldg(g.pos + c * nvt + M.vert_off + v[j]);
            const float u[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
            const float w[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
            m0 += u[1] * w[2] - u[2] * w[1];
            m1 += u[2] * w[0] - u[0] * w[2];
            m2 += u[0] * w[1] - u[1] * w[0];
        }
        const float l = sqrtf(m0 * m0 + m1 * m1 + m2 * m2);
        const float s = l > 0.f ? 1.f / l : 0.f;
        g.nrm[gv] = make_float4(m0 * s, m1 * s, m2 * s, l);
    }
}

// ---------------------------------------------------------------------------
// tile binning: every live face goes into the list of each tile that its
// bounding box, grown by bin_R pixels (r plus the edge-mask halo plus a guard),
// touches.  The face table kernel counts, k_bin fills.  Order inside a list is
// irrelevant: the peel keeps the K smallest (key, id) pairs.
// ---------------------------------------------------------------------------
// the tiles [tx0, tx1] x [ty0, ty1] that the grown box of screen corners (xh, yh)
// touches; false when it misses the view
__device__ __forceinline__ bool bin_rect(const Globals &g, const ViewK &V, const float (&xh)[3], const float (&yh)[3],
                                         int &tx0, int &tx1, int &ty0, int &ty1)
{
    const float Tinv = 1.f / (float)g.tile;
    const float x0 = fminf(xh[0], fminf(xh[1], xh[2])) - V.bin_R;
    const float x1 = fmaxf(xh[0], fmaxf(xh[1], xh[2])) + V.bin_R;
    const float y0 = fminf(yh[0], fminf(yh[1], yh[2])) - V.bin_R;
    const float y1 = fmaxf(yh[0], fmaxf(yh[1], yh[2])) + V.bin_R;
    if (x1 < 0.f || y1 < 0.f || x0 > (float)V.W || y0 > (float)V.H) return false;
    tx0 = max(0, (int)floorf(x0 * Tinv));
    tx1 = min(V.tiles_x - 1, (int)floorf(x1 * Tinv));
    ty0 = max(0, (int)floorf(y0 * Tinv));
    ty1 = min(V.tiles_y - 1, (int)floorf(y1 * Tinv));
    return tx0 <= tx1 && ty0 <= ty1;
}

// A face's tile rect [tx0, tx1] x [ty0, ty1], packed into one word for the list fill:
// tx0 | ty0 << 11 | (tx1 - tx0) << 22 | (ty1 - ty0) << 27.  Tile coordinates are below
// 2048 (views of at most 32,768 pixels at 16 px tiles); a rect more than 32 tiles wide or
// high is BRECT_WIDE, and the list fill takes it from the face record.  Neither marker
// is a valid packing (both would put tx0 + (tx1 - tx0) past 2047).
constexpr unsigned BRECT_NONE = 0xffffffffu;   // no tile: culled, or off the view
constexpr unsigned BRECT_WIDE = 0xfffffffeu;

__device__ __forceinline__ unsigned pack_brect(bool any, int tx0, int tx1, int ty0, int ty1)
{
    if (!any) return BRECT_NONE;
    if (tx1 - tx0 > 31 || ty1 - ty0 > 31) return BRECT_WIDE;
    return (unsigned)tx0 | ((unsigned)ty0 << 11) | ((unsigned)(tx1 - tx0) << 22) | ((unsigned)(ty1 - ty0) << 27);
}

// the (face, tile) pairs of a warp's faces, one step per tile of each lane's box: the
// lanes at the same tile in a step share one atomic (consecutive faces of a mesh are
// mostly neighbours), and PASS 1 gives them consecutive list slots.  All 32 lanes call it.
template <int PASS>
__device__ __forceinline__ void bin_walk(const Globals &g, const ViewK &V, int f, bool any, int tx0, int tx1,
                                         int ty0, int ty1)
{
    const int lane = threadIdx.x & 31;
    int tx = tx0, ty = ty0;
    bool more = any;
    while (__any_sync(0xffffffffu, more)) {
        const int t = more ? V.tile_base + ty * V.tiles_x + tx : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, t);
        if (more) {
            const int leader = __ffs(grp) - 1;
            if (PASS == 0) {
                if (lane == leader) atomicAdd(g.tile_count + t, __popc(grp));
            } else {
                int base = 0;
                if (lane == leader) base = atomicAdd(g.tile_cursor + t, __popc(grp));
                base = __shfl_sync(grp, base, leader) + __popc(grp & ((1u << lane) - 1u));
                const long long idx = (long long)g.tile_off[t] + base;
                if (idx < g.list_cap) g.lists[idx] = f;
            }
            if (++tx > tx1) {
                tx = tx0;
                if (++ty > ty1) more = false;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// face table: the record of every (view, face) -- screen corners, canonical edges,
// lengths, area, flags -- built once per call and read by binning, staging,
// shading and the adjoint (112 bytes each).  COUNT: also the tile counts of the
// binning (the lists' lengths).
// ---------------------------------------------------------------------------
template <bool COUNT>
__global__ void __launch_bounds__(256) k_face(Globals g)
{
    // each warp's 32 records (7 float4 each) go through shared memory so that the warp
    // writes its 3,584 contiguous bytes with full-line stores
    __shared__ float4 stage[256 / 32][32 * 7];
    const ViewK V = g.views[blockIdx.y];   // copies: the fields stay in registers across the stores
    const MeshK M = g.meshes[V.mesh];
    const VRec *vr = g.vrec + V.vrec_off;
    const int lane = threadIdx.x & 31;
    float4 *ws = stage[threadIdx.x >> 5];
    bool bad = false;
    // block-uniform trip count: every lane of a warp takes part in the binning steps
    for (int f0 = blockIdx.x * blockDim.x; f0 < M.nF; f0 += gridDim.x * blockDim.x) {
        const int f = f0 + threadIdx.x;
        bool live = false;
        FaceRec R;
        if (f < M.nF) {
            face_load(g, M, vr, f, R);
            if (R.flags & FLAG_RANGE) {
                // out of range: nothing else of the record is meaningful
                bad = true;
#pragma unroll
                for (int i = 0; i < 3; ++i) { R.vi[i] = 0; R.xh[i] = R.xl[i] = R.yh[i] = R.yl[i] = 0.f; }
            }
            live = (R.flags & FLAG_LIVE) != 0;
            float4 *d = ws + lane * 7;   // 112-byte lane stride: no bank conflict within 8 lanes
            d[0] = make_float4(R.xh[0], R.xh[1], R.xh[2], R.xl[0]);
            d[1] = make_float4(R.xl[1], R.xl[2], R.yh[0], R.yh[1]);
            d[2] = make_float4(R.yh[2], R.yl[0], R.yl[1], R.yl[2]);
            d[3] = make_float4(R.invL[0], R.invL[1], R.invL[2], R.z[0]);
            d[4] = make_float4(R.z[1], R.z[2], R.invA, __int_as_float(R.flags));
            d[5] = make_float4(__int_as_float(R.id), __int_as_float(R.vi[0]), __int_as_float(R.vi[1]),
                               __int_as_float(R.vi[2]));
            d[6] = make_float4(R.iw[0], R.iw[1], R.iw[2], 0.f);
        }
        __syncwarp();
        {
            const int wf0 = f0 + (threadIdx.x & ~31);   // the warp's first face
            const int nrec = max(0, min(32, M.nF - wf0));
            float4 *dst = reinterpret_cast<float4 *>(g.frec + V.frec_off + wf0);
            for (int i = lane; i < nrec * 7; i += 32) dst[i] = ws[i];
        }
        __syncwarp();   // the staged records are read before the next iteration writes them
        if (COUNT) {
            int tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;
            const bool any = live && bin_rect(g, V, R.xh, R.yh, tx0, tx1, ty0, ty1);
            if (f < M.nF) g.brect[V.frec_off + f] = pack_brect(any, tx0, tx1, ty0, ty1);
            bin_walk<0>(g, V, f, any, tx0, tx1, ty0, ty1);
        }
    }
    if (bad) atomicOr(g.status, DRESSI_DEV_FACE_RANGE);
}

// the list entries of every (face, tile) pair, into the slots the counts' prefix gives;
// each face's tile rect comes packed from the face table kernel
__global__ void k_bin(Globals g)
{
    const ViewK V = g.views[blockIdx.y];   // copies: the fields stay in registers across the stores
    const MeshK M = g.meshes[V.mesh];
    for (int f0 = blockIdx.x * blockDim.x; f0 < M.nF; f0 += gridDim.x * blockDim.x) {
        const int f = f0 + threadIdx.x;
        int tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;
        const unsigned b = f < M.nF ? __ldg(g.brect + V.frec_off + f) : BRECT_NONE;
        bool any = false;
        if (b == BRECT_WIDE) {
            FaceRec R;
            any = face_get(g, V, M, f, R) && bin_rect(g, V, R.xh, R.yh, tx0, tx1, ty0, ty1);
        } else if (b != BRECT_NONE) {
            tx0 = b & 2047;
            ty0 = (b >> 11) & 2047;
            tx1 = tx0 + ((b >> 22) & 31);
            ty1 = ty0 + (b >> 27);
            any = true;
        }
        bin_walk<1>(g, V, f, any, tx0, tx1, ty0, ty1);
    }
}

// ---------------------------------------------------------------------------
// longest-first tile order for the persistent tile kernel: a counting sort of the
// tiles by descending face-list length (lengths bucketed, ties in any order)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lpt_bin(int count) { return LPT_BINS - 1 - min(count, LPT_BINS - 1); }

__global__ void k_lpt_hist(Globals g)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.total_tiles; t += gridDim.x * blockDim.x)
        atomicAdd(g.lpt_hist + lpt_bin(g.tile_count[t]), 1);
}

__global__ void __launch_bounds__(LPT_BINS) k_lpt_scan(Globals g)
{
    __shared__ int warp_sums[LPT_BINS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int v = g.lpt_hist[tid];
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    g.lpt_hist[tid] = x - v + (warp > 0 ? warp_sums[warp - 1] : 0);   // exclusive offsets
}

__global__ void k_lpt_scatter(Globals g)
{
    int *order = const_cast<int *>(g.tile_order);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.total_tiles; t += gridDim.x * blockDim.x)
        order[atomicAdd(g.lpt_hist + lpt_bin(g.tile_count[t]), 1)] = t;
}

// ---------------------------------------------------------------------------
// adjoint, per (view, vertex): (dX, dY, d(1/w)) -> clip -> object space
// ---------------------------------------------------------------------------
__global__ void k_vertex_bwd(Globals g)
{
    const ViewK &V = g.views[blockIdx.y];
    const MeshK &M = g.meshes[V.mesh];
    const float4 *sg = g.sgrad + V.vrec_off;
    const long long nvt = g.n_verts_total;
    // dL/dMVP of this view: dL/dclip_r (p, 1)_c for the x, y and w rows (depth only
    // orders the layers and has no gradient)
    float am[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) am[q] = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M.nV; i += gridDim.x * blockDim.x) {
        float4 s = sg[i];
        if (s.x == 0.f && s.y == 0.f && s.z == 0.f) continue;
        const long long gi = M.vert_off + i;
        const float p[3] = {__ldg(g.pos + gi), __ldg(g.pos + nvt + gi), __ldg(g.pos + 2 * nvt + gi)};
        float c[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float *m = V.mvp + 4 * r;
            c[r] = m[0] * p[0] + m[1] * p[1] + m[2] * p[2] + m[3];
        }
        const float iw = 1.f / c[3];
        const float hx = 0.5f * (float)V.W * iw, hy = 0.5f * (float)V.H * iw;
        const float gcx = s.x * hx, gcy = s.y * hy;
        const float gcw = -(s.x * hx * c[0] + s.y * hy * c[1]) * iw - s.z * iw * iw;
#pragma unroll
        for (int col = 0; col < 3; ++col) {
            float gp = V.mvp[col] * gcx + V.mvp[4 + col] * gcy + V.mvp[12 + col] * gcw;
            atomicAdd(g.gpos + col * nvt + gi, gp);
        }
        if (g.gmvp) {
            const float ph[4] = {p[0], p[1], p[2], 1.f};
#pragma unroll
            for (int col = 0; col < 4; ++col) {
                am[col] = fmaf(gcx, ph[col], am[col]);
                am[4 + col] = fmaf(gcy, ph[col], am[4 + col]);
                am[8 + col] = fmaf(gcw, ph[col], am[8 + col]);
            }
        }
    }
    if (g.gmvp) {
        float *out = g.gmvp + 16 * (long long)blockIdx.y;
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            float v = am[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0 && v != 0.f) atomicAdd(out + (q < 8 ? q : q + 4), v);
        }
    }
}

// normals -> positions: dm_v = (dn_v - n_v (n_v . dn_v)) / |m_v|; per face
// da = sum of dm over its corners; a = u x w gives du = w x da, dw = da x u
__global__ void k_normal_bwd(Globals g)
{
    const MeshK &M = g.meshes[blockIdx.y];
    const long long nvt = g.n_verts_total;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < M.nF; f += gridDim.x * blockDim.x) {
        const int *fv = g.faces + 3 * (M.face_off + f);
        int v[3] = {__ldg(fv), __ldg(fv + 1), __ldg(fv + 2)};
        if ((unsigned)v[0] >= (unsigned)M.nV || (unsigned)v[1] >= (unsigned)M.nV || (unsigned)v[2] >= (unsigned)M.nV)
            continue;
        float ga[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const long long gi = M.vert_off + v[j];
            float4 n = g.nrm[gi];
            float4 dn = g.ngrad[gi];
            if (!(n.w > 0.f)) continue;
            float nd = n.x * dn.x + n.y * dn.y + n.z * dn.z;
            float il = 1.f / n.w;
            ga[0] += (dn.x - n.x * nd) * il;
            ga[1] += (dn.y - n.y * nd) * il;
            ga[2] += (dn.z - n.z * nd) * il;
        }
        if (ga[0] == 0.f && ga[1] == 0.f && ga[2] == 0.f) continue;
        float P[3][3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c) P[j][c] = __ldg(g.pos + c * nvt + M.vert_off + v[j]);
        float u[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
        float w[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
        float gu[3] = {w[1] * ga[2] - w[2] * ga[1], w[2] * ga[0] - w[0] * ga[2], w[0] * ga[1] - w[1] * ga[0]};
        float gw[3] = {ga[1] * u[2] - ga[2] * u[1], ga[2] * u[0] - ga[0] * u[2], ga[0] * u[1] - ga[1] * u[0]};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            atomicAdd(g.gpos + c * nvt + M.vert_off + v[1], gu[c]);
            atomicAdd(g.gpos + c * nvt + M.vert_off + v[2], gw[c]);
            atomicAdd(g.gpos + c * nvt + M.vert_off + v[0], -(gu[c] + gw[c]));
        }
    }
}

// L2 loss helper
__global__ void k_l2(const float *out, const float *tgt, long long n, float *grad, float *loss)
{
    float acc = 0.f;
    const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long done = 0;
    if (((reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(tgt) | reinterpret_cast<uintptr_t>(grad)) &
         15) == 0) {
        // 16-byte accesses over the whole float4s, then the scalar tail
        const long long n4 = n >> 2;
        const float4 *o4 = reinterpret_cast<const float4 *>(out), *t4 = reinterpret_cast<const float4 *>(tgt);
        float4 *g4 = reinterpret_cast<float4 *>(grad);
        for (long long i = i0; i < n4; i += stride) {
            const float4 a = __ldg(o4 + i), b = __ldg(t4 + i);
            const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, dw = a.w - b.w;
            g4[i] = make_float4(2.f * dx, 2.f * dy, 2.f * dz, 2.f * dw);
            acc += dx * dx + dy * dy + dz * dz + dw * dw;
        }
        done = n4 << 2;
    }
    for (long long i = done + i0; i < n; i += stride) {
        const float d = out[i] - tgt[i];
        grad[i] = 2.f * d;
        acc += d * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, acc);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int grid_x(long long n, int block, int cap)
{
    long long b = (n + block - 1) / block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

void launch_vertex(const Globals &g, int n_views, int max_nv, cudaStream_t s)
{
    dim3 grid(grid_x(max_nv, 256, 1024), n_views);
    k_vertex<<<grid, 256, 0, s>>>(g);
    count_launch(1);
}

void launch_normals(const Globals &g, int n_meshes, int max_nf, int max_nv, cudaStream_t s)
{
    // adj_off and adj_cur are zeroed by the caller
    dim3 gf(grid_x(max_nf, 256, 2048), n_meshes), gv(grid_x(max_nv, 256, 2048), n_meshes);
    k_adjacency<0><<<gf, 256, 0, s>>>(g);
    launch_scan_inplace(g.adj_off, (int)(g.n_verts_total + 1), g.scan_partial, s);
    k_adjacency<1><<<gf, 256, 0, s>>>(g);
    k_normal_csr<<<gv, 256, 0, s>>>(g);
    count_launch(3);
}

void launch_face(const Globals &g, int n_views, int max_nf, bool count, cudaStream_t s)
{
    dim3 grid(grid_x(max_nf, 256, 2048), n_views);
    if (count) k_face<true><<<grid, 256, 0, s>>>(g);
    else k_face<false><<<grid, 256, 0, s>>>(g);
    count_launch(1);
}

// after launch_face(count = true): the counts' prefix and the lists
void launch_bin(const Globals &g, int n_views, int max_nf, cudaStream_t s)
{
    dim3 grid(grid_x(max_nf, 256, 2048), n_views);
    // exclusive prefix of the tile counts: tile_off[n] = total list entries
    cudaMemcpyAsync(g.tile_off, g.tile_count, sizeof(int) * (size_t)g.total_tiles, cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(g.tile_off + g.total_tiles, 0, sizeof(int), s);
    launch_scan_inplace(g.tile_off, g.total_tiles + 1, g.scan_partial, s);
    k_bin<<<grid, 256, 0, s>>>(g);
    count_launch(1);
}

void launch_lpt_order(const Globals &g, cudaStream_t s)
{
    const int grid = grid_x(g.total_tiles, 256, 1024);
    k_lpt_hist<<<grid, 256, 0, s>>>(g);
    k_lpt_scan<<<1, LPT_BINS, 0, s>>>(g);
    k_lpt_scatter<<<grid, 256, 0, s>>>(g);
    count_launch(3);
}

void launch_vertex_bwd(const Globals &g, int n_views, int max_nv, int n_meshes, int max_nf, bool normals,
                       cudaStream_t s)
{
    dim3 grid(grid_x(max_nv, 256, 1024), n_views);
    k_vertex_bwd<<<grid, 256, 0, s>>>(g);
    count_launch(1);
    if (normals) {
        dim3 g2(grid_x(max_nf, 256, 2048), n_meshes);
        k_normal_bwd<<<g2, 256, 0, s>>>(g);
        count_launch(1);
    }
}

void launch_l2(const float *out, const float *tgt, long long n, float *grad, float *loss, cudaStream_t s)
{
    k_l2<<<grid_x(n, 256, 152 * 8), 256, 0, s>>>(out, tgt, n, grad, loss);
    count_launch(1);
}

}  // namespace dressi
