/*
 * HardSoftRas FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, brute-force restatement of the soft rasterizer of
 * "Dressi: A Hardware-Agnostic Differentiable Renderer with Reactive Shader
 * Packing and Soft Rasterization" (arXiv 2204.01386), Sec. 3.4, used to check
 * the CUDA path.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline may load it; the product never does.  It shares no code, header or
 * constant with the CUDA library.
 *
 * Everything is FP64.  Per view and per pixel centre p = (x + 1/2, y + 1/2)
 * (pixel units, y down) it evaluates every face and takes, in order:
 *   1. transform      clip = MVP (pos, 1); X = (x/w + 1)/2 W, Y = (y/w + 1)/2 H,
 *                     depth z/w (Eq. of f_render, Sec. 3.4.1; Vulkan clip space)
 *   2. culling        a face is skipped when a corner has w <= 1e-6 or depth
 *                     outside [0, 1], or its screen area is zero (reading: the
 *                     paper does not clip; no back-face culling because depth
 *                     peeling must see occluded and back faces)
 *   3. SignedDist     Euclidean pixel-to-boundary distance, positive inside the
 *                     hard face (Sec. 3.4.2, Alg. 2).  Each edge is evaluated
 *                     from its lexicographically smaller endpoint so that two
 *                     faces sharing an edge or a vertex get identical values.
 *   4. Enlarge        a face is a candidate at p iff dist >= -r (reading of
 *                     Enlarge(): the enlarged face reaches r from the edges)
 *   5. hard test      inside the closed triangle with the top-left fill rule
 *   6. Shift          key = depth/2 if hard else |dist|/2 + 1/2  (Eq. Shift)
 *   7. peel           the K smallest (key, face id) pairs (Alg. 2 outer loop)
 *   8. barycentrics   perspective correct; a soft fragment takes the barycentrics
 *                     of its closest point of the hard face (reading: soft faces
 *                     extend the hard face, Sec. 3.4.2)
 *   9. normals        area-weighted vertex normals (listing BuildNormalCompute)
 *  10. texture        bilinear, texel centres at i + 1/2, REPEAT wrap
 *  11. shading        vertex colour / unlit texture / texture * max(0, n.l) /
 *                     texture * max(0, n'.l) with n' from a tangent-space normal map
 *  12. D_k = sigmoid(dist_k / sigma)                      (Sec. 3.4.3)
 *  13. S^H, edge mask E by a Chebyshev window of radius rho (Sec. 3.4.3)
 *  14-16. blend: I = E I^e + (1 - E) I^ne for colour and silhouette
 *                     (the three blend equations of Sec. 3.4.3)
 * and the reverse-mode adjoint of 8-16 back to positions, colours, texels.
 * Distances handed to sigmoid and Shift are in normalised screen units:
 * pixel distance / max(W, H).
 *
 * Parity unpinned (the paper fixes no value for them, so no pin can): the width rule
 * of E (rho = max(1, round(delta max(W, H))) pixels, a Chebyshev window), perspective-
 * correct rather than screen-linear barycentrics, the colour blend's normalisation by
 * the sum of D_k, and Enlarge read as dist >= -r instead of the paper's grown polygons.
 * These steps follow the readings above; everything else is pinned by closed forms,
 * brute force, a ray-cast renderer and finite differences in the tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXK 8

typedef struct {
    int32_t n_verts, n_faces;
    const double *pos;    /* [n_verts][3] */
    const double *col;    /* [n_verts][3] or NULL */
    const double *uv;     /* [n_verts][2] or NULL */
    const int32_t *faces; /* [n_faces][3] */
    int32_t tex_w, tex_h;
    const double *tex;    /* [tex_h][tex_w][4] or NULL */
    double mvp[16];       /* row-major, clip = mvp (p, 1) */
    double light[3];
    int32_t width, height;
    const double *ntex;   /* [tex_h][tex_w][4] tangent-space normal map (shade_mode 3) or NULL */
} orc_view;

typedef struct {
    int32_t K;
    double r, sigma, delta;
    int32_t edge_mode;  /* 0 edge mask, 1 E = 1 everywhere, 2 E = 0 everywhere */
    int32_t shade_mode; /* 0 vertex colour, 1 unlit texture, 2 texture * Lambert,
                           3 texture * Lambert with a tangent-space normal map */
    int32_t brute_force;/* 1: every face at every pixel; 0: same result, bbox pre-test */
} orc_params;

typedef struct { int32_t x0, y0, w, h; } orc_window;

typedef struct {           /* every pointer optional; sizes in units of the window */
    double *rgba;          /* [h][w][4] */
    int32_t *ids;          /* [K][h][w], -1 where the layer is empty */
    int32_t *hard;         /* [K][h][w] */
    double *dist;          /* [K][h][w] normalised units */
    double *key;           /* [K+1][h][w]; slot K = best unselected candidate (+inf if none) */
    uint8_t *sh;           /* [h][w] hard stencil of the front layer */
    uint8_t *edge;         /* [h][w] edge mask */
    double *margin_hard;   /* [h][w] min |dist| in pixels over faces within r of p */
    double *margin_cand;   /* [h][w] min |dist + r| in pixels over faces */
    int32_t *n_hard;       /* [h][w] number of faces whose hard region holds p */
    uint64_t *feat_hash;   /* [K+1][h][w] identity of each fragment's closest boundary feature
                              (hash of the corner, or of the two corners of the edge, in pixel
                              coordinates; hard fragments hash their face id) -- tells exact ties
                              of one shared feature from coincidences of distinct features */
} orc_fwd_out;

enum { ORC_OK = 0, ORC_BAD_ARG = 1, ORC_FACE_RANGE = 4 };

/* ------------------------------------------------------------------------- */
/* step 1: vertex transform                                                   */
/* ------------------------------------------------------------------------- */
typedef struct { double X, Y, Z, w; } scr_t;

static scr_t transform(const orc_view *v, int i)
{
    const double *p = v->pos + 3 * (size_t)i;
    double c[4];
    for (int r = 0; r < 4; ++r) {
        const double *m = v->mvp + 4 * r;
        c[r] = m[0] * p[0] + m[1] * p[1] + m[2] * p[2] + m[3];
    }
    scr_t s;
    s.X = (c[0] / c[3] + 1.0) * 0.5 * (double)v->width;
    s.Y = (c[1] / c[3] + 1.0) * 0.5 * (double)v->height;
    s.Z = c[2] / c[3];
    s.w = c[3];
    return s;
}

/* ------------------------------------------------------------------------- */
/* step 2: face setup                                                         */
/* ------------------------------------------------------------------------- */
typedef struct {
    int live;
    int vi[3];
    double X[3], Y[3], Z[3], IW[3];
    double A2;      /* twice the signed area (pixel units) */
    double orient;  /* sign of A2 */
    int owns[3];    /* top-left rule: edge i (corner i -> i+1) owns its boundary points */
    double bx0, bx1, by0, by1; /* bbox grown by r (pixels) */
} face_t;

static int setup_faces(const orc_view *v, double r_px, face_t *F)
{
    int status = ORC_OK;
    scr_t *S = (scr_t *)malloc(sizeof(scr_t) * (size_t)(v->n_verts > 0 ? v->n_verts : 1));
    for (int i = 0; i < v->n_verts; ++i) S[i] = transform(v, i);
    for (int f = 0; f < v->n_faces; ++f) {
        face_t *t = &F[f];
        memset(t, 0, sizeof(*t));
        int ok = 1;
        for (int j = 0; j < 3; ++j) {
            int vi = v->faces[3 * f + j];
            if (vi < 0 || vi >= v->n_verts) { ok = 0; status |= ORC_FACE_RANGE; break; }
            t->vi[j] = vi;
        }
        if (!ok) continue;
        for (int j = 0; j < 3; ++j) {
            scr_t s = S[t->vi[j]];
            if (!(s.w > 1e-6) || !(s.Z >= 0.0 && s.Z <= 1.0)) ok = 0;
            t->X[j] = s.X; t->Y[j] = s.Y; t->Z[j] = s.Z; t->IW[j] = 1.0 / s.w;
        }
        if (!ok) continue;
        t->A2 = (t->X[1] - t->X[0]) * (t->Y[2] - t->Y[0]) - (t->X[2] - t->X[0]) * (t->Y[1] - t->Y[0]);
        if (!(t->A2 != 0.0) || !isfinite(t->A2)) continue;
        t->orient = t->A2 > 0 ? 1.0 : -1.0;
        for (int i = 0; i < 3; ++i) {
            int j = (i + 1) % 3;
            double ex = t->X[j] - t->X[i], ey = t->Y[j] - t->Y[i];
            /* inward normal orient * (-ey, ex): a left edge has it pointing to +x,
               a top edge (horizontal, y down) has it pointing to +y */
            t->owns[i] = (t->orient * ey < 0.0) || (ey == 0.0 && t->orient * ex > 0.0);
        }
        t->bx0 = fmin(t->X[0], fmin(t->X[1], t->X[2])) - r_px;
        t->bx1 = fmax(t->X[0], fmax(t->X[1], t->X[2])) + r_px;
        t->by0 = fmin(t->Y[0], fmin(t->Y[1], t->Y[2])) - r_px;
        t->by1 = fmax(t->Y[0], fmax(t->Y[1], t->Y[2])) + r_px;
        t->live = 1;
    }
    free(S);
    return status;
}

/* ------------------------------------------------------------------------- */
/* steps 3-6: SignedDist, candidate rule, hard test, Shift                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    int id, hard;
    double dist_px;   /* signed pixel distance */
    double key;
    double lam[3];    /* screen-space barycentrics (of the closest point for soft fragments) */
    int feat;         /* closest boundary feature: 0..2 edge i interior, 3..5 corner i-3 */
    int segP, segQ;   /* edge feature: canonical endpoints; closest point = P + t (Q - P) */
    double segt;
} frag_t;

static int lex_less(double ax, double ay, double bx, double by)
{
    return ax < bx || (ax == bx && ay < by);
}

/* evaluates face t at p; fills fr and returns the signed pixel distance */
static double eval_face(const face_t *t, int id, double px, double py, double S, frag_t *fr)
{
    double Fnum[3], L[3], seg[3], segt[3];
    int segfeat[3], segP[3], segQ[3];
    int inside = 1;
    for (int i = 0; i < 3; ++i) {
        int a = i, b = (i + 1) % 3;
        int sw = lex_less(t->X[b], t->Y[b], t->X[a], t->Y[a]);
        int P = sw ? b : a, Q = sw ? a : b;
        double dPx = px - t->X[P], dPy = py - t->Y[P];
        double dQx = px - t->X[Q], dQy = py - t->Y[Q];
        double c = dPx * dQy - dPy * dQx;            /* = cross(Q - P, p - P) */
        double ex = t->X[Q] - t->X[P], ey = t->Y[Q] - t->Y[P];
        L[i] = sqrt(ex * ex + ey * ey);
        Fnum[i] = t->orient * (sw ? -c : c);         /* inward-positive, times L */
        if (!(Fnum[i] > 0.0 || (Fnum[i] == 0.0 && t->owns[i]))) inside = 0;
        double tP = dPx * ex + dPy * ey;
        double tQ = dQx * ex + dQy * ey;
        segP[i] = P; segQ[i] = Q; segt[i] = 0.0;
        if (tP <= 0.0) { seg[i] = sqrt(dPx * dPx + dPy * dPy); segfeat[i] = 3 + P; }
        else if (tQ >= 0.0) { seg[i] = sqrt(dQx * dQx + dQy * dQy); segfeat[i] = 3 + Q; }
        else { seg[i] = fabs(c) / L[i]; segfeat[i] = i; segt[i] = tP / (ex * ex + ey * ey); }
    }
    double dist;
    int feat, mseg = 0;
    if (inside) {
        int m = 0;
        double best = Fnum[0] / L[0];
        for (int i = 1; i < 3; ++i) { double d = Fnum[i] / L[i]; if (d < best) { best = d; m = i; } }
        dist = best; feat = m;
    } else {
        int m = 0;
        for (int i = 1; i < 3; ++i) if (seg[i] < seg[m]) m = i;
        dist = -seg[m]; feat = segfeat[m]; mseg = m;
    }
    double absA = fabs(t->A2);
    fr->id = id;
    fr->hard = inside;
    fr->dist_px = dist;
    fr->feat = feat;
    fr->segP = segP[mseg]; fr->segQ = segQ[mseg]; fr->segt = segt[mseg];
    if (inside) {
        /* area ratios; the vertex opposite edge i is (i + 2) % 3 */
        fr->lam[2] = Fnum[0] / absA;
        fr->lam[0] = Fnum[1] / absA;
        fr->lam[1] = Fnum[2] / absA;
    } else {
        /* the closest point of the hard face: a corner, or a point of an edge */
        fr->lam[0] = fr->lam[1] = fr->lam[2] = 0.0;
        if (feat >= 3) {
            fr->lam[feat - 3] = 1.0;
        } else {
            fr->lam[fr->segP] = 1.0 - fr->segt;
            fr->lam[fr->segQ] = fr->segt;
        }
    }
    if (inside) {
        double z = fr->lam[0] * t->Z[0] + fr->lam[1] * t->Z[1] + fr->lam[2] * t->Z[2];
        fr->key = 0.5 * z;
    } else {
        fr->key = 0.5 * fabs(dist / S) + 0.5;
    }
    return dist;
}

static uint64_t mix64(uint64_t h, double x)
{
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    h ^= b + 0x9E3779B97F4A7C15ULL + (h << 6) + (h >> 2);
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ULL;
    return h ^ (h >> 29);
}

static uint64_t feature_hash(const face_t *t, const frag_t *fr)
{
    if (fr->hard) return mix64(0x1234567ULL, (double)fr->id);
    if (fr->feat >= 3) {
        int m = fr->feat - 3;
        return mix64(mix64(0x77ULL, t->X[m]), t->Y[m]);
    }
    return mix64(mix64(mix64(mix64(0x99ULL, t->X[fr->segP]), t->Y[fr->segP]), t->X[fr->segQ]), t->Y[fr->segQ]);
}

static int frag_less(const frag_t *a, const frag_t *b)
{
    return a->key < b->key || (a->key == b->key && a->id < b->id);
}

/* per-pixel accumulator of the K+1 smallest fragments (step 7) */
typedef struct {
    int n;
    frag_t f[ORC_MAXK + 1];
    double m_hard, m_cand;
    int n_hard;
} pix_t;

static void pix_init(pix_t *p)
{
    p->n = 0; p->m_hard = INFINITY; p->m_cand = INFINITY; p->n_hard = 0;
}

static void pix_offer(pix_t *p, const frag_t *fr, int cap)
{
    int pos = p->n;
    while (pos > 0 && frag_less(fr, &p->f[pos - 1])) --pos;
    if (pos >= cap) return;
    int last = p->n < cap ? p->n : cap - 1;
    for (int j = last; j > pos; --j) p->f[j] = p->f[j - 1];
    p->f[pos] = *fr;
    if (p->n < cap) p->n++;
}

/* ------------------------------------------------------------------------- */
/* rasterization of a pixel rectangle (Alg. 2 restated per pixel)             */
/* ------------------------------------------------------------------------- */
typedef struct { int x0, y0, w, h; } rect_t;

static void raster_rect(const orc_view *v, const orc_params *prm, const face_t *F, rect_t R,
                        double S, double r_px, pix_t *pix)
{
    const double tau = 1e-3; /* faces this close to a decision are tracked for margins */
    int cap = prm->K + 1;
    for (int i = 0; i < R.w * R.h; ++i) pix_init(&pix[i]);
    if (prm->brute_force) {
        for (int yy = 0; yy < R.h; ++yy)
            for (int xx = 0; xx < R.w; ++xx) {
                double px = R.x0 + xx + 0.5, py = R.y0 + yy + 0.5;
                pix_t *P = &pix[yy * R.w + xx];
                for (int f = 0; f < v->n_faces; ++f) {
                    if (!F[f].live) continue;
                    frag_t fr;
                    double d = eval_face(&F[f], f, px, py, S, &fr);
                    if (fr.hard) P->n_hard++;
                    if (d >= -r_px - tau) {
                        if (fabs(d) < P->m_hard) P->m_hard = fabs(d);
                        if (fabs(d + r_px) < P->m_cand) P->m_cand = fabs(d + r_px);
                    }
                    if (d >= -r_px) pix_offer(P, &fr, cap);
                }
            }
    } else {
        for (int f = 0; f < v->n_faces; ++f) {
            const face_t *t = &F[f];
            if (!t->live) continue;
            /* a pixel centre outside the r-grown bbox is farther than r from the face
               (the +-1 guards the pixel-centre offset against rounding) */
            int xa = (int)floor(t->bx0 - 1.0) - R.x0, xb = (int)ceil(t->bx1 + 1.0) - R.x0;
            int ya = (int)floor(t->by0 - 1.0) - R.y0, yb = (int)ceil(t->by1 + 1.0) - R.y0;
            if (xa < 0) xa = 0;
            if (ya < 0) ya = 0;
            if (xb > R.w - 1) xb = R.w - 1;
            if (yb > R.h - 1) yb = R.h - 1;
            for (int yy = ya; yy <= yb; ++yy)
                for (int xx = xa; xx <= xb; ++xx) {
                    double px = R.x0 + xx + 0.5, py = R.y0 + yy + 0.5;
                    pix_t *P = &pix[yy * R.w + xx];
                    frag_t fr;
                    double d = eval_face(t, f, px, py, S, &fr);
                    if (fr.hard) P->n_hard++;
                    if (d >= -r_px - tau) {
                        if (fabs(d) < P->m_hard) P->m_hard = fabs(d);
                        if (fabs(d + r_px) < P->m_cand) P->m_cand = fabs(d + r_px);
                    }
                    if (d >= -r_px) pix_offer(P, &fr, cap);
                }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* steps 8-11: barycentrics, normals, texture, shading                        */
/* ------------------------------------------------------------------------- */
static void vertex_normals(const orc_view *v, double *N /*[nV][3]*/, double *M /*[nV][3] unnormalised*/)
{
    memset(M, 0, sizeof(double) * 3 * (size_t)v->n_verts);
    for (int f = 0; f < v->n_faces; ++f) {
        const int32_t *fv = v->faces + 3 * f;
        if (fv[0] < 0 || fv[0] >= v->n_verts || fv[1] < 0 || fv[1] >= v->n_verts ||
            fv[2] < 0 || fv[2] >= v->n_verts) continue;
        const double *p0 = v->pos + 3 * fv[0], *p1 = v->pos + 3 * fv[1], *p2 = v->pos + 3 * fv[2];
        double u[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
        double w[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
        double a[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        for (int j = 0; j < 3; ++j)
            for (int c = 0; c < 3; ++c) M[3 * fv[j] + c] += a[c];
    }
    for (int i = 0; i < v->n_verts; ++i) {
        double *m = M + 3 * i;
        double l = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
        for (int c = 0; c < 3; ++c) N[3 * i + c] = l > 0 ? m[c] / l : 0.0;
    }
}

typedef struct {
    int ix[2], iy[2];
    double fx, fy;
} bil_t;

static int wrap(long long i, int n) { long long m = i % n; return (int)(m < 0 ? m + n : m); }

static bil_t bilinear_coords(const orc_view *v, double u, double vv)
{
    bil_t b;
    double x = u * v->tex_w - 0.5, y = vv * v->tex_h - 0.5;
    double x0 = floor(x), y0 = floor(y);
    b.fx = x - x0; b.fy = y - y0;
    b.ix[0] = wrap((long long)x0, v->tex_w); b.ix[1] = wrap((long long)x0 + 1, v->tex_w);
    b.iy[0] = wrap((long long)y0, v->tex_h); b.iy[1] = wrap((long long)y0 + 1, v->tex_h);
    return b;
}

static const double *texel_of(const orc_view *v, const double *tex, int ix, int iy)
{
    return tex + 4 * ((size_t)iy * v->tex_w + ix);
}

static const double *texel(const orc_view *v, int ix, int iy) { return texel_of(v, v->tex, ix, iy); }

/* bilinear sample of `tex` (the albedo or the normal map: same size and addressing) */
static void bilinear_sample_of(const orc_view *v, const double *tex, const bil_t *b, double out[3])
{
    const double *t00 = texel_of(v, tex, b->ix[0], b->iy[0]), *t10 = texel_of(v, tex, b->ix[1], b->iy[0]);
    const double *t01 = texel_of(v, tex, b->ix[0], b->iy[1]), *t11 = texel_of(v, tex, b->ix[1], b->iy[1]);
    for (int c = 0; c < 3; ++c)
        out[c] = (1 - b->fx) * (1 - b->fy) * t00[c] + b->fx * (1 - b->fy) * t10[c] +
                 (1 - b->fx) * b->fy * t01[c] + b->fx * b->fy * t11[c];
}

static void bilinear_sample(const orc_view *v, const bil_t *b, double out[3]) { bilinear_sample_of(v, v->tex, b, out); }

typedef struct {
    double b[3];      /* perspective-correct barycentrics */
    double q[3], Q;   /* q_i = lam_i / w_i, Q = sum q */
    double uv[2];
    bil_t bil;
    double albedo[3];
    double m[3], mlen, n[3], ndl; /* interpolated normal and Lambert term */
    /* normal map (shade_mode 3): face tangent Tf and handedness h (sign of the UV
       determinant) from the object-space edges and UV differences; T' = normalize(Tf - n (n.Tf)),
       B' = h n x T'; map value t, nt = 2 t - 1; m' = nt0 T' + nt1 B' + nt2 n, n' = m' / |m'| */
    double Tf[3], h, e1[3], e2[3], duv[2][2], idet;
    double tau[3], tl, Tp[3], Bp[3], nt[3], mp[3], mpl, np[3];
    double C[3];      /* shaded colour */
} shade_t;

static void shade(const orc_view *v, const orc_params *prm, const face_t *t, const frag_t *fr,
                  const double *N, shade_t *s)
{
    memset(s, 0, sizeof(*s));
    s->Q = 0;
    for (int i = 0; i < 3; ++i) { s->q[i] = fr->lam[i] * t->IW[i]; s->Q += s->q[i]; }
    for (int i = 0; i < 3; ++i) s->b[i] = s->q[i] / s->Q;
    if (prm->shade_mode == 0) {
        for (int c = 0; c < 3; ++c) {
            double a = 0;
            for (int i = 0; i < 3; ++i) a += s->b[i] * (v->col ? v->col[3 * t->vi[i] + c] : 1.0);
            s->C[c] = a;
        }
        return;
    }
    for (int k = 0; k < 2; ++k) {
        double a = 0;
        for (int i = 0; i < 3; ++i) a += s->b[i] * v->uv[2 * t->vi[i] + k];
        s->uv[k] = a;
    }
    s->bil = bilinear_coords(v, s->uv[0], s->uv[1]);
    bilinear_sample(v, &s->bil, s->albedo);
    if (prm->shade_mode == 1) {
        for (int c = 0; c < 3; ++c) s->C[c] = s->albedo[c];
        return;
    }
    for (int c = 0; c < 3; ++c) {
        double a = 0;
        for (int i = 0; i < 3; ++i) a += s->b[i] * N[3 * t->vi[i] + c];
        s->m[c] = a;
    }
    s->mlen = sqrt(s->m[0] * s->m[0] + s->m[1] * s->m[1] + s->m[2] * s->m[2]);
    for (int c = 0; c < 3; ++c) s->n[c] = s->mlen > 0 ? s->m[c] / s->mlen : 0.0;
    const double *sn = s->n;
    if (prm->shade_mode == 3) {
        const double *P0 = v->pos + 3 * t->vi[0], *P1 = v->pos + 3 * t->vi[1], *P2 = v->pos + 3 * t->vi[2];
        const double *U0 = v->uv + 2 * t->vi[0], *U1 = v->uv + 2 * t->vi[1], *U2 = v->uv + 2 * t->vi[2];
        for (int c = 0; c < 3; ++c) { s->e1[c] = P1[c] - P0[c]; s->e2[c] = P2[c] - P0[c]; }
        for (int k = 0; k < 2; ++k) { s->duv[0][k] = U1[k] - U0[k]; s->duv[1][k] = U2[k] - U0[k]; }
        double det = s->duv[0][0] * s->duv[1][1] - s->duv[1][0] * s->duv[0][1];
        s->idet = det != 0 ? 1.0 / det : 0.0;
        s->h = det < 0 ? -1.0 : 1.0;
        for (int c = 0; c < 3; ++c) {
            s->Tf[c] = (s->e1[c] * s->duv[1][1] - s->e2[c] * s->duv[0][1]) * s->idet;
        }
        double nT = sn[0] * s->Tf[0] + sn[1] * s->Tf[1] + sn[2] * s->Tf[2];
        for (int c = 0; c < 3; ++c) s->tau[c] = s->Tf[c] - sn[c] * nT;
        s->tl = sqrt(s->tau[0] * s->tau[0] + s->tau[1] * s->tau[1] + s->tau[2] * s->tau[2]);
        for (int c = 0; c < 3; ++c) s->Tp[c] = s->tl > 0 ? s->tau[c] / s->tl : 0.0;
        s->Bp[0] = s->h * (sn[1] * s->Tp[2] - sn[2] * s->Tp[1]);
        s->Bp[1] = s->h * (sn[2] * s->Tp[0] - sn[0] * s->Tp[2]);
        s->Bp[2] = s->h * (sn[0] * s->Tp[1] - sn[1] * s->Tp[0]);
        double tv[3];
        bilinear_sample_of(v, v->ntex, &s->bil, tv);
        for (int c = 0; c < 3; ++c) s->nt[c] = 2.0 * tv[c] - 1.0;
        for (int c = 0; c < 3; ++c) s->mp[c] = s->nt[0] * s->Tp[c] + s->nt[1] * s->Bp[c] + s->nt[2] * sn[c];
        s->mpl = sqrt(s->mp[0] * s->mp[0] + s->mp[1] * s->mp[1] + s->mp[2] * s->mp[2]);
        for (int c = 0; c < 3; ++c) s->np[c] = s->mpl > 0 ? s->mp[c] / s->mpl : 0.0;
        sn = s->np;
    }
    s->ndl = sn[0] * v->light[0] + sn[1] * v->light[1] + sn[2] * v->light[2];
    double lam = s->ndl > 0 ? s->ndl : 0.0;
    for (int c = 0; c < 3; ++c) s->C[c] = s->albedo[c] * lam;
}

/* ------------------------------------------------------------------------- */
/* step 12: soft probability                                                  */
/* ------------------------------------------------------------------------- */
static double sigmoid(double x)
{
    if (x >= 0) return 1.0 / (1.0 + exp(-x));
    double e = exp(x);
    return e / (1.0 + e);
}

/* ------------------------------------------------------------------------- */
/* common driver                                                              */
/* ------------------------------------------------------------------------- */
typedef struct {
    double S, r_px, sigma_px;
    int rho;
    rect_t win, ext;   /* requested window; window grown by rho (clipped) */
    face_t *F;
    pix_t *pix;        /* over ext */
    uint8_t *sh;       /* over ext */
    double *N, *Mn;    /* vertex normals */
    int status;
} ctx_t;

static int check_args(const orc_view *v, const orc_params *prm, const orc_window *w)
{
    if (!v || !prm || !w) return 0;
    if (prm->K < 1 || prm->K > ORC_MAXK) return 0;
    if (v->width <= 0 || v->height <= 0 || v->n_verts < 0 || v->n_faces < 0) return 0;
    if (!(prm->sigma > 0) || !(prm->r >= 0)) return 0;
    if (w->x0 < 0 || w->y0 < 0 || w->w < 0 || w->h < 0 ||
        w->x0 + w->w > v->width || w->y0 + w->h > v->height) return 0;
    if (prm->shade_mode == 0 && !v->col) return 0;
    if (prm->shade_mode > 0 && (!v->uv || !v->tex || v->tex_w <= 0 || v->tex_h <= 0)) return 0;
    if (prm->shade_mode == 3 && !v->ntex) return 0;
    if (prm->shade_mode < 0 || prm->shade_mode > 3) return 0;
    return 1;
}

static void ctx_build(ctx_t *c, const orc_view *v, const orc_params *prm, const orc_window *w)
{
    c->S = (double)(v->width > v->height ? v->width : v->height);
    c->r_px = prm->r * c->S;
    c->sigma_px = prm->sigma * c->S;
    c->rho = (int)round(prm->delta * c->S);
    if (c->rho < 1) c->rho = 1;
    c->win.x0 = w->x0; c->win.y0 = w->y0; c->win.w = w->w; c->win.h = w->h;
    int g = prm->edge_mode == 0 ? c->rho : 0;
    int x0 = w->x0 - g, y0 = w->y0 - g, x1 = w->x0 + w->w + g, y1 = w->y0 + w->h + g;
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > v->width) x1 = v->width;
    if (y1 > v->height) y1 = v->height;
    c->ext.x0 = x0; c->ext.y0 = y0; c->ext.w = x1 - x0; c->ext.h = y1 - y0;
    c->F = (face_t *)calloc((size_t)(v->n_faces > 0 ? v->n_faces : 1), sizeof(face_t));
    c->status = setup_faces(v, c->r_px, c->F);
    size_t ne = (size_t)c->ext.w * c->ext.h;
    c->pix = (pix_t *)malloc(sizeof(pix_t) * (ne > 0 ? ne : 1));
    c->sh = (uint8_t *)calloc(ne > 0 ? ne : 1, 1);
    raster_rect(v, prm, c->F, c->ext, c->S, c->r_px, c->pix);
    for (size_t i = 0; i < ne; ++i) c->sh[i] = (uint8_t)(c->pix[i].n > 0 && c->pix[i].f[0].hard);
    c->N = (double *)malloc(sizeof(double) * 3 * (size_t)(v->n_verts > 0 ? v->n_verts : 1));
    c->Mn = (double *)malloc(sizeof(double) * 3 * (size_t)(v->n_verts > 0 ? v->n_verts : 1));
    if (prm->shade_mode >= 2) vertex_normals(v, c->N, c->Mn);
}

static void ctx_free(ctx_t *c)
{
    free(c->F); free(c->pix); free(c->sh); free(c->N); free(c->Mn);
}

/* step 13: edge mask from the hard stencil S^H by a Chebyshev window */
static int edge_mask_at(const ctx_t *c, const orc_params *prm, int X, int Y)
{
    if (prm->edge_mode == 1) return 1;
    if (prm->edge_mode == 2) return 0;
    int seen0 = 0, seen1 = 0;
    for (int yy = Y - c->rho; yy <= Y + c->rho; ++yy)
        for (int xx = X - c->rho; xx <= X + c->rho; ++xx) {
            int lx = xx - c->ext.x0, ly = yy - c->ext.y0;
            if (lx < 0 || ly < 0 || lx >= c->ext.w || ly >= c->ext.h) continue; /* clipped to the image */
            if (c->sh[ly * c->ext.w + lx]) seen1 = 1; else seen0 = 1;
        }
    return seen0 && seen1;
}

static const pix_t *pix_at(const ctx_t *c, int X, int Y)
{
    return &c->pix[(Y - c->ext.y0) * c->ext.w + (X - c->ext.x0)];
}

/* ------------------------------------------------------------------------- */
/* forward                                                                    */
/* ------------------------------------------------------------------------- */
int orc_forward(const orc_view *v, const orc_params *prm, const orc_window *w, orc_fwd_out *out)
{
    if (!check_args(v, prm, w)) return ORC_BAD_ARG;
    ctx_t c;
    ctx_build(&c, v, prm, w);
    int K = prm->K;
    size_t plane = (size_t)w->w * w->h;
    for (int yy = 0; yy < w->h; ++yy)
        for (int xx = 0; xx < w->w; ++xx) {
            int X = w->x0 + xx, Y = w->y0 + yy;
            size_t o = (size_t)yy * w->w + xx;
            const pix_t *P = pix_at(&c, X, Y);
            int nl = P->n < K ? P->n : K;
            int SH = nl > 0 && P->f[0].hard;
            int E = edge_mask_at(&c, prm, X, Y);
            double Csum[3] = {0, 0, 0}, Dsum = 0, prod = 1, C1[3] = {0, 0, 0};
            for (int k = 0; k < nl; ++k) {
                const frag_t *fr = &P->f[k];
                shade_t s;
                shade(v, prm, &c.F[fr->id], fr, c.N, &s);
                double D = sigmoid(fr->dist_px / c.sigma_px);
                for (int ch = 0; ch < 3; ++ch) Csum[ch] += D * s.C[ch];
                Dsum += D;
                prod *= 1.0 - D;
                if (k == 0) for (int ch = 0; ch < 3; ++ch) C1[ch] = s.C[ch];
            }
            double rgba[4];
            for (int ch = 0; ch < 3; ++ch) {
                double Ie = Dsum > 0 ? Csum[ch] / Dsum : 0.0;
                double Ine = SH ? C1[ch] : 0.0;
                rgba[ch] = E ? Ie : Ine;
            }
            rgba[3] = E ? 1.0 - prod : (double)SH;
            if (out->rgba) for (int ch = 0; ch < 4; ++ch) out->rgba[4 * o + ch] = rgba[ch];
            for (int k = 0; k < K; ++k) {
                if (out->ids) out->ids[k * plane + o] = k < nl ? P->f[k].id : -1;
                if (out->hard) out->hard[k * plane + o] = k < nl ? P->f[k].hard : 0;
                if (out->dist) out->dist[k * plane + o] = k < nl ? P->f[k].dist_px / c.S : 0.0;
            }
            if (out->key)
                for (int k = 0; k <= K; ++k) out->key[k * plane + o] = k < P->n ? P->f[k].key : INFINITY;
            if (out->feat_hash)
                for (int k = 0; k <= K; ++k)
                    out->feat_hash[k * plane + o] = k < P->n ? feature_hash(&c.F[P->f[k].id], &P->f[k]) : 0;
            if (out->sh) out->sh[o] = (uint8_t)SH;
            if (out->edge) out->edge[o] = (uint8_t)E;
            if (out->margin_hard) out->margin_hard[o] = P->m_hard;
            if (out->margin_cand) out->margin_cand[o] = P->m_cand;
            if (out->n_hard) out->n_hard[o] = P->n_hard;
        }
    int st = c.status;
    ctx_free(&c);
    return st;
}

/* ------------------------------------------------------------------------- */
/* adjoint                                                                    */
/* ------------------------------------------------------------------------- */
typedef struct { double X[3], Y[3], IW[3]; } corner_grad_t;

/* d dist_px / d corners for the closest feature of fr */
static void dist_grad(const face_t *t, const frag_t *fr, double px, double py, double g, corner_grad_t *cg)
{
    if (fr->feat < 3) {
        int a = fr->feat, b = (fr->feat + 1) % 3;
        double ex = t->X[b] - t->X[a], ey = t->Y[b] - t->Y[a];
        double dx = px - t->X[a], dy = py - t->Y[a];
        double L = sqrt(ex * ex + ey * ey);
        double c = ex * dy - ey * dx;
        /* F = orient * c / L */
        double gex = t->orient * (dy / L - c * ex / (L * L * L));
        double gey = t->orient * (-dx / L - c * ey / (L * L * L));
        double gdx = t->orient * (-ey / L), gdy = t->orient * (ex / L);
        cg->X[b] += g * gex; cg->Y[b] += g * gey;
        cg->X[a] += g * (-gex - gdx); cg->Y[a] += g * (-gey - gdy);
    } else {
        int m = fr->feat - 3;
        double dx = px - t->X[m], dy = py - t->Y[m];
        double l = sqrt(dx * dx + dy * dy);
        if (l > 0) {           /* dist = -|p - V_m| */
            cg->X[m] += g * dx / l;
            cg->Y[m] += g * dy / l;
        }
    }
}

/* d lam_i / d corners.  Hard fragment: lam_i = cross(V_{i+2} - V_{i+1}, p - V_{i+1}) / A2.
   Soft fragment on an edge: lam_P = 1 - s, lam_Q = s, s = (p - P).(Q - P) / |Q - P|^2.
   Soft fragment at a corner: constant. */
static void lam_grad(const face_t *t, const frag_t *fr, double px, double py, const double glam[3],
                     corner_grad_t *cg)
{
    if (!fr->hard) {
        if (fr->feat >= 3) return;
        int P = fr->segP, Q = fr->segQ;
        double ex = t->X[Q] - t->X[P], ey = t->Y[Q] - t->Y[P];
        double dx = px - t->X[P], dy = py - t->Y[P];
        double ee = ex * ex + ey * ey, s = fr->segt;
        double gs = glam[Q] - glam[P];
        /* ds/dd = e/ee, ds/de = (d - 2 s e)/ee; d = p - P, e = Q - P */
        double gex = (dx - 2 * s * ex) / ee, gey = (dy - 2 * s * ey) / ee;
        double gdx = ex / ee, gdy = ey / ee;
        cg->X[Q] += gs * gex; cg->Y[Q] += gs * gey;
        cg->X[P] += gs * (-gex - gdx); cg->Y[P] += gs * (-gey - gdy);
        return;
    }
    double gA2 = 0;
    for (int i = 0; i < 3; ++i) {
        int A = (i + 1) % 3, B = (i + 2) % 3;
        double gn = glam[i] / t->A2;
        gA2 -= glam[i] * fr->lam[i] / t->A2;
        double ex = t->X[B] - t->X[A], ey = t->Y[B] - t->Y[A];
        double dx = px - t->X[A], dy = py - t->Y[A];
        /* n = ex*dy - ey*dx */
        double gex = dy, gey = -dx, gdx = -ey, gdy = ex;
        cg->X[B] += gn * gex; cg->Y[B] += gn * gey;
        cg->X[A] += gn * (-gex - gdx); cg->Y[A] += gn * (-gey - gdy);
    }
    /* A2 = (X1-X0)(Y2-Y0) - (X2-X0)(Y1-Y0) */
    double ux = t->X[1] - t->X[0], uy = t->Y[1] - t->Y[0];
    double wx = t->X[2] - t->X[0], wy = t->Y[2] - t->Y[0];
    cg->X[1] += gA2 * wy;  cg->Y[1] += gA2 * (-wx);
    cg->X[2] += gA2 * (-uy); cg->Y[2] += gA2 * ux;
    cg->X[0] += gA2 * (-wy + uy); cg->Y[0] += gA2 * (wx - ux);
}

/* adjoint of the bilinear sample of `tex` at the layer's UV: texel gradients into gtex
   (if not NULL) and the UV gradient */
static void tex_backward_of(const orc_view *v, const double *tex, const shade_t *s, const double gA[3], double *gtex,
                            double guv[2])
{
    const bil_t *b = &s->bil;
    double w00 = (1 - b->fx) * (1 - b->fy), w10 = b->fx * (1 - b->fy), w01 = (1 - b->fx) * b->fy, w11 = b->fx * b->fy;
    const double *t00 = texel_of(v, tex, b->ix[0], b->iy[0]), *t10 = texel_of(v, tex, b->ix[1], b->iy[0]);
    const double *t01 = texel_of(v, tex, b->ix[0], b->iy[1]), *t11 = texel_of(v, tex, b->ix[1], b->iy[1]);
    double gx = 0, gy = 0;
    for (int c = 0; c < 3; ++c) {
        if (gtex) {
            gtex[4 * ((size_t)b->iy[0] * v->tex_w + b->ix[0]) + c] += w00 * gA[c];
            gtex[4 * ((size_t)b->iy[0] * v->tex_w + b->ix[1]) + c] += w10 * gA[c];
            gtex[4 * ((size_t)b->iy[1] * v->tex_w + b->ix[0]) + c] += w01 * gA[c];
            gtex[4 * ((size_t)b->iy[1] * v->tex_w + b->ix[1]) + c] += w11 * gA[c];
        }
        gx += gA[c] * ((1 - b->fy) * (t10[c] - t00[c]) + b->fy * (t11[c] - t01[c]));
        gy += gA[c] * ((1 - b->fx) * (t01[c] - t00[c]) + b->fx * (t11[c] - t10[c]));
    }
    guv[0] = gx * v->tex_w;
    guv[1] = gy * v->tex_h;
}

static void tex_backward(const orc_view *v, const shade_t *s, const double gA[3], double *gtex, double guv[2])
{
    tex_backward_of(v, v->tex, s, gA, gtex, guv);
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* adjoint of the normal-mapped shading normal (shade_mode 3) for dL/dn' = gs l: the
   normal-map texel gradients (grad_ntex), the UV gradient of the map sample (guv), the
   object-space corner gradients through the face tangent (grad_pos), and dL/dn of the
   smooth interpolated normal (gn, for the vertex-normal chain) */
static void normal_map_backward(const orc_view *v, const face_t *t, const shade_t *s, double gs, double gn[3],
                                double *grad_ntex, double guv[2], double *grad_pos)
{
    double gnp[3], gmp[3], gTp[3], gBp[3], tmp[3], gtau[3], gTf[3];
    for (int c = 0; c < 3; ++c) gnp[c] = gs * v->light[c];
    double d = dot3(s->np, gnp);
    for (int c = 0; c < 3; ++c) gmp[c] = (gnp[c] - s->np[c] * d) / s->mpl;     /* n' = m' / |m'| */
    /* m' = nt0 T' + nt1 B' + nt2 n, nt = 2 t - 1 */
    double gt[3] = {2.0 * dot3(gmp, s->Tp), 2.0 * dot3(gmp, s->Bp), 2.0 * dot3(gmp, s->n)};
    tex_backward_of(v, v->ntex, s, gt, grad_ntex, guv);
    for (int c = 0; c < 3; ++c) { gTp[c] = s->nt[0] * gmp[c]; gBp[c] = s->nt[1] * gmp[c]; gn[c] = s->nt[2] * gmp[c]; }
    /* B' = h n x T' */
    cross3(s->Tp, gBp, tmp);
    for (int c = 0; c < 3; ++c) gn[c] += s->h * tmp[c];
    cross3(gBp, s->n, tmp);
    for (int c = 0; c < 3; ++c) gTp[c] += s->h * tmp[c];
    /* T' = tau / |tau| */
    double dT = dot3(s->Tp, gTp);
    for (int c = 0; c < 3; ++c) gtau[c] = s->tl > 0 ? (gTp[c] - s->Tp[c] * dT) / s->tl : 0.0;
    /* tau = Tf - n (n . Tf) */
    double nT = dot3(s->n, s->Tf), ng = dot3(s->n, gtau);
    for (int c = 0; c < 3; ++c) {
        gTf[c] = gtau[c] - s->n[c] * ng;
        gn[c] += -nT * gtau[c] - s->Tf[c] * ng;
    }
    /* Tf = (e1 dv2 - e2 dv1) / det, e1 = P1 - P0, e2 = P2 - P0 (the UVs are constants) */
    if (grad_pos)
        for (int c = 0; c < 3; ++c) {
            double ge1 = gTf[c] * s->duv[1][1] * s->idet, ge2 = -gTf[c] * s->duv[0][1] * s->idet;
            grad_pos[3 * (size_t)t->vi[1] + c] += ge1;
            grad_pos[3 * (size_t)t->vi[2] + c] += ge2;
            grad_pos[3 * (size_t)t->vi[0] + c] -= ge1 + ge2;
        }
}

/* Inverse UV (Sec. 3.3.2, Alg. 1): the texture-gradient lookup of the paper's Vulkan
   path.  Every shaded sample (a pixel's layer that the forward shades) has a screen
   position, the pixel centre plus a jitter given by the caller (the paper adds a Sobol
   point per frame), and writes its sample number into the texel that holds the layer's
   UV at that position; the last writer of a texel wins, and the texel's gradient is
   the winner's dL/d(albedo).  The oracle lists every write as a record (in sample
   order) with the margins of its discrete decisions; oracle/__init__.py resolves the
   winners (largest sample number) and the texel gradients from them. */
typedef struct {
    double jitter[2];      /* sample offset from the pixel centre, in pixels */
    int64_t pix_base;      /* the view's first pixel in the packed numbering of all views */
    int64_t cap, n;        /* record capacity; records written */
    int64_t *slot;         /* [cap] sample number (pix_base + Y W + X) K + k */
    int32_t *texel;        /* [cap] texel ty * tex_w + tx written */
    double *m_tex;         /* [cap] distance of the sample's u W, v H to the nearest texel edge */
    double *m_cand;        /* [cap] |dist + r| in pixels of the jittered evaluation */
    double *gA;            /* [cap][3] the sample's dL/d(albedo) at its pixel centre */
} orc_inv_uv;

static void inv_uv_write(const orc_view *v, const orc_params *prm, const ctx_t *c, const face_t *t, int id,
                         int X, int Y, int k, const double gA[3], orc_inv_uv *inv)
{
    double qx = X + 0.5 + inv->jitter[0], qy = Y + 0.5 + inv->jitter[1];
    frag_t fj;
    double d = eval_face(t, id, qx, qy, c->S, &fj);
    if (!(d >= -c->r_px)) return;          /* not a candidate at the jittered position */
    shade_t sj;
    shade(v, prm, t, &fj, c->N, &sj);
    double x = sj.uv[0] * v->tex_w, y = sj.uv[1] * v->tex_h;
    double fx = floor(x), fy = floor(y);
    if (inv->n >= inv->cap) return;
    int64_t r = inv->n++;
    inv->slot[r] = (inv->pix_base + (int64_t)Y * v->width + X) * prm->K + k;
    inv->texel[r] = wrap((long long)fy, v->tex_h) * v->tex_w + wrap((long long)fx, v->tex_w);
    double mx = fmin(x - fx, fx + 1.0 - x), my = fmin(y - fy, fy + 1.0 - y);
    inv->m_tex[r] = fmin(mx, my);
    inv->m_cand[r] = fabs(d + c->r_px);
    for (int ch = 0; ch < 3; ++ch) inv->gA[3 * r + ch] = gA[ch];
}

/* The adjoint also gives the gradients of the camera and the light, the parameters
   theta_C and theta_L of Theta (Sec. 3.4.1): grad_mvp [16] (row-major, as mvp; the
   depth row stays 0, depth only enters the discrete Shift keys) and grad_light [3]
   (the light treated as a free 3-vector, as the forward uses it).  Either may be NULL. */
int orc_backward_ex(const orc_view *v, const orc_params *prm, const orc_window *w,
                    const double *grad_rgba, double *grad_pos, double *grad_col, double *grad_tex,
                    double *grad_mvp, double *grad_light, orc_inv_uv *inv, double *grad_ntex)
{
    if (!check_args(v, prm, w) || !grad_rgba) return ORC_BAD_ARG;
    ctx_t c;
    ctx_build(&c, v, prm, w);
    int K = prm->K;
    /* per (face corner) screen gradients, accumulated over pixels */
    corner_grad_t *CG = (corner_grad_t *)calloc((size_t)(v->n_faces > 0 ? v->n_faces : 1), sizeof(corner_grad_t));
    double *gN = (double *)calloc(3 * (size_t)(v->n_verts > 0 ? v->n_verts : 1), sizeof(double));
    for (int yy = 0; yy < w->h; ++yy)
        for (int xx = 0; xx < w->w; ++xx) {
            int X = w->x0 + xx, Y = w->y0 + yy;
            double px = X + 0.5, py = Y + 0.5;
            const double *g = grad_rgba + 4 * ((size_t)yy * w->w + xx);
            const pix_t *P = pix_at(&c, X, Y);
            int nl = P->n < K ? P->n : K;
            if (nl == 0) continue;
            int SH = P->f[0].hard;
            int E = edge_mask_at(&c, prm, X, Y);
            shade_t s[ORC_MAXK];
            double D[ORC_MAXK], gC[ORC_MAXK][3], gD[ORC_MAXK];
            for (int k = 0; k < nl; ++k) {
                shade(v, prm, &c.F[P->f[k].id], &P->f[k], c.N, &s[k]);
                D[k] = sigmoid(P->f[k].dist_px / c.sigma_px);
                gD[k] = 0; gC[k][0] = gC[k][1] = gC[k][2] = 0;
            }
            if (E) {
                double Dsum = 0, Ie[3] = {0, 0, 0};
                for (int k = 0; k < nl; ++k) { Dsum += D[k]; for (int ch = 0; ch < 3; ++ch) Ie[ch] += D[k] * s[k].C[ch]; }
                if (Dsum > 0) {
                    for (int ch = 0; ch < 3; ++ch) Ie[ch] /= Dsum;
                    for (int k = 0; k < nl; ++k) {
                        double acc = 0;
                        for (int ch = 0; ch < 3; ++ch) {
                            gC[k][ch] += D[k] / Dsum * g[ch];
                            acc += g[ch] * (s[k].C[ch] - Ie[ch]);
                        }
                        gD[k] += acc / Dsum;
                    }
                }
                for (int k = 0; k < nl; ++k) {
                    double others = 1;
                    for (int j = 0; j < nl; ++j) if (j != k) others *= 1.0 - D[j];
                    gD[k] += g[3] * others;
                }
            } else if (SH) {
                for (int ch = 0; ch < 3; ++ch) gC[0][ch] += g[ch];
            }
            for (int k = 0; k < nl; ++k) {
                const frag_t *fr = &P->f[k];
                const face_t *t = &c.F[fr->id];
                corner_grad_t *cg = &CG[fr->id];
                /* sigmoid -> dist -> corners */
                double gdist = gD[k] * D[k] * (1.0 - D[k]) / c.sigma_px;
                if (gdist != 0) dist_grad(t, fr, px, py, gdist, cg);
                /* shading -> barycentrics and attributes */
                const shade_t *sk = &s[k];
                double gb[3] = {0, 0, 0};
                if (prm->shade_mode == 0) {
                    for (int i = 0; i < 3; ++i)
                        for (int ch = 0; ch < 3; ++ch) {
                            if (grad_col) grad_col[3 * t->vi[i] + ch] += sk->b[i] * gC[k][ch];
                            gb[i] += gC[k][ch] * v->col[3 * t->vi[i] + ch];
                        }
                } else {
                    double gA[3], guv_n[2] = {0, 0};
                    if (prm->shade_mode == 1) {
                        for (int ch = 0; ch < 3; ++ch) gA[ch] = gC[k][ch];
                    } else {
                        double lam = sk->ndl > 0 ? sk->ndl : 0.0;
                        double gs = 0;
                        for (int ch = 0; ch < 3; ++ch) { gA[ch] = gC[k][ch] * lam; gs += gC[k][ch] * sk->albedo[ch]; }
                        const int nmap = prm->shade_mode == 3;
                        if (sk->ndl > 0 && sk->mlen > 0 && (!nmap || sk->mpl > 0)) {
                            /* C = albedo max(0, n.l): dL/dl = (sum_c gC_c albedo_c) n (n' with a map) */
                            if (grad_light)
                                for (int ch = 0; ch < 3; ++ch) grad_light[ch] += gs * (nmap ? sk->np[ch] : sk->n[ch]);
                            double gn[3] = {gs * v->light[0], gs * v->light[1], gs * v->light[2]};
                            if (nmap) normal_map_backward(v, t, sk, gs, gn, grad_ntex, guv_n, grad_pos);
                            double nd = sk->n[0] * gn[0] + sk->n[1] * gn[1] + sk->n[2] * gn[2];
                            double gm[3];
                            for (int ch = 0; ch < 3; ++ch) gm[ch] = (gn[ch] - sk->n[ch] * nd) / sk->mlen;
                            for (int i = 0; i < 3; ++i)
                                for (int ch = 0; ch < 3; ++ch) {
                                    gN[3 * t->vi[i] + ch] += sk->b[i] * gm[ch];
                                    gb[i] += gm[ch] * c.N[3 * t->vi[i] + ch];
                                }
                        }
                    }
                    double guv[2];
                    tex_backward(v, sk, gA, grad_tex, guv);
                    if (inv && (E || k == 0)) inv_uv_write(v, prm, &c, t, fr->id, X, Y, k, gA, inv);
                    for (int i = 0; i < 3; ++i)
                        gb[i] += (guv[0] + guv_n[0]) * v->uv[2 * t->vi[i]] + (guv[1] + guv_n[1]) * v->uv[2 * t->vi[i] + 1];
                }
                /* perspective-correct barycentrics -> screen barycentrics and 1/w */
                double bdot = sk->b[0] * gb[0] + sk->b[1] * gb[1] + sk->b[2] * gb[2];
                double glam[3];
                for (int i = 0; i < 3; ++i) {
                    double gq = (gb[i] - bdot) / sk->Q;
                    glam[i] = gq * t->IW[i];
                    cg->IW[i] += gq * fr->lam[i];
                }
                lam_grad(t, fr, px, py, glam, cg);
            }
        }
    /* corners -> clip -> object-space positions and the matrix */
    if (grad_pos || grad_mvp) {
        for (int f = 0; f < v->n_faces; ++f) {
            const face_t *t = &c.F[f];
            if (!t->live) continue;
            for (int j = 0; j < 3; ++j) {
                int vi = t->vi[j];
                const double *p = v->pos + 3 * (size_t)vi;
                double cl[4];
                for (int r = 0; r < 4; ++r) {
                    const double *m = v->mvp + 4 * r;
                    cl[r] = m[0] * p[0] + m[1] * p[1] + m[2] * p[2] + m[3];
                }
                double cw = cl[3];
                double gcx = CG[f].X[j] * 0.5 * v->width / cw;
                double gcy = CG[f].Y[j] * 0.5 * v->height / cw;
                double gcw = -CG[f].X[j] * 0.5 * v->width * cl[0] / (cw * cw)
                             - CG[f].Y[j] * 0.5 * v->height * cl[1] / (cw * cw)
                             - CG[f].IW[j] / (cw * cw);
                if (grad_pos)
                    for (int col = 0; col < 3; ++col)
                        grad_pos[3 * (size_t)vi + col] += v->mvp[0 * 4 + col] * gcx + v->mvp[1 * 4 + col] * gcy +
                                                          v->mvp[3 * 4 + col] * gcw;
                if (grad_mvp) {
                    /* clip_r = sum_c mvp[r][c] (p, 1)_c */
                    const double ph[4] = {p[0], p[1], p[2], 1.0};
                    for (int col = 0; col < 4; ++col) {
                        grad_mvp[0 * 4 + col] += gcx * ph[col];
                        grad_mvp[1 * 4 + col] += gcy * ph[col];
                        grad_mvp[3 * 4 + col] += gcw * ph[col];
                    }
                }
            }
        }
        /* normals -> positions: n_v = m_v / |m_v|, m_v = sum of face cross products */
        if (grad_pos && prm->shade_mode >= 2) {
            double *gM = (double *)calloc(3 * (size_t)(v->n_verts > 0 ? v->n_verts : 1), sizeof(double));
            for (int i = 0; i < v->n_verts; ++i) {
                const double *m = c.Mn + 3 * i, *n = c.N + 3 * i, *gn = gN + 3 * i;
                double l = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
                if (!(l > 0)) continue;
                double nd = n[0] * gn[0] + n[1] * gn[1] + n[2] * gn[2];
                for (int ch = 0; ch < 3; ++ch) gM[3 * i + ch] = (gn[ch] - n[ch] * nd) / l;
            }
            for (int f = 0; f < v->n_faces; ++f) {
                const int32_t *fv = v->faces + 3 * f;
                if (fv[0] < 0 || fv[0] >= v->n_verts || fv[1] < 0 || fv[1] >= v->n_verts ||
                    fv[2] < 0 || fv[2] >= v->n_verts) continue;
                const double *p0 = v->pos + 3 * fv[0], *p1 = v->pos + 3 * fv[1], *p2 = v->pos + 3 * fv[2];
                double u[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
                double ww[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
                double ga[3];
                for (int ch = 0; ch < 3; ++ch) ga[ch] = gM[3 * fv[0] + ch] + gM[3 * fv[1] + ch] + gM[3 * fv[2] + ch];
                /* a = u x w:  du = w x ga, dw = ga x u */
                double gu[3] = {ww[1] * ga[2] - ww[2] * ga[1], ww[2] * ga[0] - ww[0] * ga[2], ww[0] * ga[1] - ww[1] * ga[0]};
                double gw[3] = {ga[1] * u[2] - ga[2] * u[1], ga[2] * u[0] - ga[0] * u[2], ga[0] * u[1] - ga[1] * u[0]};
                for (int ch = 0; ch < 3; ++ch) {
                    grad_pos[3 * fv[1] + ch] += gu[ch];
                    grad_pos[3 * fv[2] + ch] += gw[ch];
                    grad_pos[3 * fv[0] + ch] -= gu[ch] + gw[ch];
                }
            }
            free(gM);
        }
    }
    free(CG);
    free(gN);
    int st = c.status;
    ctx_free(&c);
    return st;
}

int orc_backward(const orc_view *v, const orc_params *prm, const orc_window *w,
                 const double *grad_rgba, double *grad_pos, double *grad_col, double *grad_tex)
{
    return orc_backward_ex(v, prm, w, grad_rgba, grad_pos, grad_col, grad_tex, NULL, NULL, NULL, NULL);
}

/* size of the structs, so the Python loader can verify its layout */
int orc_sizeof_view(void) { return (int)sizeof(orc_view); }
int orc_sizeof_params(void) { return (int)sizeof(orc_params); }
int orc_sizeof_fwd_out(void) { return (int)sizeof(orc_fwd_out); }
