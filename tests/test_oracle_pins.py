"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

The paper prints no worked numeric example (no image or gradient value), so the
oracle is pinned by closed forms, textbook routines written differently
(ray casting with Moller-Trumbore, scipy's bilinear map_coordinates), limits,
invariants and central finite differences of its own forward pass.
"""
import math

import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth
from scenes_small import grid_mesh, identity_mvp, pixel_mesh, pixel_scene


def _render(scene, **kw):
    return oracle.render(scene.meshes[0], scene.views[0], scene.params, **kw)


# ----------------------------------------------------------------------------
# fill rule (Sec. 3.4.2 hard faces; top-left rule is the reading for points on edges)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("a", [1, 2, 5, 8, 13])
def test_right_triangle_hard_counts(a):
    """(0,0),(a,0),(0,a) covers a(a-1)/2 pixel centres, its mirror a(a+1)/2; together a^2."""
    W = H = 16
    s1 = pixel_scene(pixel_mesh([(0, 0), (a, 0), (0, a)], [(0, 1, 2)], W, H), W, H, K=1, r=0.0, sigma=1e-3, delta=1e-3)
    s2 = pixel_scene(pixel_mesh([(a, a), (0, a), (a, 0)], [(0, 1, 2)], W, H), W, H, K=1, r=0.0, sigma=1e-3, delta=1e-3)
    n1 = _render(s1)["n_hard"].sum()
    n2 = _render(s2)["n_hard"].sum()
    assert n1 == a * (a - 1) // 2
    assert n2 == a * (a + 1) // 2
    both = pixel_scene(pixel_mesh([(0, 0), (a, 0), (0, a), (a, a)], [(0, 1, 2), (3, 2, 1)], W, H), W, H,
                       K=1, r=0.0, sigma=1e-3, delta=1e-3)
    nh = _render(both)["n_hard"]
    assert nh.sum() == a * a and nh.max() == 1


@pytest.mark.parametrize("jitter", [0.0, 0.4])
def test_screen_filling_triangulation_partitions_pixels(jitter):
    """A planar triangulation covering the image: exactly one hard face per pixel.
    With zero jitter many pixel centres sit exactly on shared diagonals."""
    W = H = 24
    V, F = grid_mesh(7, W, H, jitter=jitter, seed=3)
    if jitter == 0.0:
        V = np.round(V)  # integer corners -> centres exactly on the diagonals
    s = pixel_scene(pixel_mesh(V, F, W, H), W, H, K=2, r=0.0, sigma=1e-3, delta=1e-3)
    r = _render(s)
    assert (r["n_hard"] == 1).all()
    assert (r["sh"] == 1).all()


def test_closed_convex_mesh_two_hard_layers():
    """Icosphere (convex, closed): a pixel centre inside the silhouette lies in exactly
    two faces (front and back), outside in none -- no back-face culling."""
    pos, faces = synth.icosphere(2)
    mesh = synth.Mesh(pos.astype(np.float32), faces, col=np.ones_like(pos, dtype=np.float32))
    view = synth.View(synth.camera_mvp((0.3, 0.2, 3.0), 48, 48), 0, 48, 48)
    r = oracle.render(mesh, view, synth.Params(K=3, r=1e-3, sigma=1e-4, delta=1e-3))
    nh = r["n_hard"]
    assert set(np.unique(nh)) == {0, 2}
    inside = nh == 2
    assert (r["hard"][0][inside] == 1).all() and (r["hard"][1][inside] == 1).all()
    # hard faces sort before every soft face (Shift): the third layer is soft
    assert (r["hard"][2][inside] == 0).all()


# ----------------------------------------------------------------------------
# SignedDist + sigmoid (Sec. 3.4.3): K = 1, E = 1 gives alpha = sigmoid(dist / sigma)
# ----------------------------------------------------------------------------

def _boundary_distance(tri, pts, n=200001):
    """Distance from points to the triangle boundary by dense sampling of the edges."""
    best = np.full(len(pts), np.inf)
    t = np.linspace(0, 1, n)
    for i in range(3):
        a, b = np.asarray(tri[i], float), np.asarray(tri[(i + 1) % 3], float)
        seg = a[None] + t[:, None] * (b - a)[None]
        for k, p in enumerate(pts):
            d = np.sqrt(((seg - p) ** 2).sum(1)).min()
            best[k] = min(best[k], d)
    return best


def test_single_triangle_alpha_is_sigmoid_of_distance():
    W = H = 16
    tri = [(3.0, 2.0), (12.0, 5.0), (5.0, 13.0)]
    r_px, sig_px = 3.0, 1.0
    s = pixel_scene(pixel_mesh(tri, [(0, 1, 2)], W, H), W, H, K=1, r=r_px / W, sigma=sig_px / W,
                    delta=r_px / W, edge_mode=1)
    out = _render(s)
    ys, xs = np.mgrid[0:H, 0:W]
    pts = np.stack([xs.ravel() + 0.5, ys.ravel() + 0.5], 1)
    d = _boundary_distance(tri, pts)
    # inside test written as three half-plane inequalities (counter-clockwise order in y-down)
    P = np.asarray(tri)

    def side(a, b, p):
        return (b[0] - a[0]) * (p[:, 1] - a[1]) - (b[1] - a[1]) * (p[:, 0] - a[0])

    s0, s1, s2 = side(P[0], P[1], pts), side(P[1], P[2], pts), side(P[2], P[0], pts)
    inside = ((s0 > 0) & (s1 > 0) & (s2 > 0)) | ((s0 < 0) & (s1 < 0) & (s2 < 0))
    sd = np.where(inside, d, -d)
    cand = sd >= -r_px
    expect = np.where(cand, 1 / (1 + np.exp(-sd / sig_px)), 0.0).reshape(H, W)
    # the sampled boundary is off by at most half a sample spacing (< 2.5e-5 px),
    # i.e. at most 0.25 * 2.5e-5 / sigma_px in alpha
    np.testing.assert_allclose(out["rgba"][..., 3], expect, atol=0.25 * 2.5e-5 / sig_px + 1e-12)
    np.testing.assert_allclose(out["dist"][0][cand.reshape(H, W)] * W, sd[cand], atol=2.5e-5)


def test_soft_fragment_takes_attributes_of_nearest_boundary_point():
    """K = 1, E = 1, w = 1 (so perspective weights are screen-linear): a soft fragment
    has the colour of the closest point of the hard face, found here by dense sampling
    of the boundary."""
    W = H = 20
    tri = [(4.0, 3.0), (15.0, 6.0), (6.0, 16.0)]
    col = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    s = pixel_scene(pixel_mesh(tri, [(0, 1, 2)], W, H, col=col), W, H, K=1, r=3.0 / W, sigma=1.0 / W,
                    delta=3.0 / W, edge_mode=1)
    out = _render(s)
    n = 100001
    t = np.linspace(0, 1, n)
    samples, cols = [], []
    for i in range(3):
        a, b = np.asarray(tri[i]), np.asarray(tri[(i + 1) % 3])
        samples.append(a[None] + t[:, None] * (b - a)[None])
        cols.append((1 - t)[:, None] * col[i][None] + t[:, None] * col[(i + 1) % 3][None])
    samples, cols = np.concatenate(samples), np.concatenate(cols)
    checked = 0
    for y in range(H):
        for x in range(W):
            if out["ids"][0, y, x] < 0 or out["hard"][0, y, x]:
                continue
            p = np.array([x + 0.5, y + 0.5])
            j = np.argmin(((samples - p) ** 2).sum(1))
            # sample spacing <= 1.5e-4 px along an edge; colours change by <= 1 per edge length
            np.testing.assert_allclose(out["rgba"][y, x, :3], cols[j], atol=2e-5)
            checked += 1
    assert checked > 40


def test_sigma_to_zero_recovers_hard_stencil():
    """As sigma -> 0 the silhouette equals S^H, because Shift puts every hard face in layer 1."""
    s = synth.config1()
    p = synth.Params(K=3, r=2 / 64, sigma=1e-12, delta=2 / 64, edge_mode=1)
    r = oracle.render(s.meshes[0], s.views[0], p)
    far = r["margin_hard"] > 1e-6
    assert far.mean() > 0.99
    np.testing.assert_array_equal(r["rgba"][..., 3][far], r["sh"][far].astype(float))


def test_two_layer_order_and_keys():
    """Two overlapping triangles at constant depths z=0.3 (id 1) and z=0.6 (id 0):
    layer 1 is the nearer hard face with key z/2, layer 2 the farther, then soft keys."""
    W = H = 32
    V = [(2, 2), (30, 2), (2, 30), (4, 4), (30, 4), (4, 30)]
    z = [0.6, 0.6, 0.6, 0.3, 0.3, 0.3]
    s = pixel_scene(pixel_mesh(V, [(0, 1, 2), (3, 4, 5)], W, H, z=z), W, H, K=3, r=4 / 32, sigma=1 / 32, delta=4 / 32)
    r = _render(s)
    # pixel (10, 10) is inside both
    assert r["ids"][0, 10, 10] == 1 and r["ids"][1, 10, 10] == 0 and r["ids"][2, 10, 10] == -1
    z03, z06 = float(np.float32(0.3)), float(np.float32(0.6))   # depths enter as float32
    assert r["key"][0, 10, 10] == pytest.approx(0.5 * z03, abs=1e-15)
    assert r["key"][1, 10, 10] == pytest.approx(0.5 * z06, abs=1e-15)
    # pixel (2, 2) (centre 2.5, 2.5) is hard for face 0 only; face 1 is soft at distance sqrt(2)*1.5
    assert r["ids"][0, 2, 2] == 0 and r["hard"][0, 2, 2] == 1
    assert r["ids"][1, 2, 2] == 1 and r["hard"][1, 2, 2] == 0
    assert r["key"][1, 2, 2] == pytest.approx(0.5 + 0.5 * math.hypot(1.5, 1.5) / 32, abs=1e-12)


# ----------------------------------------------------------------------------
# edge mask (Sec. 3.4.3): window of radius rho around p sees both S^H = 0 and 1
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("rho_px", [1, 2, 3])
def test_edge_mask_half_plane(rho_px):
    W = H = 32
    V = [(-100, -100), (16, -100), (16, 200), (-100, 200)]
    s = pixel_scene(pixel_mesh(V, [(0, 1, 2), (0, 2, 3)], W, H), W, H, K=1, r=rho_px / W,
                    sigma=0.5 / W, delta=rho_px / W, edge_mode=0)
    r = _render(s)
    cols = np.arange(W)
    assert (r["sh"] == (cols < 16)[None, :]).all()
    expect = (cols >= 16 - rho_px) & (cols <= 15 + rho_px)
    assert (r["edge"] == expect[None, :]).all()


# ----------------------------------------------------------------------------
# ray casting: E = 0 output equals a textbook z-buffer render
# ----------------------------------------------------------------------------

def _raycast(mesh, view):
    """Nearest ray-triangle hit per pixel centre (Moller-Trumbore in FP64).
    Returns face index (-1 none), barycentrics (b0, b1, b2), NDC depth, min barycentric."""
    W, H = view.width, view.height
    M = np.asarray(view.mvp, np.float64).reshape(4, 4)
    Mi = np.linalg.inv(M)
    P = np.asarray(mesh.pos, np.float64)
    F = np.asarray(mesh.faces)
    v0, v1, v2 = P[F[:, 0]], P[F[:, 1]], P[F[:, 2]]
    e1, e2 = v1 - v0, v2 - v0
    fid = np.full((H, W), -1)
    bary = np.zeros((H, W, 3))
    depth = np.zeros((H, W))
    margin = np.full((H, W), np.inf)
    for y in range(H):
        for x in range(W):
            nx, ny = 2 * (x + 0.5) / W - 1, 2 * (y + 0.5) / H - 1
            a = Mi @ np.array([nx, ny, 0.0, 1.0])
            b = Mi @ np.array([nx, ny, 1.0, 1.0])
            o, d = a[:3] / a[3], b[:3] / b[3] - a[:3] / a[3]
            h = np.cross(d[None], e2)
            det = (e1 * h).sum(1)
            ok = np.abs(det) > 1e-14
            inv = np.where(ok, 1 / np.where(ok, det, 1), 0)
            s = o[None] - v0
            u = (s * h).sum(1) * inv
            q = np.cross(s, e1)
            v = (q * d[None]).sum(1) * inv
            t = (q * e2).sum(1) * inv
            hit = ok & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)
            if not hit.any():
                continue
            j = np.nonzero(hit)[0][np.argmin(t[hit])]
            fid[y, x] = j
            bary[y, x] = (1 - u[j] - v[j], u[j], v[j])
            pt = o + t[j] * d
            c = M @ np.append(pt, 1.0)
            depth[y, x] = c[2] / c[3]
            margin[y, x] = min(u[j], v[j], 1 - u[j] - v[j])
            # depth gap to the next hit (ties would make the nearest ambiguous)
            ts = np.sort(t[hit])
            if len(ts) > 1 and ts[1] - ts[0] < 1e-9:
                margin[y, x] = 0
    return fid, bary, depth, margin


def _lambert_normals(mesh):
    """Area-weighted vertex normals: unit face normal times face area, summed."""
    P = np.asarray(mesh.pos, np.float64)
    F = np.asarray(mesh.faces)
    cr = np.cross(P[F[:, 1]] - P[F[:, 0]], P[F[:, 2]] - P[F[:, 0]])
    area = 0.5 * np.linalg.norm(cr, axis=1)
    unit = cr / np.linalg.norm(cr, axis=1, keepdims=True)
    acc = np.zeros_like(P)
    for k in range(3):
        np.add.at(acc, F[:, k], unit * area[:, None])
    return acc / np.linalg.norm(acc, axis=1, keepdims=True)


@pytest.mark.parametrize("shade_mode", [0, 1, 2])
def test_hard_mode_matches_raycast(shade_mode):
    g = synth.rng(11)
    pos, faces = synth.icosphere(1)
    pos = synth.displace(pos, 0.15, 5)
    if shade_mode == 0:
        mesh = synth.Mesh(pos.astype(np.float32), faces, col=g.random(pos.shape).astype(np.float32))
    else:
        pos, faces, uv = synth.icosphere_uv(pos, faces)
        tex = np.zeros((16, 8, 4), np.float32)
        tex[..., :3] = g.random((16, 8, 3))
        mesh = synth.Mesh(pos.astype(np.float32), faces, uv=uv.astype(np.float32), tex=tex)
    view = synth.View(synth.camera_mvp((0.5, 0.8, 2.6), 40, 40), 0, 40, 40)
    prm = synth.Params(K=2, r=2 / 40, sigma=0.5 / 40, delta=2 / 40, edge_mode=2, shade_mode=shade_mode)
    r = oracle.render(mesh, view, prm)
    fid, bary, depth, margin = _raycast(mesh, view)
    ok = margin > 1e-7
    assert ok.mean() > 0.98
    np.testing.assert_array_equal(r["sh"][ok], (fid >= 0)[ok])
    hit = ok & (fid >= 0)
    np.testing.assert_array_equal(r["ids"][0][hit], fid[hit])
    np.testing.assert_allclose(r["key"][0][hit], 0.5 * depth[hit], atol=1e-12)
    F = np.asarray(mesh.faces)
    vi = F[fid[hit]]
    b = bary[hit]
    if shade_mode == 0:
        col = (b[..., None] * mesh.col.astype(np.float64)[vi]).sum(1)
    else:
        uv = (b[..., None] * mesh.uv.astype(np.float64)[vi]).sum(1)
        x = uv[:, 0] * tex.shape[1] - 0.5
        y = uv[:, 1] * tex.shape[0] - 0.5
        col = np.stack([ndimage.map_coordinates(tex[..., c].astype(np.float64), [y, x], order=1, mode="grid-wrap")
                        for c in range(3)], 1)
        if shade_mode == 2:
            N = _lambert_normals(mesh)
            n = (b[..., None] * N[vi]).sum(1)
            n /= np.linalg.norm(n, axis=1, keepdims=True)
            col = col * np.maximum(0, n @ view.light.astype(np.float64))[:, None]
    np.testing.assert_allclose(r["rgba"][..., :3][hit], col, atol=1e-9)
    np.testing.assert_array_equal(r["rgba"][..., 3][ok], (fid >= 0)[ok].astype(float))


def test_planar_mesh_normals_equal_plane_normal():
    """Lambert on a flat mesh: every fragment normal is the plane normal."""
    W = H = 16
    V, F = grid_mesh(4, W, H, jitter=1.0, seed=2)
    tex = np.zeros((4, 4, 4), np.float32)
    tex[..., :3] = 1.0
    uv = (V / np.array([W, H])).astype(np.float32)
    mesh = pixel_mesh(V, F, W, H, uv=uv, tex=tex)
    # identity MVP keeps y down: the triangle winding decides the normal sign, so
    # light along +-z gives shading 1 (facing) or 0
    s = pixel_scene(mesh, W, H, K=1, r=1 / 16, sigma=0.2 / 16, delta=1 / 16, edge_mode=2, shade_mode=2)
    seen = []
    for lz in (1.0, -1.0):
        s.views[0].light = np.array([0, 0, lz], np.float32)
        vals = np.unique(np.round(_render(s)["rgba"][..., 0], 12))
        assert len(vals) == 1
        seen.append(vals[0])
    assert sorted(seen) == [0.0, 1.0]          # one of +-z faces the plane, the other not
    facing = 1.0 if seen[0] == 1.0 else -1.0
    s.views[0].light = np.array([0.6, 0.0, 0.8 * facing], np.float32)
    vals = _render(s)["rgba"][..., 0]
    assert np.abs(vals - float(np.float32(0.8))).max() < 1e-12



# ----------------------------------------------------------------------------
# invariants of the adjoint
# ----------------------------------------------------------------------------

def test_colour_gradient_conservation():
    """E = 1, vertex colours: the blend weights and perspective barycentrics each sum
    to 1, so sum_v dL/dcol_v = sum over covered pixels of dL/dI_rgb."""
    s = synth.config1()
    p = synth.Params(K=3, r=2 / 64, sigma=0.3 / 64, delta=2 / 64, edge_mode=1, shade_mode=0)
    g = np.random.default_rng(1).normal(size=(64, 64, 4))
    r = oracle.render(s.meshes[0], s.views[0], p)
    _, gc, _ = oracle.backward(s.meshes[0], s.views[0], p, g)
    covered = r["ids"][0] >= 0
    np.testing.assert_allclose(gc.sum(0), g[..., :3][covered].sum(0), rtol=1e-12, atol=1e-10)


def test_texel_gradient_conservation():
    """E = 1, unlit texture: bilinear weights sum to 1, so the texel gradient sums to
    the summed pixel colour gradient over covered pixels."""
    s = synth.config2()
    m = s.meshes[0]
    p = synth.Params(K=3, r=2 / 256, sigma=0.3 / 256, delta=2 / 256, edge_mode=1, shade_mode=1)
    g = np.random.default_rng(2).normal(size=(64, 64, 4))
    win = (96, 96, 64, 64)
    r = oracle.render(m, s.views[0], p, window=win)
    _, _, gt = oracle.backward(m, s.views[0], p, g, window=win)
    covered = r["ids"][0] >= 0
    np.testing.assert_allclose(gt[..., :3].sum((0, 1)), g[..., :3][covered].sum(0), rtol=1e-11, atol=1e-9)
    assert np.all(gt[..., 3] == 0)


def test_uniform_colour_single_face_has_no_colour_position_gradient():
    """One face, uniform colour, E = 1: I_c^e = sum D C / sum D = C, so only the
    silhouette carries a position gradient."""
    W = H = 24
    s = pixel_scene(pixel_mesh([(4, 3), (20, 6), (7, 19)], [(0, 1, 2)], W, H, col=np.full((3, 3), 0.7)), W, H,
                    K=3, r=3 / 24, sigma=1 / 24, delta=3 / 24, edge_mode=1)
    g = np.random.default_rng(3).normal(size=(H, W, 4))
    g[..., 3] = 0
    gp, _, _ = oracle.backward(s.meshes[0], s.views[0], s.params, g)
    assert np.abs(gp).max() < 1e-12


# ----------------------------------------------------------------------------
# central finite differences of the forward vs the adjoint
# ----------------------------------------------------------------------------

def _fd_scene(shade_mode, seed):
    g = np.random.default_rng(seed)
    pos = np.array([[-0.6, -0.5, 0.1], [0.5, -0.4, -0.2], [-0.1, 0.6, 0.0], [0.7, 0.5, 0.3], [-0.7, 0.4, -0.3]])
    pos += g.uniform(-0.05, 0.05, pos.shape)
    faces = np.array([[0, 1, 2], [1, 3, 2], [0, 2, 4]], np.int32)
    col = g.random((5, 3))
    uv = g.uniform(0.05, 0.95, (5, 2))
    tex = np.zeros((6, 5, 4))
    tex[..., :3] = g.random((6, 5, 3))
    ntex = np.zeros((6, 5, 4))   # tangent-space normals near +z: x, y in 0.5 +- 0.2, z in [0.75, 1]
    ntex[..., :2] = 0.5 + g.uniform(-0.2, 0.2, (6, 5, 2))
    ntex[..., 2] = g.uniform(0.75, 1.0, (6, 5))
    mesh = synth.Mesh(pos, faces, col=col, uv=uv, tex=tex, ntex=ntex)
    view = synth.View(synth.camera_mvp((0.4, 0.3, 2.2), 28, 28).astype(np.float64), 0, 28, 28,
                      light=np.array([0.48, 0.6, 0.64]))
    return mesh, view


def _state(r):
    return (r["ids"].tobytes(), r["hard"].tobytes(), r["sh"].tobytes(), r["edge"].tobytes())


@pytest.mark.parametrize("shade_mode,edge_mode,K", [(0, 0, 3), (0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 1, 3), (2, 0, 3), (2, 1, 2),
                                                    (3, 0, 3), (3, 1, 2), (3, 2, 1)])
def test_adjoint_matches_central_differences(shade_mode, edge_mode, K):
    mesh, view = _fd_scene(shade_mode, 7 + shade_mode)
    r_px = 3.0
    prm = synth.Params(K=K, r=r_px / 28, sigma=r_px / 28 / 5, delta=2 / 28, edge_mode=edge_mode, shade_mode=shade_mode)
    g = np.random.default_rng(5).normal(size=(28, 28, 4))
    base = oracle.render(mesh, view, prm)
    st0 = _state(base)
    gp, gc, gt, gnt = oracle.backward(mesh, view, prm, g, want_ntex=True)

    def loss(m):
        r = oracle.render(m, view, prm)
        return (g * r["rgba"]).sum(), _state(r)

    def fd(attr, idx, h):
        arr = getattr(mesh, attr)
        plus, minus = arr.copy(), arr.copy()
        plus[idx] += h
        minus[idx] -= h
        mp = synth.Mesh(**{**mesh.__dict__, attr: plus})
        mm = synth.Mesh(**{**mesh.__dict__, attr: minus})
        lp, sp = loss(mp)
        lm, sm = loss(mm)
        if sp != st0 or sm != st0:
            return None
        return (lp - lm) / (2 * h)

    checked = 0
    num, ana = [], []
    for i in range(mesh.pos.shape[0]):
        for c in range(3):
            d = fd("pos", (i, c), 1e-6)
            if d is None:
                continue
            num.append(d)
            ana.append(gp[i, c])
            checked += 1
    if shade_mode == 0:
        for i in range(mesh.col.shape[0]):
            for c in range(3):
                num.append(fd("col", (i, c), 1e-4))
                ana.append(gc[i, c])
    else:
        nz = np.argwhere(np.abs(gt) > 0)
        for idx in nz[:: max(1, len(nz) // 40)]:
            d = fd("tex", tuple(idx), 1e-4)
            if d is not None:
                num.append(d)
                ana.append(gt[tuple(idx)])
    if shade_mode == 3:
        nz = np.argwhere(np.abs(gnt) > 0)
        assert len(nz) > 0
        for idx in nz[:: max(1, len(nz) // 40)]:
            d = fd("ntex", tuple(idx), 1e-5)
            if d is not None:
                num.append(d)
                ana.append(gnt[tuple(idx)])
    num, ana = np.array(num), np.array(ana)
    assert checked >= 12
    assert np.abs(ana).max() > 0
    err = np.linalg.norm(num - ana) / np.linalg.norm(ana)
    assert err < 1e-6, err
    assert np.abs(num - ana).max() < 1e-5 * np.abs(ana).max()


@pytest.mark.parametrize("shade_mode,edge_mode,K", [(0, 0, 3), (1, 1, 2), (2, 0, 3), (2, 1, 2), (2, 2, 1), (3, 0, 3)])
def test_camera_and_light_adjoint_match_central_differences(shade_mode, edge_mode, K):
    """dL/dMVP and dL/dlight (the camera and light parameters of Theta, Sec. 3.4.1)
    against central differences of the oracle's forward; the depth row of the matrix
    has no gradient (depth only orders the layers), nor has the light without Lambert."""
    mesh, view = _fd_scene(shade_mode, 17 + shade_mode)
    r_px = 3.0
    prm = synth.Params(K=K, r=r_px / 28, sigma=r_px / 28 / 5, delta=2 / 28, edge_mode=edge_mode, shade_mode=shade_mode)
    g = np.random.default_rng(9).normal(size=(28, 28, 4))
    st0 = _state(oracle.render(mesh, view, prm))
    _, _, _, gm, gl = oracle.backward(mesh, view, prm, g, camera=True)

    def fd(attr, idx, h):
        arr = np.asarray(getattr(view, attr), np.float64)
        plus, minus = arr.copy(), arr.copy()
        plus[idx] += h
        minus[idx] -= h
        vp = synth.View(**{**view.__dict__, attr: plus})
        vm = synth.View(**{**view.__dict__, attr: minus})
        rp, rm = oracle.render(mesh, vp, prm), oracle.render(mesh, vm, prm)
        if _state(rp) != st0 or _state(rm) != st0:
            return None
        return ((g * rp["rgba"]).sum() - (g * rm["rgba"]).sum()) / (2 * h)

    num, ana = [], []
    for e in range(16):
        d = fd("mvp", e, 1e-6)
        if d is not None:
            num.append(d)
            ana.append(gm[e])
    assert len(num) >= 12
    assert np.all(gm[8:12] == 0)
    for c in range(3):
        d = fd("light", c, 1e-6)
        if d is not None:
            num.append(d)
            ana.append(gl[c])
    if shade_mode < 2:
        assert np.all(gl == 0)
    else:
        assert np.abs(gl).max() > 0
    num, ana = np.array(num), np.array(ana)
    assert np.abs(ana).max() > 0
    err = np.linalg.norm(num - ana) / np.linalg.norm(ana)
    assert err < 1e-6, err
    assert np.abs(num - ana).max() < 1e-5 * np.abs(ana).max()


# ----------------------------------------------------------------------------
# inverse UV (Sec. 3.3.2, Alg. 1): closed forms on a pixel-aligned textured quad
# ----------------------------------------------------------------------------

def _uv_quad(tex_w, W=16):
    """Screen-filling quad whose UV puts pixel centre X + 1/2 at u W = X + 1/2 (so at
    u tex_w = (X + 1/2) tex_w / W); unlit texture, one hard layer."""
    V = np.array([[-1, -1], [W + 1, -1], [W + 1, W + 1], [-1, W + 1]], np.float64)
    uv = V / W
    tex = np.zeros((W, tex_w, 4))
    tex[..., :3] = np.random.default_rng(2).random((W, tex_w, 3))
    mesh = pixel_mesh(V, [[0, 1, 2], [0, 2, 3]], W, W, uv=uv, tex=tex)
    return pixel_scene(mesh, W, W, K=1, r=1 / W, sigma=0.3 / W, delta=1 / W, edge_mode=2, shade_mode=1)


@pytest.mark.parametrize("jitter,shift", [((0.0, 0.0), 0), ((0.6, 0.0), 1), ((0.0, -0.7), -1)])
def test_inverse_uv_pixel_aligned(jitter, shift):
    """One texel per pixel: the inverse UV is the identity, shifted by one texel when the
    jitter moves the sample across a texel edge (REPEAT wrap); the texel gradient is
    the pixel gradient moved the same way."""
    W = 16
    s = _uv_quad(W, W)
    g = np.random.default_rng(4).normal(size=(W, W, 4))
    *_, rec = oracle.backward(s.meshes[0], s.views[0], s.params, g, inverse_uv=(jitter, 0))
    grad, winner, stable = oracle.inverse_uv_texels([rec], W, W)
    axis = 1 if jitter[0] else 0
    expect = np.roll(g[..., :3], shift, axis=axis).reshape(-1, 3)
    np.testing.assert_allclose(grad, expect, rtol=0, atol=1e-12)
    assert stable.all() and (winner >= 0).all()


def test_inverse_uv_last_writer_wins():
    """Two pixels per texel (the texture is half as wide as the view): the texel keeps
    the later sample, the right pixel of each pair."""
    W = 16
    s = _uv_quad(W // 2, W)
    g = np.random.default_rng(6).normal(size=(W, W, 4))
    *_, rec = oracle.backward(s.meshes[0], s.views[0], s.params, g, inverse_uv=((0.0, 0.0), 0))
    assert len(rec["slot"]) == W * W
    grad, winner, _ = oracle.inverse_uv_texels([rec], W // 2, W)
    np.testing.assert_allclose(grad, g[:, 1::2, :3].reshape(-1, 3), rtol=0, atol=1e-12)
    ys, xs = np.divmod(np.arange(W * W // 2), W // 2)
    np.testing.assert_array_equal(winner, ys * W + 2 * xs + 1)   # K = 1: sample = pixel


# ----------------------------------------------------------------------------
# brute force equals the bbox pre-tested variant bit for bit
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("cfg", [1, 2])
def test_brute_force_equals_bbox(cfg):
    s = synth.CONFIGS[cfg]()
    win = None if cfg == 1 else (100, 80, 40, 40)
    a = oracle.render(s.meshes[0], s.views[0], s.params, window=win, brute_force=False)
    b = oracle.render(s.meshes[0], s.views[0], s.params, window=win, brute_force=True)
    for k in ("rgba", "ids", "hard", "dist", "key", "sh", "edge", "margin_hard", "margin_cand", "n_hard"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


# ----------------------------------------------------------------------------
# K >= 2 blend (Sec. 3.4.3): I_c^e = sum D_k C_k / sum D_k, I_s^e = 1 - prod (1 - D_k)
# ----------------------------------------------------------------------------

def _blend_scene(K):
    """Three nested right triangles with legs on the pixel axes (w = 1, constant depths,
    one uniform colour per face, so C_k is the face colour whatever the barycentrics):
    id 0 red at depth 0.6, id 1 blue at depth 0.3, id 2 green at depth 0.45."""
    W = H = 32
    V = [(2, 2), (30, 2), (2, 30), (6, 6), (30, 6), (6, 30), (4, 4), (30, 4), (4, 30)]
    z = [0.6] * 3 + [0.3] * 3 + [0.45] * 3
    col = [(1, 0, 0)] * 3 + [(0, 0, 1)] * 3 + [(0, 1, 0)] * 3
    return pixel_scene(pixel_mesh(V, [(0, 1, 2), (3, 4, 5), (6, 7, 8)], W, H, z=z, col=col), W, H, K=K,
                       r=8 / 32, sigma=4 / 32, delta=8 / 32, edge_mode=1)


# per pixel: (face id, signed pixel distance) in Shift order, distances read off the
# geometry by hand (legs x = a, y = a and hypotenuse x + y = 32 + a of the face at a)
_BLEND_PIXELS = {
    # (10.5, 10.5): inside all three; nearest feature of each face is a leg
    (10, 10): [(1, 4.5), (2, 6.5), (0, (32 - 21) / math.sqrt(2))],
    # (4.5, 10.5): inside faces 2 (leg x = 4 at 0.5 px) and 0 (leg x = 2 at 2.5 px); face 1
    # is soft, 1.5 px left of its leg x = 6 (foot (6, 10.5) inside the leg)
    (4, 10): [(2, 0.5), (0, 2.5), (1, -1.5)],
    # (1.5, 1.5): outside all three; each nearest feature is the corner (a, a)
    (1, 1): [(0, -math.sqrt(0.5)), (2, -2.5 * math.sqrt(2)), (1, -4.5 * math.sqrt(2))],
}
_BLEND_COLOUR = {0: (1.0, 0.0, 0.0), 1: (0.0, 0.0, 1.0), 2: (0.0, 1.0, 0.0)}


@pytest.mark.parametrize("K", [2, 3])
def test_multi_layer_blend_equations(K):
    """With E = 1 the pixel is the D-weighted mean of its K layers' colours and the
    silhouette is 1 - prod_k (1 - D_k), D_k = sigmoid(d_k / sigma) (the colour and
    silhouette blend equations of Sec. 3.4.3), from hand-computed distances; with
    K = 2 the farthest of the three layers is dropped."""
    s = _blend_scene(K)
    r = _render(s)
    sig_px = 4.0
    for (x, y), layers in _BLEND_PIXELS.items():
        kept = layers[:K]
        assert [int(i) for i in r["ids"][:, y, x]] == [i for i, _ in kept]
        D = np.array([1.0 / (1.0 + math.exp(-d / sig_px)) for _, d in kept])
        C = np.array([_BLEND_COLOUR[i] for i, _ in kept])
        rgb = (D[:, None] * C).sum(0) / D.sum()
        alpha = 1.0 - np.prod(1.0 - D)
        np.testing.assert_allclose(r["rgba"][y, x, :3], rgb, rtol=0, atol=1e-12)
        assert r["rgba"][y, x, 3] == pytest.approx(alpha, abs=1e-12)
        np.testing.assert_allclose(r["dist"][:K, y, x] * 32, [d for _, d in kept], atol=1e-12)


# ----------------------------------------------------------------------------
# culling (reading: a face with a corner at w <= 1e-6 or depth outside [0, 1] is dropped)
# ----------------------------------------------------------------------------

def _cull_scene(bad_corner, mvp):
    """A quad of two faces (ids 0, 1) over the whole image at depth 1/2 and, in front of
    it, face 2 whose first corner is ``bad_corner`` = (x, y, z) in object space (the other
    two corners are ordinary)."""
    W = H = 24
    pos = np.array([[-1.2, -1.2, 1.0], [1.2, -1.2, 1.0], [1.2, 1.2, 1.0], [-1.2, 1.2, 1.0],
                    bad_corner, [0.6, -0.5, 1.0], [-0.3, 0.7, 1.0]], np.float32)
    faces = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6]], np.int32)
    col = synth.rng(4).random((7, 3)).astype(np.float32)
    mesh = synth.Mesh(pos, faces, col=col)
    view = synth.View(np.asarray(mvp, np.float32).reshape(16), 0, W, H)
    return synth.Scene("cull", [mesh], [view], synth.Params(K=3, r=2 / 24, sigma=1 / 24, delta=2 / 24))


# clip = (x, y, z_depth, w): depth from the z row; the w row either 1 (depth = the z row)
# or the object z (so w follows the corner's z while depth stays 1/2 wherever w != 0)
_MVP_DEPTH = [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0.5, 0], [0, 0, 0, 1]]
_MVP_W = [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0.5, 0], [0, 0, 1, 0]]


@pytest.mark.parametrize("mvp,bad,kept", [
    (_MVP_DEPTH, (-0.5, -0.4, 2.5), False),    # depth 1.25 > 1
    (_MVP_DEPTH, (-0.5, -0.4, -0.5), False),   # depth -0.25 < 0
    (_MVP_DEPTH, (-0.5, -0.4, 2.0), True),     # depth exactly 1: kept
    (_MVP_DEPTH, (-0.5, -0.4, 0.0), True),     # depth exactly 0: kept
    (_MVP_W, (-0.5, -0.4, -0.5), False),       # w = -0.5 (depth 1/2)
    (_MVP_W, (-0.5, -0.4, 1e-7), False),       # 0 < w <= 1e-6 (depth 1/2)
    (_MVP_W, (-0.5, -0.4, 0.5), True),         # w = 1/2: kept
])
def test_culling_near_and_far(mvp, bad, kept):
    """A culled face is absent from every layer and the other faces' layers, keys and
    image are exactly those of the scene without it; a face at the limits is kept."""
    s = _cull_scene(bad, mvp)
    r = _render(s)
    m = s.meshes[0]
    without = synth.Scene("cull2", [synth.Mesh(m.pos, m.faces[:2], col=m.col)], s.views, s.params)
    r2 = _render(without)
    if kept:
        assert (r["ids"] == 2).any()
        return
    assert not (r["ids"] == 2).any()
    for k in ("ids", "hard", "key", "rgba", "dist", "sh", "edge"):
        np.testing.assert_array_equal(r[k], r2[k], err_msg=k)
