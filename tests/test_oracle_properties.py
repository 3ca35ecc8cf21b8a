"""Seeded property tests of the oracle over random tiny scenes (hypothesis): invariants
that hold for any input.  The bbox-culled oracle equals its brute-force mode; the K
layers are in (key, id) order with empty layers last; hard layers have Shift keys at most
1/2 and soft ones at least 1/2 (Eq. Shift: 0.5 z inside the face, 0.5 + 0.5 |d| / S
outside); S^H is the front layer's hard flag; E is recomputed from S^H by its definition
(the Chebyshev window of radius rho holds both values, Sec. 3.4.3); colours and coverage
stay in [0, 1] (the blend is convex); the adjoint of a zero image gradient is zero."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
from scenes_small import pixel_mesh, pixel_scene  # noqa: E402

W = H = 16


@st.composite
def scenes(draw):
    n_faces = draw(st.integers(1, 5))
    coords = st.floats(-4.0, W + 4.0, allow_nan=False, allow_infinity=False)
    V = [(draw(coords), draw(coords)) for _ in range(3 * n_faces)]
    z = [draw(st.floats(0.05, 0.95)) for _ in range(3 * n_faces)]
    col = [(draw(st.floats(0, 1)), draw(st.floats(0, 1)), draw(st.floats(0, 1))) for _ in range(3 * n_faces)]
    F = [(3 * i, 3 * i + 1, 3 * i + 2) for i in range(n_faces)]
    K = draw(st.integers(1, 4))
    r_px = draw(st.floats(0.25, 3.0))
    rho_px = draw(st.integers(1, 3))
    edge_mode = draw(st.integers(0, 2))
    m = pixel_mesh(V, F, W, H, z=z, col=col)
    return pixel_scene(m, W, H, K=K, r=r_px / W, sigma=r_px / W / 7, delta=rho_px / W, edge_mode=edge_mode,
                       shade_mode=0)


def _window_has_both(sh, rho):
    h, w = sh.shape
    e = np.zeros_like(sh)
    for y in range(h):
        for x in range(w):
            win = sh[max(0, y - rho):y + rho + 1, max(0, x - rho):x + rho + 1]
            e[y, x] = 1 if (win.min() == 0 and win.max() == 1) else 0
    return e


@settings(max_examples=30, deadline=None, derandomize=True)
@given(scenes())
def test_oracle_invariants(s):
    m, v, p = s.meshes[0], s.views[0], s.params
    o = oracle.render(m, v, p)
    b = oracle.render(m, v, p, brute_force=True)
    for k in ("rgba", "ids", "hard", "key", "sh", "edge"):
        assert np.array_equal(o[k], b[k]), k
    K = p.K
    ids, hard, key = o["ids"], o["hard"], o["key"]
    empty = ids < 0
    # empty layers only after the filled ones
    assert not np.any(empty[:-1] & ~empty[1:])
    # (key, id) ascending over the filled layers
    for k in range(K - 1):
        both = ~empty[k] & ~empty[k + 1]
        kk, kn = key[k][both], key[k + 1][both]
        assert np.all((kk < kn) | ((kk == kn) & (ids[k][both] < ids[k + 1][both])))
    # hard keys are at most 1/2, soft keys at least 1/2 (a soft fragment on an edge its
    # face does not own, or a hard one at depth 1, sits at exactly 1/2)
    filled = ~empty
    kf, hf = key[:K][filled], hard[filled] != 0
    assert np.all(kf[hf] <= 0.5) and np.all(kf[~hf] >= 0.5)
    # S^H: the front layer exists and is hard
    assert np.array_equal(o["sh"] != 0, (~empty[0]) & (hard[0] != 0))
    # E from S^H by its definition (edge_mode 0), or constant
    if p.edge_mode == 0:
        rho = max(1, int(round(p.delta * max(W, H))))
        assert np.array_equal(o["edge"], _window_has_both(o["sh"].astype(np.int64), rho))
    else:
        assert np.all(o["edge"] == (1 if p.edge_mode == 1 else 0))
    # convex blend: colours and coverage in [0, 1]
    assert np.all(o["rgba"] >= -1e-15) and np.all(o["rgba"] <= 1 + 1e-12)
    # outside every candidate the image is zero
    assert np.all(o["rgba"][empty[0]] == 0)
    # the adjoint is linear: a zero image gradient gives zero gradients
    gp, gc, _ = oracle.backward(m, v, p, np.zeros((H, W, 4)))
    assert not np.any(gp) and not np.any(gc)
