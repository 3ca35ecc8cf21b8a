"""Inverse-UV texel gradient (texgrad_mode 2; Sec. 3.3.2, Alg. 1) on the GPU:
closed forms on a pixel-aligned textured quad, and the oracle's sequential
last-writer rule on textured spheres (one view and several).  Texel winners are
sample numbers (pixel * K + layer): compared exactly where the oracle's discrete
decisions have margin and both winners come from pixels whose layers are stable."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2204_01386_gb300 import PackedScene, Renderer
from paper_2204_01386_gb300 import binding as B
from parity import GRAD_TOL, masks, rel_l2
from scenes_small import pixel_mesh, pixel_scene

pytestmark = pytest.mark.gpu


def _with_mode(scene, jitter):
    p = dataclasses.replace(scene.params, texgrad_mode=2)
    p.uv_jitter = tuple(jitter)
    return dataclasses.replace(scene, params=p)


def _gpu_inverse_uv(scene, grads, store_layers=True, tile=0, schedule=0):
    """Runs forward + adjoint; returns (texel gradient [n_texels, 3], winners [n_texels])."""
    ps = PackedScene(scene.meshes, "cuda")
    r = Renderer(ps, scene.views, scene.params, tile=tile, schedule=schedule)
    _, ids = r.forward(store_layers=True)
    g = torch.zeros(r.n_pix, 4, device="cuda")
    for i, v in enumerate(r.views):
        g[v.pix_off: v.pix_off + v.width * v.height] = torch.as_tensor(
            np.asarray(grads[i], np.float32).reshape(-1, 4), device="cuda")
    win = torch.full((ps.n_texels,), -7, dtype=torch.int32, device="cuda")
    lib = B.load()
    lib.dressi_set_inverse_uv_buffer(win.data_ptr())
    try:
        _, _, gt = r.backward(g, ids=ids if store_layers else None)
        torch.cuda.synchronize()
    finally:
        lib.dressi_set_inverse_uv_buffer(None)
    assert r.device_status() == 0
    gt = gt.cpu().numpy().astype(np.float64)
    assert not np.any(gt[:, 3])
    return gt[:, :3], win.cpu().numpy().astype(np.int64)


def _quad(tex_w, W=16):
    V = np.array([[-1, -1], [W + 1, -1], [W + 1, W + 1], [-1, W + 1]], np.float64)
    tex = np.zeros((W, tex_w, 4), np.float32)
    tex[..., :3] = np.random.default_rng(2).random((W, tex_w, 3))
    mesh = pixel_mesh(V, [[0, 1, 2], [0, 2, 3]], W, W, uv=V / W, tex=tex)
    return pixel_scene(mesh, W, W, K=1, r=1 / W, sigma=0.3 / W, delta=1 / W, edge_mode=2, shade_mode=1)


@pytest.mark.parametrize("jitter,axis,shift", [((0.0, 0.0), 1, 0), ((0.6, 0.0), 1, 1), ((0.0, -0.7), 0, -1)])
def test_inverse_uv_pixel_aligned_quad(jitter, axis, shift):
    W = 16
    s = _with_mode(_quad(W, W), jitter)
    g = np.random.default_rng(4).normal(size=(W, W, 4)).astype(np.float32)
    gt, win = _gpu_inverse_uv(s, [g])
    np.testing.assert_array_equal(gt, np.roll(g[..., :3], shift, axis=axis).reshape(-1, 3))
    expect = np.roll(np.arange(W * W).reshape(W, W), shift, axis=axis).reshape(-1)
    np.testing.assert_array_equal(win, expect)


def _compare(scene, jitter, store_layers=True, seed=0, tile=0, schedule=0):
    s = _with_mode(scene, jitter)
    rng = np.random.default_rng(seed)
    grads, recs, pix_stable = [], [], []
    base = 0
    for v in s.views:
        o = oracle.render(s.meshes[v.mesh], v, s.params)
        s_ids, s_val = masks(o, s.params, v)
        gv = np.where(s_val[..., None], rng.normal(size=(v.height, v.width, 4)), 0.0)
        grads.append(gv)
        *_, rec = oracle.backward(s.meshes[v.mesh], v, s.params, gv, inverse_uv=(jitter, base))
        recs.append(rec)
        pix_stable.append(s_ids.reshape(-1))
        base += v.width * v.height
    pix_stable = np.concatenate(pix_stable)
    gt, win = _gpu_inverse_uv(s, grads, store_layers, tile, schedule)
    m = s.meshes[0]
    o_grad, o_win, stable = oracle.inverse_uv_texels(recs, m.tex.shape[1], m.tex.shape[0])
    K = s.params.K
    ok_pix = lambda w: (w < 0) | pix_stable[np.maximum(w, 0) // K]
    cmp = stable & ok_pix(o_win) & ok_pix(win)
    written = o_win >= 0
    # soft fragments at a mesh corner sample exactly that vertex's UV, which here lies
    # on a texel edge: their texel is decided by rounding and is left out
    assert cmp[written].mean() > 0.6, cmp[written].mean()
    np.testing.assert_array_equal(win[cmp], o_win[cmp])
    e = rel_l2(gt[cmp], o_grad[cmp])
    assert e <= GRAD_TOL, e
    return cmp.sum()


@pytest.mark.parametrize("store_layers", [True, False])
@pytest.mark.parametrize("jitter", [(0.0, 0.0), (0.23, -0.17)])
def test_inverse_uv_textured_sphere(store_layers, jitter):
    assert _compare(synth.config2(), jitter, store_layers) > 1000


@pytest.mark.parametrize("tile,schedule", [(0, 0), (32, 2)])
def test_inverse_uv_several_views(tile, schedule):
    """Three views of one sphere: a texel seen in several views keeps the last view's
    sample, whichever order the tiles run in."""
    assert _compare(synth.config3(n_views=3, res=128), (-0.31, 0.12), tile=tile, schedule=schedule) > 1000
