"""Forward from stored layers (the static-geometry raster cache): re-shading the layer
ids that an earlier forward stored equals a full forward with the new shading inputs,
bit for bit, and matches the FP64 oracle for those inputs."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2204_01386_gb300 import PackedScene, Renderer
from parity import FWD_TOL, masks

pytestmark = pytest.mark.gpu


def _renderer(scene, tile=0, schedule=0):
    ps = PackedScene(scene.meshes, "cuda")
    return Renderer(ps, scene.views, scene.params, tile=tile, schedule=schedule)


def _restyled(scene, seed, sigma_scale=1.0, delta_scale=1.0, edge_mode=None):
    """Same geometry and views; new colours / textures, light and blend parameters."""
    rng = np.random.default_rng(seed)
    meshes = []
    for m in scene.meshes:
        col = None if m.col is None else rng.uniform(0, 1, m.col.shape).astype(np.float32)
        tex = None
        if m.tex is not None:
            tex = np.clip(m.tex.astype(np.float32) * 0.6 + rng.uniform(0, 0.4, m.tex.shape), 0, 1).astype(m.tex.dtype)
        meshes.append(dataclasses.replace(m, col=col, tex=tex))
    light = rng.normal(size=3)
    light = (light / np.linalg.norm(light)).astype(np.float32)
    views = [dataclasses.replace(v, light=light) for v in scene.views]
    p = dataclasses.replace(scene.params, sigma=scene.params.sigma * sigma_scale,
                            delta=scene.params.delta * delta_scale,
                            edge_mode=scene.params.edge_mode if edge_mode is None else edge_mode)
    return dataclasses.replace(scene, meshes=meshes, views=views, params=p)


@pytest.mark.parametrize("tile,schedule", [(0, 0), (32, 2), (16, 1)])
@pytest.mark.parametrize("cfg", ["config1", "config2"])
def test_from_layers_reproduces_forward(cfg, tile, schedule):
    s = getattr(synth, cfg)()
    r = _renderer(s, tile, schedule)
    out, ids = r.forward(store_layers=True)
    again = r.forward_from_layers(ids)
    torch.cuda.synchronize()
    assert r.device_status() == 0
    d = (out - again).abs().max().item()
    print("max diff", d, "pixels differing", int((out != again).any(1).sum()))
    assert torch.equal(out, again), d


@pytest.mark.parametrize("cfg,kw", [("config1", {}), ("config2", {}),
                                    ("config2", dict(sigma_scale=2.0, delta_scale=2.0)),
                                    ("config2", dict(edge_mode=1))])
def test_from_layers_with_new_shading_inputs(cfg, kw):
    """Layers of the original scene, shading inputs of a restyled one: equal to the
    restyled scene's own forward, and within the forward tolerance of the oracle."""
    s = getattr(synth, cfg)()
    s2 = _restyled(s, 7, **kw)
    _, ids = _renderer(s).forward(store_layers=True)
    r2 = _renderer(s2)
    full, ids2 = r2.forward(store_layers=True)
    cached = r2.forward_from_layers(ids)
    torch.cuda.synchronize()
    assert torch.equal(ids, ids2)          # the layers do not depend on the shading inputs
    assert torch.equal(full, cached)
    v = s2.views[0]
    o = oracle.render(s2.meshes[v.mesh], v, s2.params)
    _, s_val = masks(o, s2.params, v)
    got = r2.view_image(cached, 0).cpu().numpy().astype(np.float64)
    err = np.abs(got - o["rgba"])[s_val]
    assert s_val.mean() > 0.5 and err.max() <= FWD_TOL, err.max()


def test_from_layers_then_backward_from_layers():
    """A texture-only optimisation step: forward from stored layers, then the adjoint
    from the same layers, equals the full forward / adjoint of the restyled scene."""
    s = synth.config2()
    s2 = _restyled(s, 11)
    _, ids = _renderer(s).forward(store_layers=True)
    r2 = _renderer(s2)
    out = r2.forward_from_layers(ids)
    g = torch.as_tensor(np.random.default_rng(3).normal(size=(r2.n_pix, 4)), dtype=torch.float32, device="cuda")
    gp_a, _, gt_a = r2.backward(g, ids=ids)
    gp_a, gt_a = gp_a.clone(), gt_a.clone()
    full, ids2 = r2.forward(store_layers=True)
    gp_b, _, gt_b = r2.backward(g, ids=ids2)
    torch.cuda.synchronize()
    assert torch.equal(out, full)
    # the gradients are sums of float atomics, whose order varies between runs
    for a, b in ((gp_a, gp_b), (gt_a, gt_b)):
        rel = (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()
        assert rel < 1e-5, rel


def test_from_layers_rejects_missing_layers():
    import ctypes as C

    from paper_2204_01386_gb300 import binding as B
    s = synth.config1()
    r = _renderer(s)
    out = torch.empty(r.n_pix, 4, device="cuda")
    sc = r.scene.c_struct()
    code = r.lib.dressi_forward_from_layers(C.byref(sc), r.views, r.n_views, C.byref(r.params), None,
                                            out.data_ptr(), r.n_pix, r.ws.data_ptr(), r.ws_bytes,
                                            r.status.data_ptr(), r._stream())
    assert code == B.DRESSI_ERR_ARG
