"""The backward taking the forward's setup (reuse_setup): vertex transform, face table,
normals and tile lists left in the workspace by the forward give the same gradients as
rebuilding them, with fewer launches; the renderer takes them only while the
positions are unchanged."""
import pytest
import torch

import synth
from paper_2204_01386_gb300 import PackedScene, Renderer, binding as B

pytestmark = pytest.mark.gpu


def _setup(cfg, store):
    s = getattr(synth, cfg)()
    ps = PackedScene(s.meshes, "cuda")
    r = Renderer(ps, s.views, s.params)
    out, ids = r.forward(store_layers=store)
    g = torch.Generator(device="cuda").manual_seed(7)
    grad = torch.randn(out.shape, device="cuda", generator=g) * 0.1
    return r, ps, ids, grad


def _backward(r, grad, ids, reuse):
    lib = B.load()
    torch.cuda.synchronize()
    c0 = lib.dressi_launch_count()
    res = r.backward(grad, ids=ids, reuse_setup=reuse)
    torch.cuda.synchronize()
    return res, lib.dressi_launch_count() - c0


def _close(a, b):
    if a is None:
        return b is None
    # float atomics accumulate in any order: equal up to summation order, far inside
    # the gradient tolerance against the oracle (relative L2 1e-4)
    return (a - b).norm().item() <= 1e-6 * max(b.norm().item(), 1e-30)


@pytest.mark.parametrize("cfg,store", [("config1", True), ("config1", False), ("config2", True),
                                       ("config2", False)])
def test_reused_setup_gives_the_rebuilt_gradients(cfg, store):
    r, ps, ids, grad = _setup(cfg, store)
    reused, n_reused = _backward(r, grad, ids, None)
    rebuilt, n_rebuilt = _backward(r, grad, ids, False)
    assert r.device_status() == 0
    # the reusing call skipped the setup launches
    assert n_reused < n_rebuilt, (n_reused, n_rebuilt)
    for a, b in zip(reused, rebuilt):
        assert _close(a, b)


def test_changed_positions_rebuild_the_setup():
    r, ps, ids, grad = _setup("config1", False)
    _, n_full = _backward(r, grad, ids, False)
    r.forward(store_layers=False)
    # an in-place change of the positions after the forward: the backward must rebuild
    with torch.no_grad():
        ps.pos.mul_(1.01)
    after, n_after = _backward(r, grad, ids, None)
    assert n_after == n_full
    # and equals a backward that rebuilt on purpose for the new positions
    again, _ = _backward(r, grad, ids, False)
    for a, b in zip(after, again):
        assert _close(a, b)


def test_lists_survive_a_setup_without_them():
    """forward (lists) -> forward from the stored layers (setup without lists, same
    positions) -> re-rasterizing backward: the lists are still the forward's."""
    r, ps, ids, grad = _setup("config2", True)
    r.forward_from_layers(ids)
    reused, n_reused = _backward(r, grad, None, None)
    rebuilt, n_rebuilt = _backward(r, grad, None, False)
    assert n_reused < n_rebuilt
    for a, b in zip(reused, rebuilt):
        assert _close(a, b)
