"""The torch.autograd.Function wrapper (DressiFn / render): its forward is the
library's forward, and loss.backward() hands PyTorch exactly the gradients of the
library's adjoint (which the parity tests check against the FP64 oracle), with stored
layer ids and with the re-rasterizing adjoint."""
import pytest
import torch

import synth
from paper_2204_01386_gb300 import PackedScene, Renderer, render

pytestmark = pytest.mark.gpu


def _target(scene, seed, **kw):
    t = synth.perturbed(scene, seed, **kw)
    ps = PackedScene(t.meshes, "cuda")
    out, _ = Renderer(ps, t.views, t.params).forward(store_layers=False)
    return out


@pytest.mark.parametrize("store_layers", [True, False])
@pytest.mark.parametrize("cfg", ["config1", "config2"])
def test_autograd_matches_library_adjoint(cfg, store_layers):
    s = getattr(synth, cfg)()
    target = _target(s, 5)
    ps = PackedScene(s.meshes, "cuda")
    r = Renderer(ps, s.views, s.params)

    pos = ps.pos.clone().requires_grad_()
    col = None if ps.col is None else ps.col.clone().requires_grad_()
    tex = None if ps.tex is None else ps.tex.clone().requires_grad_()
    img = render(pos, col, tex, r, store_layers)
    loss = (img - target).square().sum()
    loss.backward()

    # the same step through the Renderer directly
    ref, ids = r.forward(store_layers=True)
    assert torch.equal(img.detach(), ref)
    g = 2.0 * (ref - target)
    gp, gc, gt = r.backward(g, ids=ids if store_layers else None)
    torch.cuda.synchronize()
    assert r.device_status() == 0
    # float atomics sum in any order: equal up to summation order
    assert torch.allclose(pos.grad, gp, rtol=1e-5, atol=1e-6 * gp.abs().max().item())
    assert pos.grad.abs().max().item() > 0
    if col is not None:
        assert torch.allclose(col.grad, gc, rtol=1e-5, atol=1e-6 * gc.abs().max().item())
        assert col.grad.abs().max().item() > 0
    if tex is not None:
        assert torch.allclose(tex.grad, gt, rtol=1e-5, atol=1e-6 * gt.abs().max().item())
        assert tex.grad.abs().max().item() > 0


def test_autograd_gradient_descent_reduces_the_loss():
    """A few texture steps of plain gradient descent through render() lower the image
    loss against a target rendered from a perturbed texture (the paper's texture
    optimisation task in miniature)."""
    s = synth.config2()
    target = _target(s, 7, pos_jitter=0.0)   # the texture alone differs
    ps = PackedScene(s.meshes, "cuda")
    r = Renderer(ps, s.views, s.params)
    tex = ps.tex.clone().requires_grad_()
    losses = []
    for _ in range(5):
        img = render(ps.pos, None, tex, r)
        loss = (img - target).square().sum()
        losses.append(loss.item())
        tex.grad = None
        loss.backward()
        with torch.no_grad():
            tex -= 1.0 * tex.grad
    assert losses[-1] < 0.9 * losses[0], losses
