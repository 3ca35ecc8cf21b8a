"""The forward with the L2 loss fused in (dressi_forward_l2) equals the forward followed
by the separate loss kernel: image and gradient bit for bit, the loss up to summation
order."""
import pytest
import torch

import synth
from paper_2204_01386_gb300 import PackedScene, Renderer

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scene,store", [(lambda: synth.config1(), True), (lambda: synth.config2(), False),
                                         (lambda: synth.config3(n_views=4, res=96), True)])
def test_fused_loss_matches_separate_kernel(scene, store):
    s = scene()
    ps = PackedScene(s.meshes, "cuda")
    r = Renderer(ps, s.views, s.params)
    g = torch.Generator(device="cuda").manual_seed(3)
    target = torch.rand(r.n_pix, 4, device="cuda", generator=g)
    out0, ids0 = r.forward(store_layers=store)
    loss0 = torch.zeros(1, device="cuda")
    grad0 = r.l2_grad(out0, target, loss=loss0)
    loss1 = torch.zeros(1, device="cuda")
    out1, ids1, grad1 = r.forward(store_layers=store, target=target, loss=loss1)
    torch.cuda.synchronize()
    assert r.device_status() == 0
    assert torch.equal(out0, out1)
    assert torch.equal(grad0, grad1)
    if store:
        assert torch.equal(ids0, ids1)
    ref = ((out0.double() - target.double()) ** 2).sum().item()
    assert abs(loss1.item() - ref) <= 1e-5 * ref
    assert abs(loss0.item() - ref) <= 1e-5 * ref
