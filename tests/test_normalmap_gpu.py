"""Lambert with a tangent-space normal map (shade_mode 3; the shading of the paper's
normal-map optimisation) against the FP64 oracle: forward within 1e-5, gradients of
positions, albedo texels, normal-map texels, camera and light within 1e-4 relative L2,
with and without stored layers, and re-shading from stored layers."""
import pytest
import torch

import synth
from paper_2204_01386_gb300 import PackedScene, Renderer
from parity import compare_scene

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tile,schedule", [(0, 0), (32, 2)])
@pytest.mark.parametrize("store_layers", [True, False])
def test_normal_map_parity(store_layers, tile, schedule):
    # the library's default execution choice, and 32 px tiles with persistent CTAs in
    # longest-first order (the kernels with the normal map compiled in)
    st = compare_scene(synth.config2n(), store_layers=store_layers, camera=True, tile=tile, schedule=schedule)
    assert {"pos0", "tex0", "ntex0", "mvp0", "light0"} <= set(st["grad_err"]), st["grad_err"]


def test_normal_map_edge_modes():
    s = synth.config2n()
    s.params.edge_mode = 1
    st = compare_scene(s)
    assert "ntex0" in st["grad_err"]


def test_normal_map_reshading_from_layers():
    s = synth.config2n()
    ps = PackedScene(s.meshes, "cuda")
    r = Renderer(ps, s.views, s.params)
    out, ids = r.forward(store_layers=True)
    again = r.forward_from_layers(ids)
    torch.cuda.synchronize()
    assert torch.equal(out, again)
