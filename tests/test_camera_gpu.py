"""Gradients of the camera matrix and the light (theta_C and theta_L of the parameter
set of Sec. 3.4.1) through dressi_backward_ex, against the FP64 oracle (relative L2
<= 1e-4 per view, on a pixel gradient that is zero where a discrete decision lacks
margin), next to the usual position / colour / texel gradients."""
import pytest

import synth
from parity import compare_scene

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("store_layers", [True, False])
def test_camera_gradient_vertex_colour(store_layers):
    st = compare_scene(synth.config1(), store_layers=store_layers, camera=True)
    assert "mvp0" in st["grad_err"]


@pytest.mark.parametrize("tile,schedule", [(0, 0), (32, 2)])
@pytest.mark.parametrize("store_layers", [True, False])
def test_camera_and_light_gradient_lambert(store_layers, tile, schedule):
    st = compare_scene(synth.config2(), store_layers=store_layers, camera=True, tile=tile, schedule=schedule)
    assert "mvp0" in st["grad_err"] and "light0" in st["grad_err"]


def test_camera_and_light_gradient_many_views():
    """64 views of 512^2 in one call; two views checked on crops (dL/dI zero elsewhere),
    the others must come out zero."""
    s = synth.config3()
    wins = [(232, 200, 48, 48) if i in (0, 37) else (0, 0, 0, 0) for i in range(len(s.views))]
    st = compare_scene(s, windows=wins, camera=True)
    assert {"mvp0", "mvp37", "light0", "light37"} <= set(st["grad_err"]), st["grad_err"]
