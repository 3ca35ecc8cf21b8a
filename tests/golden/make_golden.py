"""Writes oracle_regression.json: outputs of the FP64 oracle on two tiny seeded scenes,
a regression fixture that catches an unintended change of the oracle's arithmetic.  It
is not a pin (the oracle is pinned against closed forms, brute force and finite
differences elsewhere), and the paper prints no worked example to store here.  Calls
only the oracle and the input generators.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
for p in (ROOT, os.path.dirname(HERE)):
    if p not in sys.path:
        sys.path.insert(0, p)

import oracle  # noqa: E402
import synth  # noqa: E402
from scenes_small import pixel_mesh, pixel_scene  # noqa: E402


def scenes():
    """(name, scene, window) of the fixture: two overlapping vertex-coloured triangles at
    16 x 16 px, and a 16 x 16 window of the 64 x 64 jittered icosphere."""
    V = [(2.0, 3.0), (13.5, 4.0), (6.0, 14.0), (4.0, 2.0), (15.0, 12.0), (1.5, 10.5)]
    F = [(0, 1, 2), (3, 4, 5)]
    col = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (0, 1, 1), (1, 0, 1)]
    m = pixel_mesh(V, F, 16, 16, z=[0.3, 0.4, 0.5, 0.6, 0.2, 0.45], col=col)
    tri = pixel_scene(m, 16, 16, K=2, r=1.5 / 16, sigma=0.3 / 16, delta=1 / 16, edge_mode=0, shade_mode=0)
    return [("two_triangles_16px", tri, None), ("icosphere_64px_window", synth.config1(), (24, 24, 16, 16))]


def compute(scene, window):
    m, v, p = scene.meshes[0], scene.views[0], scene.params
    o = oracle.render(m, v, p, window=window)
    h, w = o["rgba"].shape[:2]
    g = np.random.default_rng(7).normal(size=(h, w, 4))
    gp, gc, _ = oracle.backward(m, v, p, g, window=window)
    return {"rgba": o["rgba"].tolist(), "ids": o["ids"].tolist(), "sh": o["sh"].tolist(),
            "edge": o["edge"].tolist(), "grad_pos": gp.tolist(), "grad_col": gc.tolist()}


def main():
    out = {"note": "FP64 oracle outputs (regression fixture, not a pin); written by make_golden.py",
           "cases": {name: compute(s, win) for name, s, win in scenes()}}
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=None, separators=(",", ":"))


if __name__ == "__main__":
    main()
