"""Tiny hand-built scenes for closed-form checks (inputs only, no method arithmetic).

Meshes are given directly in pixel coordinates and mapped to object space
with an identity MVP (w = 1), so that the pixel-space corner positions are
exact binary fractions.
"""
import numpy as np

import synth


def identity_mvp():
    return np.eye(4, dtype=np.float32).reshape(16)


def pixel_mesh(verts_px, faces, width, height, z=0.5, col=None, uv=None, tex=None):
    """Object coordinates x = 2X/W - 1, y = 2Y/H - 1 so that the identity MVP
    puts corner (X, Y) exactly at pixel position (X, Y)."""
    v = np.asarray(verts_px, np.float64)
    zz = np.broadcast_to(np.asarray(z, np.float64), (v.shape[0],))
    pos = np.stack([2 * v[:, 0] / width - 1, 2 * v[:, 1] / height - 1, zz], 1).astype(np.float32)
    if col is None:
        col = np.ones((v.shape[0], 3), np.float32)
    return synth.Mesh(pos, np.asarray(faces, np.int32), col=np.asarray(col, np.float32),
                      uv=None if uv is None else np.asarray(uv, np.float32), tex=tex)


def pixel_scene(mesh, width, height, **params):
    view = synth.View(identity_mvp(), 0, width, height)
    p = synth.Params(**params)
    return synth.Scene("pixel", [mesh], [view], p)


def grid_mesh(n, width, height, jitter=0.0, seed=0, z=0.5):
    """Screen-filling planar triangulation of [-1, W+1] x [-1, H+1] with an
    n x n vertex grid; interior vertices optionally jittered."""
    g = np.random.default_rng(seed)
    xs = np.linspace(-1, width + 1, n)
    ys = np.linspace(-1, height + 1, n)
    X, Y = np.meshgrid(xs, ys)
    V = np.stack([X.ravel(), Y.ravel()], 1)
    if jitter:
        inner = (X.ravel() > -1) & (X.ravel() < width + 1) & (Y.ravel() > -1) & (Y.ravel() < height + 1)
        V[inner] += g.uniform(-jitter, jitter, (inner.sum(), 2))
    F = []
    for i in range(n - 1):
        for j in range(n - 1):
            a, b, c, d = i * n + j, i * n + j + 1, (i + 1) * n + j, (i + 1) * n + j + 1
            F += [(a, b, d), (a, d, c)]
    return V, np.asarray(F, np.int32)
