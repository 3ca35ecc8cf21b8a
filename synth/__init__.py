"""Seeded synthetic inputs shaped like the paper's benchmark workloads.

This module only makes inputs: meshes, per-vertex colours, UVs, textures,
cameras and soft-raster parameters.  It holds none of the renderer's
arithmetic (no projection to pixels, no coverage, no blending), so both the
CUDA path and the CPU oracle can be fed from it without sharing any code.

The paper benchmarks on its own meshes and cc0 textures (Tables in Sec. 5.1),
which are not available; seeded displaced spheres with random textures stand
in for them at the same triangle counts, window sizes and texture sizes.

Conventions (shared by every consumer):
  * positions ``pos`` float32 ``[V, 3]``, faces ``int32 [F, 3]``,
    colours float32 ``[V, 3]``, UVs float32 ``[V, 2]``;
  * textures ``[Ht, Wt, 4]`` (RGB plus a zero pad channel), float32 or float16;
  * ``mvp`` float32 row-major 4x4, column-vector convention
    ``clip = mvp @ (x, y, z, 1)``, Vulkan clip space (depth z/w in [0, 1],
    +y of NDC pointing down the image).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# ----------------------------------------------------------------------------
# random numbers
# ----------------------------------------------------------------------------

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea, Flood 2014) on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------

def _orient_outward(pos: np.ndarray, faces: np.ndarray) -> np.ndarray:
    """Flip faces whose winding points towards the origin (closed star-shaped meshes)."""
    p0, p1, p2 = pos[faces[:, 0]], pos[faces[:, 1]], pos[faces[:, 2]]
    n = np.cross(p1 - p0, p2 - p0)
    c = (p0 + p1 + p2) / 3.0
    flip = np.einsum("ij,ij->i", n, c) < 0
    out = faces.copy()
    out[flip, 1], out[flip, 2] = faces[flip, 2], faces[flip, 1]
    return out


def icosphere(subdiv: int):
    """Unit icosphere: 20 * 4**subdiv faces, 10 * 4**subdiv + 2 vertices."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    for _ in range(subdiv):
        nv = v.shape[0]
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        e.sort(axis=1)
        key = e[:, 0] * (nv + 1) + e[:, 1]
        uk, inv = np.unique(key, return_inverse=True)
        a, b = uk // (nv + 1), uk % (nv + 1)
        mid = v[a] + v[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.concatenate([v, mid], axis=0)
        nf = f.shape[0]
        m01, m12, m20 = (inv[:nf] + nv, inv[nf:2 * nf] + nv, inv[2 * nf:] + nv)
        f = np.concatenate([
            np.stack([f[:, 0], m01, m20], 1), np.stack([f[:, 1], m12, m01], 1),
            np.stack([f[:, 2], m20, m12], 1), np.stack([m01, m12, m20], 1)], axis=0)
    return v, _orient_outward(v, f).astype(np.int32)


def icosphere_uv(pos: np.ndarray, faces: np.ndarray):
    """Spherical UVs for an icosphere, seam-split: a face straddling u = 0/1
    gets duplicated corners with u + 1 (sampled with REPEAT wrap)."""
    d = pos / np.linalg.norm(pos, axis=1, keepdims=True)
    u = 0.5 + np.arctan2(d[:, 2], d[:, 0]) / (2 * math.pi)
    v = np.arccos(np.clip(d[:, 1], -1, 1)) / math.pi
    fu = u[faces]
    wrap = (fu.max(1) - fu.min(1)) > 0.5
    new_pos, new_u, new_v = [pos], [u], [v]
    faces = faces.copy()
    nxt = pos.shape[0]
    wf = np.nonzero(wrap)[0]
    if wf.size:
        corners = faces[wf]
        low = u[corners] < 0.5
        ci = np.nonzero(low)
        src = corners[ci]
        ids = np.arange(nxt, nxt + src.size)
        new_pos.append(pos[src])
        new_u.append(u[src] + 1.0)
        new_v.append(v[src])
        corners[ci] = ids
        faces[wf] = corners
    pos2 = np.concatenate(new_pos, 0)
    uv = np.stack([np.concatenate(new_u), np.concatenate(new_v)], 1)
    return pos2, faces.astype(np.int32), uv


def uv_sphere(slices: int, stacks: int):
    """UV sphere with ``stacks`` latitude bands and ``slices`` longitude bands.

    Seam and pole vertices are duplicated per slice so UVs are single valued;
    the pole bands hold one triangle per slice, so there are
    2 * slices * (stacks - 1) faces and (stacks + 1) * (slices + 1) vertices.
    """
    i = np.arange(stacks + 1)[:, None]
    j = np.arange(slices + 1)[None, :]
    th = math.pi * i / stacks
    ph = 2 * math.pi * j / slices
    x = np.sin(th) * np.cos(ph)
    y = np.cos(th) * np.ones_like(ph)
    z = np.sin(th) * np.sin(ph)
    pos = np.stack([x, y, z], -1).reshape(-1, 3)
    uv = np.stack([(j / slices) * np.ones_like(th), (i / stacks) * np.ones_like(ph)], -1).reshape(-1, 2)

    def vid(a, b):
        return a * (slices + 1) + b

    faces = []
    for a in range(stacks):
        for b in range(slices):
            v00, v01, v10, v11 = vid(a, b), vid(a, b + 1), vid(a + 1, b), vid(a + 1, b + 1)
            if a == 0:
                faces.append((v00, v11, v10))
            elif a == stacks - 1:
                faces.append((v00, v01, v10))
            else:
                faces.append((v00, v01, v11))
                faces.append((v00, v11, v10))
    faces = np.asarray(faces, dtype=np.int64)
    return pos, _orient_outward(pos, faces).astype(np.int32), uv


def value_noise(d: np.ndarray, seed: int, octaves: int = 3, base_freq: float = 2.0,
                lacunarity: float = 2.0, gain: float = 0.5) -> np.ndarray:
    """Seeded 3-D value noise in [-1, 1]: lattice values hashed from
    (i, j, k, seed), trilinear interpolation with smoothstep weights, summed
    over octaves and normalised by the total amplitude."""
    total = np.zeros(d.shape[0])
    amp, freq, norm = 1.0, base_freq, 0.0
    for o in range(octaves):
        p = d * freq
        f0 = np.floor(p)
        t = p - f0
        w = t * t * (3 - 2 * t)
        acc = np.zeros(d.shape[0])
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    c = (f0 + np.array([dx, dy, dz])).astype(np.int64)
                    with np.errstate(over="ignore"):
                        h = (c[:, 0].astype(np.uint64) * np.uint64(73856093)) ^ \
                            (c[:, 1].astype(np.uint64) * np.uint64(19349663)) ^ \
                            (c[:, 2].astype(np.uint64) * np.uint64(83492791)) ^ \
                            np.uint64((seed * 1000003 + o) & 0xFFFFFFFF)
                    h = _splitmix64(h)
                    val = (h >> np.uint64(11)).astype(np.float64) / float(1 << 53) * 2.0 - 1.0
                    wx = w[:, 0] if dx else 1 - w[:, 0]
                    wy = w[:, 1] if dy else 1 - w[:, 1]
                    wz = w[:, 2] if dz else 1 - w[:, 2]
                    acc += wx * wy * wz * val
        total += amp * acc
        norm += amp
        amp *= gain
        freq *= lacunarity
    return total / norm


def displace(pos: np.ndarray, amp: float, seed: int) -> np.ndarray:
    """Radius 1 + amp * noise(direction)."""
    d = pos / np.linalg.norm(pos, axis=1, keepdims=True)
    return d * (1.0 + amp * value_noise(d, seed))[:, None]


# ----------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------

def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)) -> np.ndarray:
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.asarray(up, np.float64)
    if abs(np.dot(f, up)) > 0.999:
        up = np.array([1.0, 0.0, 0.0])
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = s, u, -f
    m[0, 3], m[1, 3], m[2, 3] = -s @ eye, -u @ eye, f @ eye
    return m


def perspective(fovy_deg: float, aspect: float, near: float, far: float) -> np.ndarray:
    """Right-handed perspective into Vulkan clip space (depth in [0, 1], y down)."""
    t = 1.0 / math.tan(math.radians(fovy_deg) / 2)
    p = np.zeros((4, 4))
    p[0, 0] = t / aspect
    p[1, 1] = -t
    p[2, 2] = far / (near - far)
    p[2, 3] = near * far / (near - far)
    p[3, 2] = -1.0
    return p


def camera_mvp(eye, width: int, height: int, fovy=45.0, near=0.1, far=10.0) -> np.ndarray:
    m = perspective(fovy, width / height, near, far) @ look_at(eye)
    return m.astype(np.float32).reshape(16)


def fibonacci_dirs(n: int) -> np.ndarray:
    i = np.arange(n) + 0.5
    y = 1 - 2 * i / n
    r = np.sqrt(1 - y * y)
    phi = np.arange(n) * math.pi * (3 - math.sqrt(5))
    return np.stack([r * np.cos(phi), y, r * np.sin(phi)], 1)


LIGHT = (np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)).astype(np.float32)

# ----------------------------------------------------------------------------
# scene containers
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Mesh:
    pos: np.ndarray                    # float32 [V, 3]
    faces: np.ndarray                  # int32 [F, 3]
    col: Optional[np.ndarray] = None   # float32 [V, 3]
    uv: Optional[np.ndarray] = None    # float32 [V, 2]
    tex: Optional[np.ndarray] = None   # float32/float16 [Ht, Wt, 4]
    ntex: Optional[np.ndarray] = None  # tangent-space normal map, like tex (shade_mode 3)


@dataclasses.dataclass
class View:
    mvp: np.ndarray                    # float32 [16]
    mesh: int
    width: int
    height: int
    light: np.ndarray = dataclasses.field(default_factory=lambda: LIGHT.copy())


@dataclasses.dataclass
class Params:
    K: int = 3
    r: float = 0.01
    sigma: float = 0.01 / 7
    delta: float = 0.01
    gamma: float = 1e-4
    edge_mode: int = 0     # 0 edge mask, 1 blend everywhere (SoftRas-like), 2 hard only
    shade_mode: int = 0    # 0 vertex colour, 1 unlit texture, 2 Lambert texture
    texgrad_mode: int = 0  # 0 atomics, 1 texel-space gather
    store_layers: int = 1  # 1 keep per-pixel layer ids for the backward, 0 recompute


@dataclasses.dataclass
class Scene:
    name: str
    meshes: List[Mesh]
    views: List[View]
    params: Params

    @property
    def pixels(self) -> int:
        return sum(v.width * v.height for v in self.views)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _tex(g: np.random.Generator, side: int, dtype=np.float32) -> np.ndarray:
    t = np.zeros((side, side, 4), np.float32)
    t[..., :3] = g.random((side, side, 3), dtype=np.float32)
    return t.astype(dtype)


def soft_params_px(width: int, px: float = 2.0, K: int = 3, **kw) -> Params:
    """r = ``px`` pixels, sigma = r / 7, delta = r (the paper's defaults)."""
    r = px / width
    return Params(K=K, r=r, sigma=r / 7, delta=r, **kw)


def config1(seed: int = 1235, jitter_seed: int = 0) -> Scene:
    """Plain single view: icosphere 2x jittered, vertex colours, 64x64."""
    g = rng(seed)
    pos, faces = icosphere(2)
    jg = rng(seed * 7919 + jitter_seed)
    pos = pos + jg.uniform(-0.05, 0.05, pos.shape)
    col = g.random((pos.shape[0], 3))
    mesh = Mesh(_f32(pos), faces, col=_f32(col))
    view = View(camera_mvp((0, 0, 3), 64, 64), 0, 64, 64)
    p = Params(K=3, r=7e-4, sigma=1e-4, delta=7e-4, gamma=1e-4, edge_mode=0, shade_mode=0)
    return Scene("icosphere2_64px_vcol", [mesh], [view], p)


def _displaced_uv_sphere(slices, stacks, seed, amp=0.1):
    pos, faces, uv = uv_sphere(slices, stacks)
    return displace(pos, amp, seed), faces, uv


def config2(seed: int = 1236, texgrad_mode: int = 0) -> Scene:
    """Textured single view: 5,120-tri displaced UV sphere, 512^2 texture, Lambert, 256^2."""
    g = rng(seed)
    pos, faces, uv = _displaced_uv_sphere(64, 41, seed)
    mesh = Mesh(_f32(pos), faces, uv=_f32(uv), tex=_tex(g, 512))
    view = View(camera_mvp((0, 0, 3), 256, 256), 0, 256, 256)
    p = soft_params_px(256, shade_mode=2, texgrad_mode=texgrad_mode)
    return Scene("uvsphere5120_256px_lambert_tex512", [mesh], [view], p)


def normal_map(g, side: int, amp: float = 0.25) -> np.ndarray:
    """Tangent-space normal map [side, side, 4]: unit normals near +z (x, y smooth value
    noise of amplitude amp), encoded t = (n + 1) / 2 as in a normal-map image."""
    seed = int(g.integers(1 << 30))
    uu, vv = np.meshgrid((np.arange(side) + 0.5) / side, (np.arange(side) + 0.5) / side)
    pts = np.stack([np.cos(2 * np.pi * uu), np.sin(2 * np.pi * uu), 2 * vv - 1], -1).reshape(-1, 3)
    nx = amp * value_noise(pts * 3.0, seed)
    ny = amp * value_noise(pts * 3.0 + 17.0, seed + 1)
    nz = np.sqrt(np.maximum(1.0 - nx * nx - ny * ny, 0.0))
    t = np.zeros((side * side, 4), np.float32)
    t[:, 0], t[:, 1], t[:, 2] = (nx + 1) / 2, (ny + 1) / 2, (nz + 1) / 2
    return t.reshape(side, side, 4)


def config2n(seed: int = 1236) -> Scene:
    """config2 with a tangent-space normal map (shade_mode 3), 256^2 map and texture."""
    g = rng(seed)
    pos, faces, uv = _displaced_uv_sphere(64, 41, seed)
    mesh = Mesh(_f32(pos), faces, uv=_f32(uv), tex=_tex(g, 256), ntex=normal_map(g, 256))
    view = View(camera_mvp((0, 0, 3), 256, 256), 0, 256, 256)
    p = soft_params_px(256, shade_mode=3)
    return Scene("uvsphere5120_256px_normalmap256", [mesh], [view], p)


def config3(seed: int = 1237, n_views: int = 64, res: int = 512) -> Scene:
    """Batched multi-view: 20,480-tri displaced UV sphere, 1024^2 texture, 64 views of 512^2."""
    g = rng(seed)
    pos, faces, uv = _displaced_uv_sphere(128, 81, seed)
    mesh = Mesh(_f32(pos), faces, uv=_f32(uv), tex=_tex(g, 1024))
    views = [View(camera_mvp(3.0 * d, res, res), 0, res, res) for d in fibonacci_dirs(n_views)]
    p = soft_params_px(res, shade_mode=2)
    return Scene(f"uvsphere20480_{n_views}x{res}px_tex1024", [mesh], views, p)


def config4(seed: int = 1238, n_meshes: int = 32) -> Scene:
    """Ragged batch: meshes of 1k..200k tris (log-uniform), mixed resolutions and textures."""
    g = rng(seed)
    meshes, views = [], []
    for m in range(n_meshes):
        T = int(round(math.exp(g.uniform(math.log(1e3), math.log(2e5)))))
        bands = max(2, int(round(math.sqrt(T / 4))))
        slices = max(3, int(round(T / (2 * bands))))
        res = int(g.choice([128, 256, 512, 1024]))
        side = int(g.choice([512, 1024, 2048]))
        pos, faces, uv = _displaced_uv_sphere(slices, bands + 1, seed * 131 + m)
        meshes.append(Mesh(_f32(pos), faces, uv=_f32(uv), tex=_tex(g, side)))
        d = g.normal(size=3)
        d /= np.linalg.norm(d)
        views.append(View(camera_mvp(3.0 * d, res, res), m, res, res))
    # r = 2 px of each view's own resolution is not expressible with one
    # parameter set; use 2 px of 512 (the median resolution)
    p = soft_params_px(512, shade_mode=2)
    return Scene(f"ragged{n_meshes}", meshes, views, p)


def config5(seed: int = 1239, subdiv: int = 8, n_views: int = 8, res: int = 2048,
            tex_side: int = 4096, tex_dtype=np.float16) -> Scene:
    """Large: icosphere 8x displaced (1.31M tris), 4096^2 FP16 texture, 8 views at 2048^2."""
    g = rng(seed)
    pos, faces = icosphere(subdiv)
    pos = displace(pos, 0.1, seed)
    pos, faces, uv = icosphere_uv(pos, faces)
    mesh = Mesh(_f32(pos), faces, uv=_f32(uv), tex=_tex(g, tex_side, tex_dtype))
    views = [View(camera_mvp(3.0 * d, res, res), 0, res, res) for d in fibonacci_dirs(n_views)]
    p = soft_params_px(res, shade_mode=2, store_layers=0)
    return Scene(f"icosphere{subdiv}_{n_views}x{res}px_tex{tex_side}h", [mesh], views, p)


def perturbed(scene: Scene, seed: int, pos_jitter: float = 0.01, tex_jitter: float = 0.1) -> Scene:
    """Target scene: vertex jitter U[-pos_jitter, pos_jitter], texture (or colour)
    offset U[-tex_jitter, tex_jitter]; used to build the L2 loss target."""
    g = rng(seed)
    meshes = []
    for m in scene.meshes:
        pos = m.pos + g.uniform(-pos_jitter, pos_jitter, m.pos.shape).astype(np.float32)
        col = None if m.col is None else _f32(np.clip(m.col + g.uniform(-tex_jitter, tex_jitter, m.col.shape), 0, 1))
        tex = None
        if m.tex is not None:
            t = m.tex.astype(np.float32)
            t[..., :3] = np.clip(t[..., :3] + g.uniform(-tex_jitter, tex_jitter, t[..., :3].shape), 0, 1)
            tex = t.astype(m.tex.dtype)
        meshes.append(Mesh(_f32(pos), m.faces, col=col, uv=m.uv, tex=tex))
    return Scene(scene.name + "_target", meshes, scene.views, scene.params)


def config1_target(seed: int = 1235) -> Scene:
    """Config-1 target: the same icosphere with a second seeded jitter."""
    return config1(seed, jitter_seed=1)


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}
