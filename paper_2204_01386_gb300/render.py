"""Python face of libdressi: packed scenes, a renderer object and a
``torch.autograd.Function``.  PyTorch provides device memory and the stream;
all arithmetic runs in the library's kernels.

Layouts (as the C ABI wants them):
  positions / colours planar ``[3, V_total]`` float32, UVs ``[2, V_total]``,
  faces ``[F_total, 3]`` int32 (indices local to their mesh), textures packed
  ``[sum texels, 4]`` float32 or float16, images ``[n_pix, 4]`` float32 with the
  views stacked row-major one after another.
"""
from __future__ import annotations

import ctypes as C
import hashlib
import json
import os
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import binding as B


def _t(x, dtype, device):
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=dtype)
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=device)


class PackedScene:
    """Meshes packed into ragged device buffers (one vertex plane set, one face
    array, one texel buffer), plus the host-side mesh table."""

    def __init__(self, meshes: Sequence, device="cuda", tex_dtype: Optional[torch.dtype] = None):
        self.device = torch.device(device)
        pos, col, uv, faces, tex, ntex = [], [], [], [], [], []
        table = []
        vo = fo = to = 0
        has_col = all(getattr(m, "col", None) is not None for m in meshes)
        has_uv = all(getattr(m, "uv", None) is not None for m in meshes)
        has_tex = all(getattr(m, "tex", None) is not None for m in meshes)
        has_ntex = has_tex and all(getattr(m, "ntex", None) is not None for m in meshes)
        if tex_dtype is None and has_tex:
            t0 = meshes[0].tex
            tex_dtype = torch.float16 if (str(getattr(t0, "dtype", "")) in ("float16", "torch.float16")) else torch.float32
        self.tex_dtype = tex_dtype or torch.float32
        for m in meshes:
            p = _t(m.pos, torch.float32, self.device)
            f = _t(m.faces, torch.int32, self.device)
            pos.append(p.t())
            faces.append(f)
            if has_col:
                col.append(_t(m.col, torch.float32, self.device).t())
            if has_uv:
                uv.append(_t(m.uv, torch.float32, self.device).t())
            th = tw = 0
            if has_tex:
                tt = _t(m.tex, self.tex_dtype, self.device)
                th, tw = int(tt.shape[0]), int(tt.shape[1])
                tex.append(tt.reshape(-1, 4))
                if has_ntex:
                    nt = _t(m.ntex, self.tex_dtype, self.device)
                    assert tuple(nt.shape) == tuple(tt.shape), "the normal map is sized like the texture"
                    ntex.append(nt.reshape(-1, 4))
            table.append(B.DressiMesh(int(p.shape[0]), int(f.shape[0]), vo, fo, to, tw, th))
            vo += int(p.shape[0])
            fo += int(f.shape[0])
            to += th * tw
        self.n_verts_total = vo
        self.n_faces_total = fo
        self.n_texels = to
        self.pos = torch.cat(pos, 1).contiguous()
        self.faces = torch.cat(faces, 0).contiguous()
        self.col = torch.cat(col, 1).contiguous() if has_col else None
        self.uv = torch.cat(uv, 1).contiguous() if has_uv else None
        self.tex = torch.cat(tex, 0).contiguous() if has_tex else None
        self.ntex = torch.cat(ntex, 0).contiguous() if has_ntex else None
        self.table = (B.DressiMesh * len(table))(*table)
        self.n_meshes = len(table)

    def c_struct(self, pos=None, col=None, tex=None, ntex=None) -> B.DressiScene:
        """C view of the scene; ``pos``/``col``/``tex``/``ntex`` override the stored
        tensors (same shapes), e.g. with tensors that require grad."""
        pos = self.pos if pos is None else pos
        col = self.col if col is None else col
        tex = self.tex if tex is None else tex
        ntex = self.ntex if ntex is None else ntex
        for t in (pos, col, tex, ntex):
            if t is not None:
                assert t.is_cuda and t.is_contiguous()
        return B.DressiScene(self.n_meshes, C.cast(self.table, C.POINTER(B.DressiMesh)), self.n_verts_total,
                             pos.data_ptr(), col.data_ptr() if col is not None else None,
                             self.uv.data_ptr() if self.uv is not None else None, self.faces.data_ptr(),
                             tex.data_ptr() if tex is not None else None,
                             B.TEX_F16 if self.tex_dtype == torch.float16 else B.TEX_F32,
                             ntex.data_ptr() if ntex is not None else None)


def make_views(views: Sequence) -> "C.Array":
    """Host array of dressi_view from objects with mvp, light, mesh, width, height;
    views are stacked one after another in the image buffers."""
    arr = (B.DressiView * len(views))()
    off = 0
    for i, v in enumerate(views):
        a = arr[i]
        a.mvp[:] = [float(x) for x in np.asarray(v.mvp, np.float32).reshape(16)]
        a.light[:] = [float(x) for x in np.asarray(v.light, np.float32).reshape(3)]
        a.mesh, a.width, a.height, a.pix_off = int(v.mesh), int(v.width), int(v.height), off
        off += int(v.width) * int(v.height)
    return arr, off


def make_params(p, list_cap: int = 0, tile: int = 0, schedule: int = 0) -> B.DressiParams:
    jit = getattr(p, "uv_jitter", (0.0, 0.0))
    return B.DressiParams(int(p.K), float(p.r), float(p.sigma), float(p.delta), float(getattr(p, "gamma", 0.0)),
                          int(p.edge_mode), int(p.shade_mode), int(getattr(p, "texgrad_mode", 0)), int(tile),
                          int(schedule), int(list_cap), (C.c_float * 2)(float(jit[0]), float(jit[1])))


class Renderer:
    """Owns the workspace and status word for one (scene, views, params) set."""

    def __init__(self, scene: PackedScene, views: Sequence, params, list_cap: int = 0, tile: int = 0,
                 schedule: int = 0):
        self.lib = B.load()
        self.scene = scene
        self.views, self.n_pix = make_views(views)
        self.n_views = len(views)
        self.params = make_params(params, list_cap, tile, schedule)
        self.K = int(params.K)
        sc = scene.c_struct()
        self.ws_bytes = int(self.lib.dressi_workspace_size(C.byref(sc), self.views, self.n_views, C.byref(self.params)))
        if self.ws_bytes == 0:
            raise B.DressiError("dressi_workspace_size rejected the arguments")
        dev = scene.device
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        # what the workspace holds from the last setup: (key, tile lists built) or None
        self._setup = None

    def _setup_key(self, pos):
        """The inputs the setup (vertex transform, face table, normals, tile lists)
        depends on: the positions (storage and version), the parameters, the workspace."""
        t = self.scene.pos if pos is None else pos
        self.params.reuse_setup = 0
        return (t.data_ptr(), t._version, bytes(self.params), self.ws.data_ptr())

    def _setup_reusable(self, key, have_ids: bool) -> bool:
        """Whether the workspace holds the setup for ``key``, with the tile lists when
        the backward re-rasterizes (no stored layer ids)."""
        return self._setup is not None and self._setup[0] == key and (have_ids or self._setup[1])

    def _begin_setup(self):
        """Before a call that rebuilds the setup: the workspace holds nothing
        reusable until it returns."""
        old, self._setup = self._setup, None
        return old

    def _end_setup(self, old, key, bins: bool):
        # the tile lists survive a setup without them when the key is unchanged
        self._setup = (key, bins or (old is not None and old[0] == key and old[1]))

    def _stream(self):
        return C.c_void_p(torch.cuda.current_stream(self.scene.device).cuda_stream)

    def signature(self) -> str:
        """Key of this workload for the autotune cache: GPU, views, meshes, parameters."""
        p = self.params
        parts = [torch.cuda.get_device_name(self.scene.device), str(self.n_views)]
        parts += ["%d:%dx%d" % (v.mesh, v.width, v.height) for v in self.views]
        parts += ["%d/%d/%dx%d" % (m.n_verts, m.n_faces, m.tex_w, m.tex_h) for m in self.scene.table]
        parts += [str(x) for x in (p.K, p.r, p.sigma, p.delta, p.edge_mode, p.shade_mode, p.texgrad_mode)]
        return hashlib.sha1("|".join(parts).encode()).hexdigest()[:20]

    def autotune(self, cache_path: Optional[str] = None, store_layers: bool = True) -> dict:
        """Chooses tile edge, schedule and tile-list capacity by timing (dressi_autotune)
        forward + adjoint passes that keep the layer ids (``store_layers``) or
        re-rasterize, as the training loop will, remembering the choice per workload in
        a JSON file (``cache_path``, else $DRESSI_AUTOTUNE_CACHE, else
        ~/.cache/dressi/autotune.json)."""
        path = cache_path or os.environ.get("DRESSI_AUTOTUNE_CACHE") or os.path.join(
            os.path.expanduser("~"), ".cache", "dressi", "autotune.json")
        key = self.signature() + ("s" if store_layers else "r")
        cache = {}
        if os.path.exists(path):
            try:
                cache = json.load(open(path))
            except (OSError, ValueError):
                cache = {}
        choice = cache.get(key)
        if choice is None:
            dev = self.scene.device
            sc = self.scene.c_struct()
            need = 0
            for tile in (16, 32):
                for sched in (1, 2):
                    q = B.DressiParams.from_buffer_copy(self.params)
                    q.tile, q.schedule, q.list_cap = tile, sched, 0
                    need = max(need, int(self.lib.dressi_workspace_size(C.byref(sc), self.views, self.n_views,
                                                                       C.byref(q))))
            ws = torch.empty(need, dtype=torch.uint8, device=dev)
            out = torch.empty(self.n_pix, 4, dtype=torch.float32, device=dev)
            gp = torch.empty(3, self.scene.n_verts_total, dtype=torch.float32, device=dev)
            gc = torch.empty_like(gp) if self.scene.col is not None and self.params.shade_mode == 0 else None
            gt = (torch.empty(self.scene.n_texels, 4, dtype=torch.float32, device=dev)
                  if self.scene.tex is not None and self.params.shade_mode != 0 else None)
            q = B.DressiParams.from_buffer_copy(self.params)
            best = C.c_float(0.0)
            ids = torch.empty(self.K, self.n_pix, dtype=torch.int32, device=dev) if store_layers else None
            code = self.lib.dressi_autotune(C.byref(sc), self.views, self.n_views, C.byref(q), out.data_ptr(),
                                            ids.data_ptr() if ids is not None else None,
                                            self.n_pix, gp.data_ptr(), gc.data_ptr() if gc is not None else None,
                                            gt.data_ptr() if gt is not None else None, ws.data_ptr(), need,
                                            self.status.data_ptr(), self._stream(), C.byref(best))
            B.check(code, "dressi_autotune")
            choice = {"tile": int(q.tile), "schedule": int(q.schedule), "list_cap": int(q.list_cap),
                      "ms": float(best.value)}
            cache[key] = choice
            try:
                os.makedirs(os.path.dirname(path), exist_ok=True)
                tmp = path + ".%d.tmp" % os.getpid()
                json.dump(cache, open(tmp, "w"), indent=1)
                os.replace(tmp, path)
            except OSError:
                pass
            del ws
        self.params.tile, self.params.schedule, self.params.list_cap = choice["tile"], choice["schedule"], choice["list_cap"]
        sc = self.scene.c_struct()
        self.ws_bytes = int(self.lib.dressi_workspace_size(C.byref(sc), self.views, self.n_views, C.byref(self.params)))
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.scene.device)
        self._setup = None
        return dict(choice)

    def forward(self, store_layers: bool = True, out: Optional[torch.Tensor] = None,
                ids: Optional[torch.Tensor] = None, pos=None, col=None, tex=None,
                target: Optional[torch.Tensor] = None, grad: Optional[torch.Tensor] = None,
                loss: Optional[torch.Tensor] = None):
        """Renders ``out [n_pix, 4]`` (and the layer ids with ``store_layers``).  With
        ``target`` the L2 loss is fused in: ``grad`` receives 2 (out - target) and
        ``loss`` (if given) accumulates sum (out - target)^2; returns (out, ids, grad)."""
        dev = self.scene.device
        if out is None:
            out = torch.empty(self.n_pix, 4, dtype=torch.float32, device=dev)
        if store_layers and ids is None:
            ids = torch.empty(self.K, self.n_pix, dtype=torch.int32, device=dev)
        if not store_layers:
            ids = None
        sc = self.scene.c_struct(pos, col, tex)
        key = self._setup_key(pos)
        old = self._begin_setup()
        if target is not None:
            target = target.contiguous()
            if grad is None:
                grad = torch.empty_like(out)
            code = self.lib.dressi_forward_l2(C.byref(sc), self.views, self.n_views, C.byref(self.params),
                                              target.data_ptr(), out.data_ptr(), grad.data_ptr(),
                                              loss.data_ptr() if loss is not None else None,
                                              ids.data_ptr() if ids is not None else None, self.n_pix,
                                              self.ws.data_ptr(), self.ws_bytes, self.status.data_ptr(),
                                              self._stream())
            B.check(code, "dressi_forward_l2")
            self._end_setup(old, key, True)
            return out, ids, grad
        code = self.lib.dressi_forward(C.byref(sc), self.views, self.n_views, C.byref(self.params), out.data_ptr(),
                                       ids.data_ptr() if ids is not None else None, self.n_pix, self.ws.data_ptr(),
                                       self.ws_bytes, self.status.data_ptr(), self._stream())
        B.check(code, "dressi_forward")
        self._end_setup(old, key, True)
        return out, ids

    def forward_from_layers(self, ids: torch.Tensor, out: Optional[torch.Tensor] = None, pos=None, col=None,
                            tex=None):
        """Re-shades the layers ``ids`` stored by an earlier ``forward`` of the same
        geometry and views (skips binning, raster and peel); colours, textures, light
        and the blend parameters may have changed."""
        dev = self.scene.device
        if out is None:
            out = torch.empty(self.n_pix, 4, dtype=torch.float32, device=dev)
        sc = self.scene.c_struct(pos, col, tex)
        key = self._setup_key(pos)
        old = self._begin_setup()
        code = self.lib.dressi_forward_from_layers(C.byref(sc), self.views, self.n_views, C.byref(self.params),
                                                   ids.data_ptr(), out.data_ptr(), self.n_pix, self.ws.data_ptr(),
                                                   self.ws_bytes, self.status.data_ptr(), self._stream())
        B.check(code, "dressi_forward_from_layers")
        self._end_setup(old, key, False)
        return out

    def backward(self, grad_rgba: torch.Tensor, ids: Optional[torch.Tensor] = None, grad_pos=None, grad_col=None,
                 grad_tex=None, pos=None, col=None, tex=None, camera: bool = False, normal_map: bool = False,
                 grad_ntex=None, reuse_setup: Optional[bool] = None):
        """Adjoint of ``forward``: ``(grad_pos, grad_col, grad_tex)``, with ``camera``
        also ``grad_mvp [n_views, 16]`` and ``grad_light [n_views, 3]``, and with
        ``normal_map`` (shade_mode 3) the normal-map texel gradient last.

        ``reuse_setup``: None takes the setup (vertex transform, face table, normals,
        tile lists) the last ``forward`` left in the workspace when it was built from
        the same positions (same storage and version) and parameters, else rebuilds
        it; False always rebuilds."""
        dev = self.scene.device
        sc = self.scene.c_struct(pos, col, tex)
        grad_rgba = grad_rgba.contiguous()
        if grad_pos is None:
            grad_pos = torch.empty(3, self.scene.n_verts_total, dtype=torch.float32, device=dev)
        if grad_col is None and self.scene.col is not None and self.params.shade_mode == 0:
            grad_col = torch.empty(3, self.scene.n_verts_total, dtype=torch.float32, device=dev)
        if grad_tex is None and self.scene.tex is not None and self.params.shade_mode != 0:
            grad_tex = torch.empty(self.scene.n_texels, 4, dtype=torch.float32, device=dev)
        if normal_map and grad_ntex is None:
            grad_ntex = torch.empty(self.scene.n_texels, 4, dtype=torch.float32, device=dev)
        gm = torch.empty(self.n_views, 16, dtype=torch.float32, device=dev) if camera else None
        gl = torch.empty(self.n_views, 3, dtype=torch.float32, device=dev) if camera else None
        key = self._setup_key(pos)
        reuse = reuse_setup is not False and self._setup_reusable(key, ids is not None)
        self.params.reuse_setup = 1 if reuse else 0
        old = self._setup if reuse else self._begin_setup()
        code = self.lib.dressi_backward_ex(C.byref(sc), self.views, self.n_views, C.byref(self.params),
                                           grad_rgba.data_ptr(), ids.data_ptr() if ids is not None else None,
                                           self.n_pix, grad_pos.data_ptr(),
                                           grad_col.data_ptr() if grad_col is not None else None,
                                           grad_tex.data_ptr() if grad_tex is not None else None,
                                           gm.data_ptr() if gm is not None else None,
                                           gl.data_ptr() if gl is not None else None,
                                           grad_ntex.data_ptr() if normal_map else None,
                                           self.ws.data_ptr(), self.ws_bytes, self.status.data_ptr(), self._stream())
        self.params.reuse_setup = 0
        B.check(code, "dressi_backward_ex")
        if not reuse:
            self._end_setup(old, key, ids is None)
        res = (grad_pos, grad_col, grad_tex)
        if camera:
            res = res + (gm, gl)
        if normal_map:
            res = res + (grad_ntex,)
        return res

    def l2_grad(self, out: torch.Tensor, target: torch.Tensor, grad: Optional[torch.Tensor] = None,
                loss: Optional[torch.Tensor] = None):
        if grad is None:
            grad = torch.empty_like(out)
        code = self.lib.dressi_l2_loss_grad(out.data_ptr(), target.data_ptr(), out.numel(), grad.data_ptr(),
                                            loss.data_ptr() if loss is not None else None, self._stream())
        B.check(code, "dressi_l2_loss_grad")
        return grad

    def device_status(self) -> int:
        return int(self.status.item())

    def view_image(self, img: torch.Tensor, i: int) -> torch.Tensor:
        v = self.views[i]
        return img[v.pix_off: v.pix_off + v.width * v.height].view(v.height, v.width, -1)


def decode_layer_ids(ids):
    """Split stored layer ids into (face index, hard flag): -1 / False where a layer
    is empty; a soft fragment is stored with bit 31 set.  Works on torch tensors and
    numpy arrays of int32."""
    if isinstance(ids, torch.Tensor):
        empty = ids == -1
        face = torch.where(empty, torch.full_like(ids, -1), ids & 0x7FFFFFFF)
        return face, ids >= 0
    import numpy as np
    ids = np.asarray(ids, dtype=np.int32)
    empty = ids == -1
    face = np.where(empty, np.int32(-1), ids & np.int32(0x7FFFFFFF))
    return face, ids >= 0


class DressiFn(torch.autograd.Function):
    """out = HardSoftRas(pos, col, tex) for a fixed renderer (faces, UVs, views, params).

    ``pos`` [3, V_total] and ``col`` [3, V_total] planar float32 and ``tex``
    [texels, 4] as packed in the renderer's scene; returns ``[n_pix, 4]``.
    With ``store_layers`` the forward keeps the per-pixel layer ids for the
    backward, otherwise the backward re-rasterizes (checkpointing)."""

    @staticmethod
    def forward(ctx, pos, col, tex, renderer: Renderer, store_layers: bool = True):
        pos = pos.detach().contiguous()
        col = None if col is None else col.detach().contiguous()
        tex = None if tex is None else tex.detach().contiguous()
        out, ids = renderer.forward(store_layers=store_layers, pos=pos, col=col, tex=tex)
        ctx.renderer = renderer
        ctx.ids = ids
        ctx.save_for_backward(pos, col if col is not None else torch.empty(0), tex if tex is not None else torch.empty(0))
        ctx.has = (col is not None, tex is not None)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        pos, col, tex = ctx.saved_tensors
        col = col if ctx.has[0] else None
        tex = tex if ctx.has[1] else None
        gp, gc, gt = ctx.renderer.backward(grad_out, ids=ctx.ids, pos=pos, col=col, tex=tex)
        return gp, (gc if col is not None else None), (gt if tex is not None else None), None, None


def render(pos, col, tex, renderer: Renderer, store_layers: bool = True):
    return DressiFn.apply(pos, col, tex, renderer, store_layers)
