"""FP64 CPU oracle for HardSoftRas -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product (``paper_2204_01386_gb300``) never
does, and this package imports nothing from it.  The arithmetic lives in
``hardsoftras_oracle.c`` (plain C, FP64, brute force); this file only
marshals numpy arrays into it.

Inputs are taken as the float32 (or float16) values the CUDA path receives and
widened exactly to float64, so the oracle evaluates the exact function of the
very same inputs.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hardsoftras_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _View(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_faces", C.c_int32),
                ("pos", C.POINTER(C.c_double)), ("col", C.POINTER(C.c_double)),
                ("uv", C.POINTER(C.c_double)), ("faces", C.POINTER(C.c_int32)),
                ("tex_w", C.c_int32), ("tex_h", C.c_int32), ("tex", C.POINTER(C.c_double)),
                ("mvp", C.c_double * 16), ("light", C.c_double * 3),
                ("width", C.c_int32), ("height", C.c_int32), ("ntex", C.POINTER(C.c_double))]


class _Params(C.Structure):
    _fields_ = [("K", C.c_int32), ("r", C.c_double), ("sigma", C.c_double), ("delta", C.c_double),
                ("edge_mode", C.c_int32), ("shade_mode", C.c_int32), ("brute_force", C.c_int32)]


class _Window(C.Structure):
    _fields_ = [("x0", C.c_int32), ("y0", C.c_int32), ("w", C.c_int32), ("h", C.c_int32)]


class _InvUV(C.Structure):
    """Inverse-UV records (Sec. 3.3.2, Alg. 1); see orc_inv_uv."""
    _fields_ = [("jitter", C.c_double * 2), ("pix_base", C.c_int64), ("cap", C.c_int64), ("n", C.c_int64),
                ("slot", C.POINTER(C.c_int64)), ("texel", C.POINTER(C.c_int32)), ("m_tex", C.POINTER(C.c_double)),
                ("m_cand", C.POINTER(C.c_double)), ("gA", C.POINTER(C.c_double))]


class _FwdOut(C.Structure):
    _fields_ = [("rgba", C.POINTER(C.c_double)), ("ids", C.POINTER(C.c_int32)),
                ("hard", C.POINTER(C.c_int32)), ("dist", C.POINTER(C.c_double)),
                ("key", C.POINTER(C.c_double)), ("sh", C.POINTER(C.c_uint8)),
                ("edge", C.POINTER(C.c_uint8)), ("margin_hard", C.POINTER(C.c_double)),
                ("margin_cand", C.POINTER(C.c_double)), ("n_hard", C.POINTER(C.c_int32)),
                ("feat_hash", C.POINTER(C.c_uint64))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            assert lib.orc_sizeof_view() == C.sizeof(_View)
            assert lib.orc_sizeof_params() == C.sizeof(_Params)
            assert lib.orc_sizeof_fwd_out() == C.sizeof(_FwdOut)
            lib.orc_forward.argtypes = [C.POINTER(_View), C.POINTER(_Params), C.POINTER(_Window), C.POINTER(_FwdOut)]
            lib.orc_backward.argtypes = [C.POINTER(_View), C.POINTER(_Params), C.POINTER(_Window),
                                         C.POINTER(C.c_double), C.POINTER(C.c_double),
                                         C.POINTER(C.c_double), C.POINTER(C.c_double)]
            lib.orc_backward_ex.argtypes = [C.POINTER(_View), C.POINTER(_Params), C.POINTER(_Window),
                                            C.POINTER(C.c_double), C.POINTER(C.c_double),
                                            C.POINTER(C.c_double), C.POINTER(C.c_double),
                                            C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(_InvUV),
                                            C.POINTER(C.c_double)]
            _lib = lib
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_int32))


def _up(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_uint8))


def _f64(a):
    return None if a is None else np.ascontiguousarray(np.asarray(a).astype(np.float64))


class _Inputs:
    """Keeps the float64 copies alive while the C call runs."""

    def __init__(self, mesh, view, params, brute_force):
        self.pos = _f64(mesh.pos)
        self.col = _f64(getattr(mesh, "col", None))
        self.uv = _f64(getattr(mesh, "uv", None))
        self.faces = np.ascontiguousarray(np.asarray(mesh.faces, dtype=np.int32))
        tex = getattr(mesh, "tex", None)
        self.tex = _f64(tex)
        self.ntex = _f64(getattr(mesh, "ntex", None))
        v = _View()
        v.n_verts, v.n_faces = self.pos.shape[0], self.faces.shape[0]
        v.pos, v.col, v.uv = _dp(self.pos), _dp(self.col), _dp(self.uv)
        v.faces = _ip(self.faces)
        if self.tex is not None:
            v.tex_h, v.tex_w = self.tex.shape[0], self.tex.shape[1]
            v.tex = _dp(self.tex)
        v.mvp[:] = [float(x) for x in np.asarray(view.mvp, np.float64).reshape(16)]
        v.light[:] = [float(x) for x in np.asarray(view.light, np.float64).reshape(3)]
        v.width, v.height = int(view.width), int(view.height)
        v.ntex = _dp(self.ntex)
        self.view = v
        p = _Params()
        # the soft-raster parameters reach the CUDA path as float32: use the same values
        f32 = lambda x: float(np.float32(x))  # noqa: E731
        p.K, p.r, p.sigma, p.delta = int(params.K), f32(params.r), f32(params.sigma), f32(params.delta)
        p.edge_mode, p.shade_mode = int(params.edge_mode), int(params.shade_mode)
        p.brute_force = int(bool(brute_force))
        self.params = p


def _window(view, window):
    w = _Window()
    if window is None:
        window = (0, 0, int(view.width), int(view.height))
    w.x0, w.y0, w.w, w.h = [int(x) for x in window]
    return w


def render(mesh, view, params, window=None, brute_force=False):
    """Forward pass of one view over ``window`` = (x0, y0, w, h) pixels.

    Returns a dict with ``rgba [h,w,4]``, ``ids``/``hard``/``dist`` ``[K,h,w]``,
    ``key [K+1,h,w]``, ``sh``/``edge [h,w]``, ``margin_hard``/``margin_cand``
    (pixel units), ``n_hard``, ``feat_hash [K+1,h,w]`` (identity of each
    fragment's closest feature) plus the oracle's status word.
    """
    lib = _load()
    inp = _Inputs(mesh, view, params, brute_force)
    win = _window(view, window)
    K, h, w = inp.params.K, win.h, win.w
    res = dict(rgba=np.zeros((h, w, 4)), ids=np.zeros((K, h, w), np.int32),
               hard=np.zeros((K, h, w), np.int32), dist=np.zeros((K, h, w)),
               key=np.zeros((K + 1, h, w)), sh=np.zeros((h, w), np.uint8),
               edge=np.zeros((h, w), np.uint8), margin_hard=np.zeros((h, w)),
               margin_cand=np.zeros((h, w)), n_hard=np.zeros((h, w), np.int32),
               feat_hash=np.zeros((K + 1, h, w), np.uint64))
    o = _FwdOut(_dp(res["rgba"]), _ip(res["ids"]), _ip(res["hard"]), _dp(res["dist"]),
                _dp(res["key"]), _up(res["sh"]), _up(res["edge"]), _dp(res["margin_hard"]),
                _dp(res["margin_cand"]), _ip(res["n_hard"]),
                res["feat_hash"].ctypes.data_as(C.POINTER(C.c_uint64)))
    st = lib.orc_forward(C.byref(inp.view), C.byref(inp.params), C.byref(win), C.byref(o))
    if st & 1:
        raise ValueError("oracle: invalid argument")
    res["status"] = st
    return res


def backward(mesh, view, params, grad_rgba, window=None, brute_force=False, camera=False, inverse_uv=None,
             want_ntex=False):
    """Adjoint of ``render`` for dL/d(rgba) = ``grad_rgba [h,w,4]`` over ``window``.

    Returns ``(grad_pos [V,3], grad_col [V,3] or None, grad_tex [Ht,Wt,4] or None)``,
    and with ``camera`` also ``grad_mvp [16]`` (row-major, as ``view.mvp``) and
    ``grad_light [3]`` (Sec. 3.4.1: the camera and light parameters of Theta).
    With ``want_ntex`` the normal-map texel gradient ``[Ht,Wt,4]`` (shade_mode 3) follows.
    With ``inverse_uv = (jitter, pix_base)`` the texel gradient is not accumulated and
    the inverse-UV writes of the window's samples are returned last, as a dict of
    arrays (see ``inverse_uv_texels``).
    """
    lib = _load()
    inp = _Inputs(mesh, view, params, brute_force)
    win = _window(view, window)
    g = np.ascontiguousarray(np.asarray(grad_rgba, np.float64).reshape(win.h, win.w, 4))
    gp = np.zeros_like(inp.pos)
    gc = np.zeros_like(inp.pos) if inp.col is not None else None
    gt = np.zeros_like(inp.tex) if inp.tex is not None and inverse_uv is None else None
    gm = np.zeros(16) if camera else None
    gl = np.zeros(3) if camera else None
    gnt = np.zeros_like(inp.ntex) if (want_ntex and inp.ntex is not None) else None
    inv, rec = None, None
    if inverse_uv is not None:
        cap = win.w * win.h * params.K
        rec = dict(slot=np.zeros(cap, np.int64), texel=np.zeros(cap, np.int32), m_tex=np.zeros(cap),
                   m_cand=np.zeros(cap), gA=np.zeros((cap, 3)))
        inv = _InvUV()
        inv.jitter[0], inv.jitter[1] = float(inverse_uv[0][0]), float(inverse_uv[0][1])
        inv.pix_base, inv.cap, inv.n = int(inverse_uv[1]), cap, 0
        inv.slot = rec["slot"].ctypes.data_as(C.POINTER(C.c_int64))
        inv.texel = _ip(rec["texel"])
        inv.m_tex, inv.m_cand, inv.gA = _dp(rec["m_tex"]), _dp(rec["m_cand"]), _dp(rec["gA"])
    st = lib.orc_backward_ex(C.byref(inp.view), C.byref(inp.params), C.byref(win), _dp(g), _dp(gp), _dp(gc),
                             _dp(gt), _dp(gm), _dp(gl), C.byref(inv) if inv is not None else None, _dp(gnt))
    if st & 1:
        raise ValueError("oracle: invalid argument")
    out = (gp, gc, gt, gm, gl) if camera else (gp, gc, gt)
    if want_ntex:
        out = out + (gnt,)
    if rec is not None:
        rec = {k: v[:inv.n] for k, v in rec.items()}
        out = out + (rec,)
    return out


def inverse_uv_texels(records, tex_w, tex_h, tau_tex=1e-4, tau_px=1e-4):
    """Resolves inverse-UV writes (records of one or more views, any order) into the
    texel gradient of Alg. 1: each texel takes the dL/d(albedo) of its last writer,
    the largest sample number.  Returns ``(grad [n_texels, 3], winner [n_texels]
    (-1: none), stable [n_texels])``.  A texel is unstable when a write whose discrete
    decisions lie within the margins could land on it: a texel floor within ``tau_tex``
    of an edge (the 3 x 3 texels around it, with REPEAT wrap) or a candidate test
    within ``tau_px`` of dist = -r (its texel)."""
    n_texels = tex_w * tex_h
    cat = (lambda k, empty: np.concatenate([r[k] for r in records]) if records else empty)
    slot, texel = cat("slot", np.zeros(0, np.int64)), cat("texel", np.zeros(0, np.int32))
    m_tex, m_cand, gA = cat("m_tex", np.zeros(0)), cat("m_cand", np.zeros(0)), cat("gA", np.zeros((0, 3)))
    winner = np.full(n_texels, -1, np.int64)
    np.maximum.at(winner, texel, slot)
    grad = np.zeros((n_texels, 3))
    row_of = dict(zip(slot.tolist(), range(len(slot))))
    for t in np.nonzero(winner >= 0)[0]:
        grad[t] = gA[row_of[int(winner[t])]]
    stable = np.ones(n_texels, bool)
    stable[texel[m_cand < tau_px]] = False
    for t in texel[m_tex < tau_tex]:
        ty, tx = divmod(int(t), tex_w)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                stable[((ty + dy) % tex_h) * tex_w + (tx + dx) % tex_w] = False
    return grad, winner, stable
