"""Helpers that run the CUDA path (through the C ABI) and the FP64 oracle on the
same seeded scene and compare them.

Tolerances:
  * layer ids: bit-exact on every pixel whose discrete decisions have margin:
    every face within r of the pixel is >= TAU_PX pixels from its hard/soft
    boundary and from the candidate boundary dist = -r, and consecutive keys of
    the K+1 best fragments differ by >= TAU_KEY, or by exactly 0 with the same
    closest feature (a shared edge or corner, broken by face id on both sides);
  * forward rgba: max-abs <= 1e-5 on pixels that are stable and whose edge-mask
    window holds only stable S^H pixels, or, where the oracle's own image moves by
    more when its float32 positions and UVs move one ulp (large textures on faces
    spanning many texels), within twice that spread (the FP32 floor);
  * gradients: relative L2 <= 1e-4 for dL/d(rgba) that is zero on unstable pixels.
"""
import numpy as np
import torch
from scipy import ndimage

import oracle
from paper_2204_01386_gb300 import PackedScene, Renderer, decode_layer_ids

TAU_PX = 1e-4
TAU_KEY = 1e-6
FWD_TOL = 1e-5
GRAD_TOL = 1e-4


def rho_of(params, view):
    S = max(view.width, view.height)
    return max(1, int(np.floor(params.delta * S + 0.5)))


def masks(o, params, view):
    """(stable_ids, stable_values) boolean [h, w] from the oracle's margins."""
    keys = o["key"]
    gaps = np.diff(keys, axis=0)
    fh = o["feat_hash"]
    same_feature = fh[1:] == fh[:-1]
    with np.errstate(invalid="ignore"):
        # an exact tie of one shared edge / corner is computed identically on both sides;
        # a tie (or near tie) of distinct features is decided by rounding
        key_bad = ((gaps < TAU_KEY) & ~((gaps == 0) & same_feature)).any(0)
    unstable = (o["margin_hard"] < TAU_PX) | (o["margin_cand"] < TAU_PX) | key_bad
    sh_bad = o["margin_hard"] < TAU_PX
    if params.edge_mode == 0:
        r = rho_of(params, view)
        sh_bad = ndimage.binary_dilation(sh_bad, structure=np.ones((2 * r + 1, 2 * r + 1), bool))
    return ~unstable, ~(unstable | sh_bad)


class CudaPath:
    """The CUDA path of one scene; ``tile`` (16, 32; 0 = library default) and ``schedule``
    (1 one CTA per tile, 2 persistent CTAs over the longest-first tile order; 0 = library
    default) choose the per-tile kernel that runs."""

    def __init__(self, scene, device="cuda", list_cap=0, tile=0, schedule=0):
        self.scene = scene
        self.ps = PackedScene(scene.meshes, device)
        self.r = Renderer(self.ps, scene.views, scene.params, list_cap=list_cap, tile=tile, schedule=schedule)

    def forward(self, store_layers=True):
        # layer ids are always kept here so they can be compared; whether the
        # backward re-rasterizes is chosen in backward()
        out, ids = self.r.forward(store_layers=True)
        if not store_layers:
            # then the pass a checkpointed step runs: no layer ids, each pixel's K-th
            # (key, id) kept in the workspace, where the re-rasterizing adjoint (which takes
            # this setup) starts its K-lists from them
            out2, _ = self.r.forward(store_layers=False)
            assert torch.equal(out, out2)
        torch.cuda.synchronize()
        self.out, self.ids = out, ids
        return out, ids

    def view_rgba(self, i):
        return self.r.view_image(self.out, i).cpu().numpy().astype(np.float64)

    def view_raw_ids(self, i):
        v = self.r.views[i]
        return self.ids[:, v.pix_off: v.pix_off + v.width * v.height].view(-1, v.height, v.width).cpu().numpy()

    def view_ids(self, i):
        """Face index of each layer, -1 where empty."""
        return decode_layer_ids(self.view_raw_ids(i))[0]

    def view_hard(self, i):
        """Hard flag of each layer (False where empty)."""
        return decode_layer_ids(self.view_raw_ids(i))[1]

    def backward(self, grads_per_view, use_ids=True, camera=False):
        """Per-mesh gradients; with ``camera`` also the per-view dL/dMVP [n_views, 16]
        and dL/dlight [n_views, 3] as numpy arrays."""
        g = torch.zeros(self.r.n_pix, 4, dtype=torch.float32, device=self.ps.device)
        for i, gv in enumerate(grads_per_view):
            v = self.r.views[i]
            g[v.pix_off: v.pix_off + v.width * v.height] = torch.as_tensor(
                np.asarray(gv, np.float32).reshape(-1, 4), device=self.ps.device)
        nmap = self.scene.params.shade_mode == 3
        res = self.r.backward(g, ids=self.ids if use_ids else None, camera=camera, normal_map=nmap)
        torch.cuda.synchronize()
        per_mesh = self.split(*res[:3], gnt=res[-1] if nmap else None)
        if camera:
            return per_mesh, res[3].cpu().numpy().astype(np.float64), res[4].cpu().numpy().astype(np.float64)
        return per_mesh

    def split(self, gp, gc, gt, gnt=None):
        """Per-mesh numpy gradients [V,3], [V,3] or None, [Ht,Wt,4] or None, and the
        normal-map gradient [Ht,Wt,4] or None."""
        res = []
        for m, t in zip(self.scene.meshes, self.ps.table):
            a, n = t.vert_off, t.n_verts
            p = gp[:, a:a + n].t().cpu().numpy().astype(np.float64)
            c = gc[:, a:a + n].t().cpu().numpy().astype(np.float64) if gc is not None else None
            texels = lambda q: q[t.tex_off: t.tex_off + t.tex_w * t.tex_h].view(t.tex_h, t.tex_w, 4).cpu().numpy().astype(np.float64)
            x = texels(gt) if gt is not None else None
            nx = texels(gnt) if gnt is not None else None
            res.append((p, c, x, nx))
        return res

    def status(self):
        return self.r.device_status()


def oracle_ulp_spread(mesh, view, params, win, rgba):
    """Per pixel, how far the oracle's image moves when every float32 position and UV
    coordinate moves one ulp up, or one ulp down: the conditioning floor of the forward
    tolerance (max(1e-5, twice this spread))."""
    import dataclasses
    spread = np.zeros(rgba.shape[:2])
    for direction in (np.inf, -np.inf):
        pert = dataclasses.replace(
            mesh, pos=np.nextafter(mesh.pos, np.float32(direction)).astype(np.float32),
            uv=None if mesh.uv is None else np.nextafter(mesh.uv, np.float32(direction)).astype(np.float32))
        o = oracle.render(pert, view, params, window=win)
        spread = np.maximum(spread, np.abs(o["rgba"] - rgba).max(-1))
    return spread


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def window_of(view, win):
    return (0, 0, view.width, view.height) if win is None else win


def compare_scene(scene, windows=None, seed=0, grad_from_target=None, store_layers=True, list_cap=0,
                  check_grads=True, report=None, tile=0, camera=False, schedule=0):
    """Runs both paths on every view (restricted to ``windows``) and asserts parity.
    Returns a dict of the measured errors."""
    gpu = CudaPath(scene, list_cap=list_cap, tile=tile, schedule=schedule)
    gpu.forward(store_layers=store_layers)
    rng = np.random.default_rng(seed)
    stats = dict(ids_checked=0, ids_unstable=0, fwd_err=0.0, fwd_checked=0)
    grads = []
    for i, v in enumerate(scene.views):
        win = windows[i] if windows is not None else None
        x0, y0, w, h = window_of(v, win)
        o = oracle.render(scene.meshes[v.mesh], v, scene.params, window=win)
        s_ids, s_val = masks(o, scene.params, v)
        gi = gpu.view_ids(i)[:, y0:y0 + h, x0:x0 + w]
        gh = gpu.view_hard(i)[:, y0:y0 + h, x0:x0 + w]
        # the stored ids carry each layer's hard / soft flag as well
        bad_hard = ((gh != (o["hard"] != 0)) & (o["ids"] >= 0)).any(0) & s_ids
        assert not bad_hard.any(), f"view {i}: {bad_hard.sum()} stable pixels with different hard flags"
        bad = (gi != o["ids"]).any(0) & s_ids
        stats["ids_checked"] += int(s_ids.sum())
        stats["ids_unstable"] += int((~s_ids).sum())
        assert not bad.any(), f"view {i}: {bad.sum()} stable pixels with different layer ids, first at {np.argwhere(bad)[:3]}"
        rgba = gpu.view_rgba(i)[y0:y0 + h, x0:x0 + w]
        err_px = np.abs(rgba - o["rgba"]).max(-1)
        err = err_px[s_val]
        if err.size:
            stats["fwd_err"] = max(stats["fwd_err"], float(err.max()))
            if err.max() > FWD_TOL:
                # the FP32 floor: where the oracle itself moves by more than the tolerance
                # when its float32 inputs move by one ulp, the bound is twice that spread
                spread = oracle_ulp_spread(scene.meshes[v.mesh], v, scene.params, win, o["rgba"])
                allowed = np.maximum(FWD_TOL, 2.0 * spread)
                over = (err_px > allowed) & s_val
                assert not over.any(), (f"view {i}: {over.sum()} stable pixels over max(1e-5, 2 x ulp spread), worst "
                                        f"{err_px[over].max():.3e} against {allowed[over].min():.3e}")
                stats["fwd_floor_pixels"] = stats.get("fwd_floor_pixels", 0) + int(((err_px > FWD_TOL) & s_val).sum())
                stats["fwd_err_over_floor"] = max(stats.get("fwd_err_over_floor", 0.0),
                                                  float((err_px / allowed)[s_val].max()))
        stats["fwd_checked"] += int(s_val.sum())
        # pixel gradient: L2 to a target image if given, else seeded noise; zero on unstable pixels
        if grad_from_target is not None:
            gv = 2.0 * (o["rgba"] - grad_from_target[i])
        else:
            gv = rng.normal(size=(h, w, 4))
        gv = np.where(s_val[..., None], gv, 0.0)
        full = np.zeros((v.height, v.width, 4))
        full[y0:y0 + h, x0:x0 + w] = gv
        grads.append(full)
        stats.setdefault("per_view", []).append((gv, win))
    # pixels past 1e-5 were checked against the ulp floor above
    assert stats["fwd_err"] <= FWD_TOL or stats.get("fwd_err_over_floor", 0.0) <= 1.0
    if check_grads:
        if camera:
            g_gpu, gm_gpu, gl_gpu = gpu.backward(grads, use_ids=store_layers, camera=True)
        else:
            g_gpu = gpu.backward(grads, use_ids=store_layers)
        nmap = scene.params.shade_mode == 3
        res = [[np.zeros(m.pos.shape), None if m.col is None else np.zeros(m.col.shape),
                None if m.tex is None else np.zeros(m.tex.shape),
                np.zeros(m.ntex.shape) if nmap else None] for m in scene.meshes]
        errs = {}
        for i, v in enumerate(scene.views):
            gv, win = stats["per_view"][i]
            gnt = None
            if camera:
                gp, gc, gt, gm, gl, *rest = oracle.backward(scene.meshes[v.mesh], v, scene.params, gv, window=win,
                                                            camera=True, want_ntex=nmap)
                gnt = rest[0] if nmap else None
                if np.any(gm):
                    e = rel_l2(gm_gpu[i], gm)
                    errs[f"mvp{i}"] = e
                    assert e <= GRAD_TOL, f"view {i} grad_mvp rel-L2 {e:.3e} > {GRAD_TOL}"
                if scene.params.shade_mode >= 2 and np.any(gl):
                    e = rel_l2(gl_gpu[i], gl)
                    errs[f"light{i}"] = e
                    assert e <= GRAD_TOL, f"view {i} grad_light rel-L2 {e:.3e} > {GRAD_TOL}"
                else:
                    assert not np.any(gl) and not np.any(gl_gpu[i])
                assert not np.any(gm_gpu[i][8:12])   # the depth row
            else:
                gp, gc, gt, *rest = oracle.backward(scene.meshes[v.mesh], v, scene.params, gv, window=win,
                                                    want_ntex=nmap)
                gnt = rest[0] if nmap else None
            res[v.mesh][0] += gp
            if gc is not None:
                res[v.mesh][1] += gc
            if gt is not None:
                res[v.mesh][2] += gt
            if gnt is not None:
                res[v.mesh][3] += gnt
        for mi, (o_, g_) in enumerate(zip(res, g_gpu)):
            for name, a, b in (("pos", g_[0], o_[0]), ("col", g_[1], o_[1]), ("tex", g_[2], o_[2]),
                               ("ntex", g_[3], o_[3])):
                if a is None or b is None or not np.any(b):
                    continue
                if name == "tex" and scene.params.shade_mode == 0:
                    continue
                e = rel_l2(a, b)
                errs[f"{name}{mi}"] = e
                assert e <= GRAD_TOL, f"mesh {mi} grad_{name} rel-L2 {e:.3e} > {GRAD_TOL}"
        stats["grad_err"] = errs
    stats.pop("per_view", None)
    assert (gpu.status() & ~1) == 0, gpu.status()
    stats["status"] = gpu.status()
    if report is not None:
        report.update(stats)
    return stats
