"""The C ABI without a GPU: the library loads, exports every symbol that
include/dressi.h declares, its structs match the binding's layout, and the
host-side argument checks and workspace sizing behave."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2204_01386_gb300 import _build_ext
from paper_2204_01386_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dressi.h")


@pytest.fixture(scope="module")
def lib():
    _build_ext.build()
    return B.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(dressi_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 7
    for n in names:
        assert hasattr(lib, n), n
        assert n in B.SIGNATURES, f"binding lacks {n}"
    nm = subprocess.run(["nm", "-D", "--defined-only", _build_ext.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (dressi_\w+)", nm))
    assert set(names) <= exported
    # nothing else leaks out under the dressi_ prefix
    assert exported <= set(names)


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "dressi.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(dressi_mesh), sizeof(dressi_scene),'
                    ' sizeof(dressi_view), sizeof(dressi_params), offsetof(dressi_view, pix_off),'
                    ' offsetof(dressi_params, list_cap), offsetof(dressi_params, schedule),'
                    ' offsetof(dressi_params, uv_jitter), offsetof(dressi_params, reuse_setup));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(B.DressiMesh), C.sizeof(B.DressiScene), C.sizeof(B.DressiView), C.sizeof(B.DressiParams),
            B.DressiView.pix_off.offset, B.DressiParams.list_cap.offset, B.DressiParams.schedule.offset,
            B.DressiParams.uv_jitter.offset, B.DressiParams.reuse_setup.offset]
    assert got == want


def _scene(nv=3, nf=1, tex=False):
    meshes = (B.DressiMesh * 1)(B.DressiMesh(nv, nf, 0, 0, 0, 4 if tex else 0, 4 if tex else 0))
    fake = 0x10000  # never dereferenced: only host-side checks run
    sc = B.DressiScene(1, C.cast(meshes, C.POINTER(B.DressiMesh)), nv, fake, fake, fake if tex else None, fake,
                       fake if tex else None, 0)
    return sc, meshes


def _views(n=1, w=64, h=48):
    arr = (B.DressiView * n)()
    for i in range(n):
        arr[i].mvp[:] = [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1]
        arr[i].mesh, arr[i].width, arr[i].height, arr[i].pix_off = 0, w, h, i * w * h
    return arr


def test_workspace_size_host_only(lib):
    sc, keep = _scene()
    v = _views(2)
    p = B.DressiParams(3, 0.01, 0.01 / 7, 0.01, 0.0, 0, 0, 0, 0, 0, 0)
    n = lib.dressi_workspace_size(C.byref(sc), v, 2, C.byref(p))
    assert n > 0 and n % 256 == 0
    p2 = B.DressiParams(3, 0.01, 0.01 / 7, 0.01, 0.0, 0, 0, 0, 0, 0, 10 ** 6)
    assert lib.dressi_workspace_size(C.byref(sc), v, 2, C.byref(p2)) > n


@pytest.mark.parametrize("bad", ["K0", "K6", "sigma0", "edge3", "shade_tex_missing", "mesh_idx", "pix_off", "tile",
                                 "rho_too_big", "nan_mvp", "schedule", "reuse2"])
def test_invalid_arguments_rejected_on_host(lib, bad):
    sc, keep = _scene()
    v = _views(1)
    p = B.DressiParams(3, 0.01, 0.01 / 7, 0.01, 0.0, 0, 0, 0, 0, 0, 0)
    n_pix = 64 * 48
    if bad == "K0":
        p.K = 0
    elif bad == "K6":
        p.K = 6
    elif bad == "sigma0":
        p.sigma = 0.0
    elif bad == "edge3":
        p.edge_mode = 3
    elif bad == "shade_tex_missing":
        p.shade_mode = 1
    elif bad == "mesh_idx":
        v[0].mesh = 1
    elif bad == "pix_off":
        v[0].pix_off = 5
    elif bad == "tile":
        p.tile = 12
    elif bad == "rho_too_big":
        p.delta = 0.5
    elif bad == "nan_mvp":
        v[0].mvp[3] = float("nan")
    elif bad == "schedule":
        p.schedule = 3
    elif bad == "reuse2":
        p.reuse_setup = 2
    if bad != "pix_off":   # the image size is only known to the passes
        assert lib.dressi_workspace_size(C.byref(sc), v, 1, C.byref(p)) == 0
    # the entry points reject before touching the device
    code = lib.dressi_forward(C.byref(sc), v, 1, C.byref(p), 0x1000, None, n_pix, 0x1000, 1 << 40, 0x1000, None)
    assert code == B.DRESSI_ERR_ARG
    code = lib.dressi_backward(C.byref(sc), v, 1, C.byref(p), 0x1000, None, n_pix, 0x1000, None, None, 0x1000,
                               1 << 40, 0x1000, None)
    assert code == B.DRESSI_ERR_ARG


def test_texture_with_too_many_texels_rejected(lib):
    """Texel counts are int32 on the device: a texture of 2^31 texels or more is refused."""
    sc, meshes = _scene(tex=True)
    v = _views(1)
    p = B.DressiParams(3, 0.01, 0.01 / 7, 0.01, 0.0, 0, 1, 0, 0, 0, 0)
    assert lib.dressi_workspace_size(C.byref(sc), v, 1, C.byref(p)) > 0
    meshes[0].tex_w, meshes[0].tex_h = 65536, 32768
    assert lib.dressi_workspace_size(C.byref(sc), v, 1, C.byref(p)) == 0


def test_texel_gather_refuses_texel_indices_past_32_bits(lib):
    """The texel gather (texgrad_mode 1) sorts 32-bit texel keys, 0xffffffff marking an
    empty slot: a packed texel buffer of 2^32 - 1 texels or more is refused for it, while
    the atomics mode (64-bit texel offsets) takes it."""
    sc, meshes = _scene(tex=True)
    v = _views(1)
    p = B.DressiParams(3, 0.01, 0.01 / 7, 0.01, 0.0, 0, 1, 1, 0, 0, 0)
    assert lib.dressi_workspace_size(C.byref(sc), v, 1, C.byref(p)) > 0
    for off, ok in ((2 ** 32 - 18, True), (2 ** 32 - 17, False), (2 ** 32 - 8, False), (2 ** 40, False)):
        meshes[0].tex_off = off           # 16 texels: the last index is off + 15
        assert (lib.dressi_workspace_size(C.byref(sc), v, 1, C.byref(p)) > 0) == ok, off
        code = lib.dressi_backward(C.byref(sc), v, 1, C.byref(p), 0x1000, None, 64 * 48, 0x1000, None, 0x1000,
                                   0x1000, 0 if ok else 1 << 40, 0x1000, None)
        assert code == (B.DRESSI_ERR_WORKSPACE if ok else B.DRESSI_ERR_ARG), off
        p.texgrad_mode = 0
        assert lib.dressi_workspace_size(C.byref(sc), v, 1, C.byref(p)) > 0, off
        p.texgrad_mode = 1


def test_fused_loss_arguments_rejected_on_host(lib):
    """dressi_forward_l2 wants a target and a gradient buffer, 16-byte aligned like the
    image; it rejects them before touching the device."""
    sc, keep = _scene()
    v = _views(1)
    p = B.DressiParams(3, 0.01, 0.01 / 7, 0.01, 0.0, 0, 0, 0, 0, 0, 0)
    n = lib.dressi_workspace_size(C.byref(sc), v, 1, C.byref(p))
    args = dict(target=0x1000, out=0x1000, grad=0x2000)
    for key, bad in (("target", None), ("grad", None), ("target", 0x1004), ("grad", 0x2008), ("out", 0x1002)):
        a = dict(args, **{key: bad})
        code = lib.dressi_forward_l2(C.byref(sc), v, 1, C.byref(p), a["target"], a["out"], a["grad"], None, None,
                                     64 * 48, 0x1000, n, 0x1000, None)
        assert code == B.DRESSI_ERR_ARG, (key, bad)


def test_workspace_too_small_rejected(lib):
    sc, keep = _scene()
    v = _views(1)
    p = B.DressiParams(3, 0.01, 0.01 / 7, 0.01, 0.0, 0, 0, 0, 0, 0, 0)
    n = lib.dressi_workspace_size(C.byref(sc), v, 1, C.byref(p))
    code = lib.dressi_forward(C.byref(sc), v, 1, C.byref(p), 0x1000, None, 64 * 48, 0x1000, n - 1, 0x1000, None)
    assert code == B.DRESSI_ERR_WORKSPACE
    code = lib.dressi_forward(C.byref(sc), v, 1, C.byref(p), 0x1000, None, 64 * 48, None, n, 0x1000, None)
    assert code == B.DRESSI_ERR_WORKSPACE


def test_status_strings(lib):
    for c in range(4):
        assert lib.dressi_status_string(c)
    for b in (0, 1, 2, 4):
        assert lib.dressi_dev_status_string(b)
    assert lib.dressi_abi_version() == B.ABI_VERSION == 3


def test_product_has_no_fallback(monkeypatch, tmp_path):
    """Without the built library the binding raises instead of computing anything."""
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(B.DressiError):
        B.load(str(tmp_path / "missing.so"))


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2204_01386_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "hardsoftras_oracle" not in txt, f


def test_decode_layer_ids():
    """Stored layer ids: face index, bit 31 set for a soft fragment, -1 for an empty layer."""
    import numpy as np
    import torch
    from paper_2204_01386_gb300 import decode_layer_ids
    raw = np.array([5, 5 | -0x80000000, -1, 0, -0x80000000, 0x7FFFFFFE, 0x7FFFFFFE | -0x80000000], np.int64).astype(np.int32)
    face, hard = decode_layer_ids(raw)
    assert face.tolist() == [5, 5, -1, 0, 0, 0x7FFFFFFE, 0x7FFFFFFE]
    assert hard.tolist() == [True, False, False, True, False, True, False]
    tf, th = decode_layer_ids(torch.as_tensor(raw))
    assert tf.tolist() == face.tolist() and th.tolist() == hard.tolist()
