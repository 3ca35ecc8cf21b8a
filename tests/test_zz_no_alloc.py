"""dressi_forward_static_scratch: the forward pass for callers that cannot allocate
device memory (for instance a plugin whose host application owns every device
allocation, or a frame loop that must not pay cudaMalloc's implicit device
synchronisation).  Its scratch lives in a fixed-size device array inside the library.

Checked here through the C ABI against dressi_forward with a caller workspace, on
consecutive calls (the array keeps the previous call's contents, so each call must
clear what it needs), and for the clear rejection of scenes that do not fit.
This file is collected last so that a failure here stops a -x run only after every
other test has run."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from paper_2204_01386_gb300 import binding as B
from paper_2204_01386_gb300.render import PackedScene, make_params, make_views

pytestmark = pytest.mark.gpu

STATIC_BYTES = 32 << 20


def _forward_with_workspace(lib, sc, views, nv, prm, n_pix, K, dev):
    ws_bytes = lib.dressi_workspace_size(C.byref(sc), views, nv, C.byref(prm))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    out = torch.full((n_pix, 4), float("nan"), device=dev)
    ids = torch.full((K, n_pix), -7, dtype=torch.int32, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    code = lib.dressi_forward(C.byref(sc), views, nv, C.byref(prm), out.data_ptr(), ids.data_ptr(), n_pix,
                              ws.data_ptr(), ws_bytes, st.data_ptr(), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == B.DRESSI_OK
    torch.cuda.synchronize()
    return out, ids, int(st.item()), ws_bytes


def _forward_static(lib, sc, views, nv, prm, n_pix, K, dev):
    out = torch.full((n_pix, 4), float("nan"), device=dev)
    ids = torch.full((K, n_pix), -7, dtype=torch.int32, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    code = lib.dressi_forward_static_scratch(C.byref(sc), views, nv, C.byref(prm), out.data_ptr(), ids.data_ptr(),
                                             n_pix, st.data_ptr(), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return code, out, ids, int(st.item())


def test_static_scratch_forward_matches_workspace_forward():
    lib = B.load()
    dev = torch.device("cuda", 0)
    # textured Lambert scene, then the vertex-colour scene, then the textured one with
    # 32 px tiles and the persistent longest-first schedule (tile counts, queue head and
    # the tile order live in the array), then the first again: every call must give the
    # workspace path's result whatever the array held before
    scenes = [(synth.config2(), 0, 0), (synth.config1(), 0, 0), (synth.config2(), 32, 2), (synth.config2(), 0, 0)]
    for s, tile, schedule in scenes:
        ps = PackedScene(s.meshes, dev)
        views, n_pix = make_views(s.views)
        prm = make_params(s.params, tile=tile, schedule=schedule)
        sc = ps.c_struct()
        K = s.params.K
        ref_out, ref_ids, ref_st, ws_bytes = _forward_with_workspace(lib, sc, views, len(s.views), prm, n_pix, K, dev)
        assert ws_bytes <= STATIC_BYTES
        code, out, ids, st = _forward_static(lib, sc, views, len(s.views), prm, n_pix, K, dev)
        assert code == B.DRESSI_OK
        assert st == ref_st == 0
        assert torch.equal(ids, ref_ids)
        err = (out - ref_out).abs().max().item()
        assert err <= 1e-5, err            # the parity tests' forward tolerance


def test_static_scratch_rejects_scenes_that_do_not_fit():
    lib = B.load()
    dev = torch.device("cuda", 0)
    s = synth.config3(n_views=64)
    ps = PackedScene(s.meshes, dev)
    views, n_pix = make_views(s.views)
    prm = make_params(s.params)
    sc = ps.c_struct()
    need = lib.dressi_workspace_size(C.byref(sc), views, len(s.views), C.byref(prm))
    assert need > STATIC_BYTES
    out = torch.zeros(8, 4, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    code = lib.dressi_forward_static_scratch(C.byref(sc), views, len(s.views), C.byref(prm), out.data_ptr(), None,
                                             n_pix, st.data_ptr(), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == B.DRESSI_ERR_WORKSPACE
    assert int(st.item()) == 0
