"""The renderer's record of what its workspace holds (host logic, no GPU): the backward
may take the forward's setup only for the same positions (storage and version),
parameters and workspace, and takes the tile lists only when a setup with them left them
there."""
import ctypes as C

import torch

from paper_2204_01386_gb300 import binding as B
from paper_2204_01386_gb300.render import Renderer


class _Scene:
    def __init__(self):
        self.pos = torch.zeros(3, 8)


def _renderer():
    r = Renderer.__new__(Renderer)   # no library, no device: only the bookkeeping
    r.scene = _Scene()
    r.params = B.DressiParams(3, 0.01, 0.01 / 7, 0.01, 0.0, 0, 0, 0, 0, 0, 0)
    r.ws = torch.empty(64, dtype=torch.uint8)
    r._setup = None
    return r


def _setup(r, pos=None, bins=True):
    key = r._setup_key(pos)
    old = r._begin_setup()
    r._end_setup(old, key, bins)


def test_forward_setup_is_reusable_for_the_same_inputs():
    r = _renderer()
    assert not r._setup_reusable(r._setup_key(None), True)
    _setup(r)
    key = r._setup_key(None)
    assert r._setup_reusable(key, True) and r._setup_reusable(key, False)


def test_changed_positions_parameters_or_workspace_are_not():
    r = _renderer()
    _setup(r)
    r.scene.pos.add_(1.0)                       # in place: the version counter moves
    assert not r._setup_reusable(r._setup_key(None), True)
    r = _renderer()
    _setup(r)
    r.params.sigma = 0.02
    assert not r._setup_reusable(r._setup_key(None), True)
    r = _renderer()
    _setup(r)
    r.ws = torch.empty(64, dtype=torch.uint8)
    assert not r._setup_reusable(r._setup_key(None), True)
    other = torch.zeros(3, 8)
    r = _renderer()
    _setup(r)
    assert not r._setup_reusable(r._setup_key(other), True)


def test_tile_lists_survive_a_setup_without_them_only_for_the_same_key():
    r = _renderer()
    _setup(r, bins=True)
    _setup(r, bins=False)                       # e.g. the forward from stored layers
    assert r._setup_reusable(r._setup_key(None), False)
    r = _renderer()
    _setup(r, bins=True)
    other = torch.zeros(3, 8)
    _setup(r, pos=other, bins=False)            # another geometry: its lists were never built
    assert r._setup_reusable(r._setup_key(other), True)
    assert not r._setup_reusable(r._setup_key(other), False)


def test_the_reuse_flag_is_not_part_of_the_key():
    r = _renderer()
    _setup(r)
    r.params.reuse_setup = 1
    assert r._setup_reusable(r._setup_key(None), True)
    assert r.params.reuse_setup == 0            # the key is taken with the flag cleared
    assert C.sizeof(r.params) == C.sizeof(B.DressiParams)
