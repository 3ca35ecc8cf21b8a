"""The multi-GPU layout of the path on CPU ranks (gloo, world size 2).

Views are independent, so ranks shard them (bench.py's workload_scene strides the
views over ranks) and the only exchange is the sum of the gradients over views (one
all-reduce of the position and texel gradients).  Here each rank computes its views'
gradients with the FP64 oracle, the ranks all-reduce them, and the result must equal
the single-process sum over all views."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _scene(rank, world):
    return bench.workload_scene(rank, world, n_views=2, res=24, workload="multiview")


def _grads(scene, seed):
    m = scene.meshes[0]
    gp = np.zeros(m.pos.shape)
    gt = np.zeros(m.tex.shape)
    for v in scene.views:
        # a pixel gradient that depends only on the view, not on the rank holding it
        key = int(abs(np.asarray(v.mvp, np.float64)).sum() * 1e6) % (2 ** 31)
        g = np.random.default_rng(seed + key).normal(size=(v.height, v.width, 4))
        p, _, t = oracle.backward(m, v, scene.params, g)
        gp += p
        gt += t
    return gp, gt


def _worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = _scene(rank, world)
        gp, gt = _grads(s, 11)
        tp, tt = torch.from_numpy(gp), torch.from_numpy(gt)
        dist.all_reduce(tp)
        dist.all_reduce(tt)
        # max-over-ranks of a per-rank timing, as bench.py reports it
        t = torch.tensor([float(rank + 1)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            np.savez(out_path, gp=tp.numpy(), gt=tt.numpy(), tmax=t.numpy())
    finally:
        dist.destroy_process_group()


def test_view_sharding_partitions_the_views():
    """Two ranks with 2 views each hold exactly the 4 views of one rank with 4."""
    parts = [_scene(r, 2) for r in range(2)]
    assert [len(p.views) for p in parts] == [2, 2]
    got = sorted(tuple(np.asarray(v.mvp).ravel()) for p in parts for v in p.views)
    want = sorted(tuple(np.asarray(v.mvp).ravel()) for v in bench.workload_scene(0, 1, n_views=4, res=24).views)
    assert got == want
    assert not set(tuple(np.asarray(v.mvp).ravel()) for v in parts[0].views) & \
        set(tuple(np.asarray(v.mvp).ravel()) for v in parts[1].views)


def test_two_rank_gradient_allreduce_equals_single_process(tmp_path):
    world = 2
    out = str(tmp_path / "r0.npz")
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    got = np.load(out)
    ref = bench.workload_scene(0, 1, n_views=4, res=24)
    gp, gt = _grads(ref, 11)
    np.testing.assert_allclose(got["gp"], gp, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(got["gt"], gt, rtol=1e-12, atol=1e-12)
    assert got["tmax"][0] == 2.0


def test_bench_self_launch_spawns_ranks():
    """bench.py --gpus 2 without a launcher starts the two ranks itself (one process
    each, rendezvous on 127.0.0.1): here with gloo and the GPU-free check of the launch
    path, which takes each rank's views, joins the timed region's barriers and the
    max-over-ranks time and sums a gradient over ranks; rank 0 alone prints."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, "bench.py", "--gpus", "2", "--backend", "gloo", "--views", "2"], cwd=root,
                       capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d == {"n_gpus": 2, "views_rank0": 2, "tmax": 2.0, "grad_sum": [3.0, 3.0, 3.0]}
