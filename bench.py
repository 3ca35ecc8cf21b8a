#!/usr/bin/env python3
"""Throughput of the HardSoftRas forward + adjoint hot path on GB300.

One step = forward (store layer ids) + L2 pixel gradient + adjoint over a
batch of views, all in libdressi kernels, inputs resident in HBM.  Default
workload: the batched multi-view configuration (64 views of 512^2 of a
20,480-triangle displaced UV sphere with a 1024^2 FP32 texture, Lambert
shading, K = 3, r = 2 px, sigma = r/7, delta = r).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "fwd+bwd Mpixel*views/s"
# FP32 arithmetic (an FMA counts 2) the method needs per unit of work, counted from
# the operations written in the kernels: one exact SignedDist + Shift evaluation of a
# candidate face at a pixel; one layer's barycentrics, texture sample, Lambert
# shading and blend; one layer's adjoint with the forward values it recomputes.
FLOP_CANDIDATE = 50
FLOP_SHADE_LAYER = 110
FLOP_ADJOINT_LAYER = 340
FP32_LANES_PER_SM = 128
UNIT = "Mpixel*views/s"
L2_FLUSH_BYTES = 512 << 20


WORKLOADS = ("multiview", "textured", "ragged", "large")


def workload_scene(rank=0, world=1, n_views=None, res=512, workload="multiview"):
    """The benchmark workloads.  multiview (default): 64 views of 512^2 of a 20,480-tri
    displaced UV sphere, 1024^2 FP32 texture, Lambert.  textured: one 256^2 view of a
    5,120-tri sphere with a 512^2 texture.  ragged: 32 meshes of 1k..200k tris at mixed
    resolutions and textures.  large: 1.31M-tri icosphere, 4096^2 FP16 texture, 8 views
    of 2048^2, checkpointed backward.  With several ranks every rank renders its own
    views (directions strided over ranks): weak scaling."""
    if workload == "multiview":
        s = synth.config3(n_views=(n_views or 64) * world, res=res)
    elif workload == "textured":
        s = synth.config2()
        s.views = s.views * world
    elif workload == "ragged":
        s = synth.config4()
    else:
        s = synth.config5(n_views=(n_views or 8) * world)
    s.views = s.views[rank::world]
    return s


def workload_desc(s, workload="multiview"):
    m = s.meshes[0]
    tris = sorted({int(x.faces.shape[0]) for x in s.meshes})
    d = {"views": len(s.views), "resolution": s.views[0].width, "triangles": tris[0] if len(tris) == 1 else tris,
         "texture": int(m.tex.shape[0]), "K": s.params.K, "store_layers": bool(s.params.store_layers),
         "l2": "512 MiB buffer written between timed steps"}
    if workload == "multiview":
        d["workload"] = ("batched multi-view: %d views x %dx%d, %d-tri displaced UV sphere, %dx%d FP32 texture, "
                         "Lambert, K=%d, r=2px" % (len(s.views), s.views[0].width, s.views[0].height,
                                                    m.faces.shape[0], m.tex.shape[1], m.tex.shape[0], s.params.K))
    else:
        d["workload"] = s.name
    return d


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------
def host_threads():
    """The host cores this process may use."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except (AttributeError, OSError):
        return max(1, os.cpu_count() or 1)


def time_oracle(scene, n_views, seed=0, threads=1):
    """Forward + adjoint of the first n_views views by the oracle; with threads > 1 the
    views run concurrently on that many host threads (the oracle's C calls release the
    GIL and keep no shared state).  Returns (pixels, wall seconds)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    views = scene.views[:n_views]
    grads = [np.random.default_rng((seed, i)).normal(size=(v.height, v.width, 4)) for i, v in enumerate(views)]

    def one(i):
        v = views[i]
        m = scene.meshes[v.mesh]
        oracle.render(m, v, scene.params)
        oracle.backward(m, v, scene.params, grads[i])
        return v.width * v.height

    oracle.render(scene.meshes[views[0].mesh], views[0], scene.params, window=(0, 0, 1, 1))   # load before threads
    t0 = time.perf_counter()
    if threads > 1:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            px = sum(ex.map(one, range(len(views))))
    else:
        px = sum(one(i) for i in range(len(views)))
    dt = time.perf_counter() - t0
    return px, dt


def reference_arm(args, rank, world):
    if rank != 0:
        return
    s = workload_scene(0, 1, n_views=args.views, workload=args.workload)
    # one view per host thread per step, the views of a step run concurrently
    threads = host_threads()
    views_per_step = min(threads, len(s.views))
    for _ in range(args.warmup):
        time_oracle(s, views_per_step, threads=threads)
    times, pxs = [], 0
    for k in range(args.steps):
        first = (k * views_per_step) % len(s.views)
        sub = synth.Scene(s.name, s.meshes, (s.views[first:] + s.views[:first])[:views_per_step], s.params)
        px, dt = time_oracle(sub, views_per_step, seed=k, threads=threads)
        times.append(dt)
        pxs += px
    total = sum(times)
    value = pxs / total / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_desc(s, args.workload),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{views_per_step} view(s) of {s.views[0].width}^2 per step on "
                                       f"{threads} host threads, FP64 C oracle (bbox pre-test)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def algorithmic_bytes(scene, K, backward, store_layers=True, fused_loss=True):
    """Bytes one launch of the per-tile kernel must move at minimum:
    forward: RGBA out 16 B (+ K layer ids 4 B when stored) per pixel, with the fused L2
    loss also the target read and dL/dout written (2 x 16 B); per view the vertex
    records (32 B) and faces (12 B) of its mesh; every texture once (texel bytes).
    adjoint: dL/dI 16 B (+ K ids 4 B when stored) per pixel; per view vertex records,
    faces and the screen-gradient accumulators (16 B read + 16 B written per vertex);
    textures read once and the FP32 texel gradient read + written once (2 x 16 B/texel)."""
    px = scene.pixels
    per_view = sum(32 * scene.meshes[v.mesh].pos.shape[0] + 12 * scene.meshes[v.mesh].faces.shape[0]
                   for v in scene.views)
    tex_bytes = sum(m.tex.shape[0] * m.tex.shape[1] * 4 * m.tex.itemsize for m in scene.meshes if m.tex is not None)
    texels = sum(m.tex.shape[0] * m.tex.shape[1] for m in scene.meshes if m.tex is not None)
    ids = 4 * K if store_layers else 0
    if not backward:
        return px * (16 + ids + (32 if fused_loss else 0)) + per_view + tex_bytes
    acc = sum(32 * scene.meshes[v.mesh].pos.shape[0] for v in scene.views)
    return px * (16 + ids) + per_view + acc + tex_bytes + 2 * 16 * texels


def kernel_source_hash(text):
    """Hash of CUDA source with comments and whitespace removed: a comment edit keeps a
    capture valid, any code change does not."""
    import hashlib
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return hashlib.sha1(re.sub(r"\s+", "", text).encode()).hexdigest()[:16]


def recorded_traffic(kernel, pixels):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled to
    `pixels`, or None when the kernel sources changed since the capture."""
    import hashlib
    try:
        rec = dict(line.split(": ", 1) for line in open(os.path.join(ROOT, "profiles", "k_tile_traffic.txt"))
                   .read().splitlines() if line and not line.startswith("#"))
    except OSError:
        return None
    csrc = os.path.join(ROOT, "paper_2204_01386_gb300", "csrc")
    h = kernel_source_hash(open(os.path.join(csrc, "dressi_tile.cuh")).read() +
                           open(os.path.join(csrc, "dressi_core.cuh")).read())
    if rec.get("source_hash") != h or kernel not in rec:
        return None
    nbytes, npix = rec[kernel].split()
    return int(nbytes) * pixels / int(npix)


def measured_peaks(lib, dev):
    """FP32 FMA TFLOP/s and red.global.add.v4.f32 GB/s (coalesced, and scattered one sector
    per lane) of this device, from the library's microbenchmarks (dressi_measure_peak), and
    the SM count."""
    import ctypes as C

    import torch
    buf = torch.zeros(64 << 18, dtype=torch.float32, device=dev)   # 64 MiB
    stream = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    res = {}
    for which, name in ((0, "fp32_tflops"), (1, "red_v4_gbs"), (2, "red_v4_scattered_gbs")):
        v = C.c_double(0.0)
        code = lib.dressi_measure_peak(which, C.c_void_p(buf.data_ptr()), buf.numel() * 4, C.byref(v), stream)
        res[name] = float(v.value) if code == 0 else None
    res["sms"] = int(torch.cuda.get_device_properties(dev).multi_processor_count)
    del buf
    return res


def measure(s, args, dev, world, rank, dist, flush, peaks, hbm_peak, main=False, n_steps=None, plain_arm=True):
    """Times the step (forward with the L2 loss fused in, then the adjoint) of scene ``s``
    on this rank: the per-tile kernels by CUDA events (non-graph steps), then whole steps
    replayed from a CUDA graph (the gradient all-reduce over ranks stays outside the graph),
    then, at one rank, the same views as a plain per-view launch sequence.  Returns the
    record and the state the main workload's extra legs reuse."""
    import ctypes as C

    import torch

    from paper_2204_01386_gb300 import PackedScene, Renderer
    from paper_2204_01386_gb300 import binding as B

    n_steps = n_steps or args.steps
    s.params.texgrad_mode = args.texgrad
    store = bool(s.params.store_layers)
    tgt_scene = synth.perturbed(s, 4321 + rank)
    ps = PackedScene(s.meshes, dev)
    r = Renderer(ps, s.views, s.params, tile=args.tile, schedule=args.schedule)
    tuned = None
    if args.tile == 0 and args.schedule == 0:
        tuned = r.autotune(cache_path=os.path.join(tempfile.gettempdir(), "dressi_bench_autotune.json"),
                           store_layers=store)
    tile = int(r.params.tile) or 16
    schedule = int(r.params.schedule) or 1
    # target images (inputs of the loss), rendered once outside the timed region
    pt = PackedScene(tgt_scene.meshes, dev)
    rt = Renderer(pt, tgt_scene.views, tgt_scene.params, tile=tile)
    target, _ = rt.forward(store_layers=False)
    torch.cuda.synchronize()
    del rt, pt
    lib = B.load()
    n_pix = r.n_pix
    out = torch.empty(n_pix, 4, device=dev)
    ids = torch.empty(s.params.K, n_pix, dtype=torch.int32, device=dev) if store else None
    grad = torch.empty_like(out)
    loss = torch.zeros(1, device=dev)
    gp = torch.empty(3, ps.n_verts_total, device=dev)
    gt = torch.empty(ps.n_texels, 4, device=dev)
    stream = torch.cuda.current_stream(dev)

    def compute():
        # forward with the L2 loss fused in (out, dL/dout, loss), then the adjoint
        loss.zero_()
        r.forward(store_layers=store, out=out, ids=ids, target=target, grad=grad, loss=loss)
        r.backward(grad, ids=ids, grad_pos=gp, grad_tex=gt)

    def exchange():
        # views are sharded over ranks: the gradients are summed over all views
        if world > 1:
            dist.all_reduce(gp)
            dist.all_reduce(gt)

    for _ in range(args.warmup):
        compute()
        exchange()
    torch.cuda.synchronize()
    assert (r.device_status() & ~1) == 0, r.device_status()
    c0 = lib.dressi_launch_count()
    compute()
    torch.cuda.synchronize()
    launches_per_step = lib.dressi_launch_count() - c0

    # 1) the per-tile kernels timed live: CUDA events recorded by the library right
    #    around them, on the stream they are launched on, in non-graph steps
    n_prof = max(3, min(n_steps, 10))
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(n_prof)]
    for e in ev:
        for x in e:
            x.record(stream)
    torch.cuda.synchronize()
    for k in range(n_prof):
        flush.fill_(float(k))
        e = ev[k]
        lib.dressi_set_profile_events(C.c_void_p(e[0].cuda_event), C.c_void_p(e[1].cuda_event),
                                      C.c_void_p(e[2].cuda_event), C.c_void_p(e[3].cuda_event))
        compute()
    torch.cuda.synchronize()
    lib.dressi_set_profile_events(None, None, None, None)
    fwd_ms = [e[0].elapsed_time(e[1]) for e in ev]
    bwd_ms = [e[2].elapsed_time(e[3]) for e in ev]

    # work counters of one forward and one adjoint launch (untimed pass)
    counters = torch.zeros(4, dtype=torch.int64, device=dev)
    lib.dressi_set_stats_buffer(C.c_void_p(counters.data_ptr()))
    r.forward(store_layers=store, out=out, ids=ids)
    torch.cuda.synchronize()
    st_fwd = [int(x) for x in counters.tolist()]
    counters.zero_()
    r.backward(grad, ids=ids, grad_pos=gp, grad_tex=gt)
    torch.cuda.synchronize()
    st_bwd = [int(x) for x in counters.tolist()]
    lib.dressi_set_stats_buffer(None)

    # 2) whole steps: the compute replayed from a CUDA graph, the exchange after it
    use_graph = not args.no_graph
    run = compute
    if use_graph:
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg):
            compute()
        cg.replay()
        torch.cuda.synchronize()
        run = cg.replay
    tev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]
    clocks = Clocks(dev.index or 0)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(n_steps):
        flush.fill_(float(k))
        tev[k][0].record(stream)
        run()
        exchange()
        tev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clock_info = clocks.stop()
    assert (r.device_status() & ~1) == 0, r.device_status()
    total_ms = sum(a.elapsed_time(b) for a, b in tev)
    if world > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = s.pixels * world * n_steps / (total_ms * 1e-3) / 1e6

    # dominant kernel roofline (live CUDA-event durations of the per-tile kernels)
    fwd_avg, bwd_avg = statistics.mean(fwd_ms), statistics.mean(bwd_ms)
    bwd_dom = bwd_avg >= fwd_avg
    kb = algorithmic_bytes(s, s.params.K, bwd_dom, store)
    dur = (bwd_avg if bwd_dom else fwd_avg) * 1e-3
    st = st_bwd if bwd_dom else st_fwd
    flops = st[2] * FLOP_CANDIDATE + st[3] * (FLOP_ADJOINT_LAYER if bwd_dom else FLOP_SHADE_LAYER)
    achieved = flops / dur / 1e12
    alu_peak = peaks.get("fp32_tflops")
    peak_source = "measured: FP32 FMA microbenchmark (dressi_measure_peak) on %d SMs" % peaks["sms"]
    if not alu_peak:
        sm_mhz = clock_info.get("sm_mhz") or 2070.0
        alu_peak = peaks["sms"] * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        peak_source = "derived: %d SMs x %d lanes x 2 FLOP x %.0f MHz" % (peaks["sms"], FP32_LANES_PER_SM, sm_mhz)
    mode = "fwd" if not bwd_dom else ("bwd" if store else "bwd_recompute")
    kname = "k_tile<%d,%s,%d>" % (s.params.K, mode, tile)
    roofline = {"kernel": kname, "bound": "alu",
                "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
                "traffic": recorded_traffic(kname, s.pixels) if args.workload == "multiview" and main else None,
                "peak_source": peak_source,
                "algorithmic_flop": flops, "fwd_tile_ms": fwd_avg, "bwd_tile_ms": bwd_avg,
                "work_fwd": dict(zip(("pairs", "exact_evals", "candidates", "layers"), st_fwd)),
                "work_bwd": dict(zip(("pairs", "exact_evals", "candidates", "layers"), st_bwd)),
                "hbm_algorithmic_bytes": kb, "hbm_achieved_gbs": kb / dur / 1e9,
                "hbm_peak_gbs": hbm_peak, "hbm_frac": kb / dur / 1e9 / hbm_peak,
                "red_v4_peak_gbs": peaks.get("red_v4_gbs"), "red_v4_scattered_peak_gbs": peaks.get("red_v4_scattered_gbs")}

    # 3) the same views as a plain per-view launch sequence (one call per view, one CTA
    #    per tile), to compare with the batched form above
    plain = None
    if len(s.views) > 1 and plain_arm and not args.no_plain and world == 1:
        rv = [Renderer(ps, [v], s.params, tile=tile, schedule=1) for v in s.views]
        offs = [int(x.pix_off) for x in r.views]
        idv = [torch.empty(s.params.K, v.width * v.height, dtype=torch.int32, device=dev) if store else None
               for v in s.views]

        def plain_step():
            for i, (rr, v) in enumerate(zip(rv, s.views)):
                sl = slice(offs[i], offs[i] + v.width * v.height)
                rr.forward(store_layers=store, out=out[sl], ids=idv[i], target=target[sl], grad=grad[sl], loss=loss)
                rr.backward(grad[sl], ids=idv[i], grad_pos=gp, grad_tex=gt)

        for _ in range(2):
            plain_step()
        torch.cuda.synchronize()
        n_plain = max(3, n_steps // 2)
        pe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_plain)]
        for k in range(n_plain):
            flush.fill_(float(k))
            pe[k][0].record(stream)
            plain_step()
            pe[k][1].record(stream)
        torch.cuda.synchronize()
        pms = sum(a.elapsed_time(b) for a, b in pe)
        plain = {"value": s.pixels * n_plain / (pms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": pms / n_plain,
                 "note": "one forward/loss/adjoint call per view, one CTA per tile, no graph"}
        del rv
    rec = {"value": value, "unit": UNIT, "ms_per_step": total_ms / n_steps, "steps": n_steps,
           "tile": tile, "schedule": "persistent longest-first" if schedule == 2 else "CTA per tile",
           "autotuned": tuned is not None, "list_cap": int(r.params.list_cap), "cuda_graph": use_graph,
           "roofline": roofline, "plain_per_view": plain, "clocks": clock_info,
           "gpu_launches_per_step": int(launches_per_step)}
    state = dict(r=r, ps=ps, out=out, ids=ids, grad=grad, loss=loss, gp=gp, gt=gt, target=target, store=store,
                 exchange=exchange, use_graph=use_graph)
    return rec, state


def extra_legs(s, args, dev, world, dist, flush, st):
    """The main workload's extra legs: the static-geometry step and the end-to-end step
    through the public API with host buffers."""
    import torch

    r, ps, out, ids, grad, loss, gp, gt, target = (st[k] for k in ("r", "ps", "out", "ids", "grad", "loss", "gp",
                                                                     "gt", "target"))
    store, exchange, use_graph = st["store"], st["exchange"], st["use_graph"]
    stream = torch.cuda.current_stream(dev)
    # the same step with a static geometry (texture / colour optimisation): the forward
    # re-shades the layers the benchmark's forward stored (binning, raster and peel
    # skipped), then the loss and the adjoint from the same layers
    cached = None
    if store and world == 1 and not args.no_cached:
        ids0 = ids.clone()

        def cached_step():
            r.forward_from_layers(ids0, out=out)
            loss.zero_()
            r.l2_grad(out, target, grad, loss)
            r.backward(grad, ids=ids0, grad_pos=gp, grad_tex=gt)

        for _ in range(2):
            cached_step()
        torch.cuda.synchronize()
        crun = cached_step
        if use_graph:
            cgc = torch.cuda.CUDAGraph()
            with torch.cuda.graph(cgc):
                cached_step()
            cgc.replay()
            torch.cuda.synchronize()
            crun = cgc.replay
        n_c = max(3, args.steps // 2)
        ce = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_c)]
        for k in range(n_c):
            flush.fill_(float(k))
            ce[k][0].record(stream)
            crun()
            ce[k][1].record(stream)
        torch.cuda.synchronize()
        cms = sum(a.elapsed_time(b) for a, b in ce)
        cached = {"value": s.pixels * n_c / (cms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": cms / n_c,
                  "note": "static geometry: forward from the stored layers (no binning, raster or peel) + loss "
                          "+ adjoint from the same layers, CUDA graph"}

    # end to end through the public API with host buffers: every step copies its inputs
    # (positions, texture, target images) from pinned host memory and reads its results
    # (loss, gradients) back.  The inputs are double-buffered: the copy stream fills one
    # set with the next step's inputs while the compute stream runs the step on the other
    # (a data loader's prefetch); the results follow each step on the compute stream.
    e2e = None
    if not args.no_e2e:
        h_pos = ps.pos.cpu().pin_memory()
        h_tex = ps.tex.cpu().pin_memory()
        h_tgt = target.cpu().pin_memory()
        h_loss = torch.empty(1).pin_memory()
        h_gp = torch.empty_like(gp, device="cpu").pin_memory()
        h_gt = torch.empty_like(gt, device="cpu").pin_memory()
        h2d = h_pos.numel() * 4 + h_tex.numel() * h_tex.element_size() + h_tgt.numel() * 4
        d2h = 4 + h_gp.numel() * 4 + h_gt.numel() * 4
        d_in = [(ps.pos, ps.tex, target),
                (torch.empty_like(ps.pos), torch.empty_like(ps.tex), torch.empty_like(target))]
        # the results are double-buffered too: step i's device-to-host copies run on their own
        # stream while step i + 1 computes into the other set
        d_out = [(loss, gp, gt), (torch.zeros_like(loss), torch.empty_like(gp), torch.empty_like(gt))]

        def make_step(pos, tex, tgt, ls, gpk, gtk):
            def f():
                ls.zero_()
                r.forward(store_layers=store, out=out, ids=ids, pos=pos, tex=tex, target=tgt, grad=grad, loss=ls)
                r.backward(grad, ids=ids, grad_pos=gpk, grad_tex=gtk, pos=pos, tex=tex)
            return f

        runs = [make_step(*d_in[k], *d_out[k]) for k in range(2)]
        if use_graph:
            graphs = []
            for f in runs:
                f()
                torch.cuda.synchronize()
                gr = torch.cuda.CUDAGraph()
                with torch.cuda.graph(gr):
                    f()
                graphs.append(gr)
            runs = [gr.replay for gr in graphs]
        copy = torch.cuda.Stream(dev)
        drain = torch.cuda.Stream(dev)
        ready = [torch.cuda.Event() for _ in range(2)]     # inputs of set k on the device
        free = [torch.cuda.Event() for _ in range(2)]      # set k's inputs no longer read
        done = [torch.cuda.Event() for _ in range(2)]      # set k's results computed
        drained = [torch.cuda.Event() for _ in range(2)]   # set k's results copied to the host

        def e2e_steps(n):
            for ev in free + drained:
                ev.record(stream)

            def fetch(k):
                with torch.cuda.stream(copy):
                    copy.wait_event(free[k])
                    for d, h in zip(d_in[k], (h_pos, h_tex, h_tgt)):
                        d.copy_(h, non_blocking=True)
                    ready[k].record(copy)

            fetch(0)
            for i in range(n):
                k = i % 2
                if i + 1 < n:
                    fetch(1 - k)
                stream.wait_event(ready[k])
                stream.wait_event(drained[k])
                runs[k]()
                if world > 1:
                    dist.all_reduce(d_out[k][1])
                    dist.all_reduce(d_out[k][2])
                done[k].record(stream)
                free[k].record(stream)
                with torch.cuda.stream(drain):
                    drain.wait_event(done[k])
                    for h, d in zip((h_loss, h_gp, h_gt), d_out[k]):
                        h.copy_(d, non_blocking=True)
                    drained[k].record(drain)
            # the last step's results are on the host before the clock stops
            stream.wait_event(drained[(n - 1) % 2])

        e2e_steps(2)
        torch.cuda.synchronize()
        n_e2e = max(3, args.steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        e0.record(stream)
        e2e_steps(n_e2e)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if world > 1:
            t = torch.tensor([ms], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        e2e = {"value": s.pixels * world * n_e2e / (ms * 1e-3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": n_e2e, "cuda_graph": use_graph,
               "note": "inputs and results double-buffered: the next step's host-to-device copies and the "
                       "previous step's device-to-host copies overlap this step"}
    return cached, e2e


# the other workloads, measured beside the main one at one GPU (sub-records of the line)
SUB_WORKLOADS = ("large", "ragged", "textured")


def ours(args, rank, world, local_rank):
    import torch

    from paper_2204_01386_gb300 import binding as B

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    lib = B.load()
    peaks = measured_peaks(lib, dev)
    try:
        hbm_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
        hbm_src = "MEASURED_PEAKS.json hbm_gbs (copy, measured)"
    except Exception:
        hbm_peak, hbm_src = 6800.0, "fallback 6.8 TB/s"
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    s = workload_scene(rank, world, n_views=args.views, workload=args.workload)
    rec, st = measure(s, args, dev, world, rank, dist, flush, peaks, hbm_peak, main=True)
    cached, e2e = extra_legs(s, args, dev, world, dist, flush, st)
    del st
    torch.cuda.empty_cache()

    subs = {}
    if world == 1 and not args.no_sub and args.workload == "multiview":
        for w in SUB_WORKLOADS:
            ss = workload_scene(0, 1, workload=w)
            sub_args = argparse.Namespace(**vars(args))
            sub_args.workload = w
            srec, sst = measure(ss, sub_args, dev, 1, 0, None, flush, peaks, hbm_peak,
                                n_steps=max(5, args.steps // 2))
            del sst
            torch.cuda.empty_cache()
            srec["workload"] = workload_desc(ss, w)["workload"]
            srec["pixels_per_step"] = ss.pixels
            subs[w] = srec

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # all host threads (one view each at a time), and one thread
        threads = host_threads()
        nvm = min(2 * threads, len(s.views))
        pxm, dtm = time_oracle(s, nvm, threads=threads)
        nv = min(args.cpu_views, len(s.views))
        px, dt = time_oracle(s, nv)
        cpu = {"value": pxm / dtm / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{nvm} of {len(s.views)} views, forward + adjoint, FP64 C oracle, {threads} host threads "
                         f"(views concurrently), {dtm:.1f} s",
               "single_thread": {"value": px / dt / 1e6, "cores": 1,
                                 "sample": f"{nv} of {len(s.views)} views, {dt:.1f} s"}}
    if rank == 0:
        cfg = workload_desc(s, args.workload)
        cfg.update({"texgrad": ["atomics", "texel-space gather", "inverse UV"][args.texgrad], "tile": rec["tile"],
                    "schedule": rec["schedule"], "autotuned": rec["autotuned"], "list_cap": rec["list_cap"],
                    "cuda_graph": rec["cuda_graph"], "ranks": world,
                    "parallelism": "views sharded over %d rank(s), gradients all-reduced" % world})
        roofline = dict(rec["roofline"])
        roofline["hbm_peak_source"] = hbm_src
        line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": cfg, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(rec["gpu_launches_per_step"] * args.steps), "clocks": rec["clocks"],
                "plain_per_view": rec["plain_per_view"], "cached_geometry": cached, "peaks_measured": peaks,
                "workloads": subs or None}
        print(json.dumps(line), flush=True)


def _rank_entry(local_rank, world, port, argv):
    """One rank of a self-launched multi-GPU run (bench.py --gpus N without a launcher)."""
    os.environ.update({"RANK": str(local_rank), "LOCAL_RANK": str(local_rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    run_rank(parse_args(argv))


def spawn_ranks(n, argv, entry=_rank_entry):
    """Starts n ranks of this script on this node (one process per GPU, 'spawn' start),
    as torch.distributed.run would, and waits for them."""
    import socket

    import torch.multiprocessing as mp
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    mp.start_processes(entry, args=(n, port, argv), nprocs=n, join=True, start_method="spawn")


def run_rank(args):
    """Runs this process's rank: the reference arm, or ours over NCCL (gloo with
    --backend gloo, which only the CPU test of the launch path uses)."""
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.backend == "nccl":
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        else:
            dist.init_process_group(args.backend)
    try:
        if args.backend == "gloo":
            launch_selfcheck(args, rank, world)
        else:
            ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


def launch_selfcheck(args, rank, world):
    """The launch path without a GPU (gloo): every rank takes its views of the workload,
    joins the barriers of the timed region and the max-over-ranks reduction of the time,
    all-reduces a per-rank gradient, and rank 0 prints one line."""
    import torch
    import torch.distributed as dist
    s = workload_scene(rank, world, n_views=args.views, res=24, workload="multiview")
    g = torch.full((3,), float(rank + 1), dtype=torch.float64)
    dist.barrier()
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(g)
    dist.barrier()
    if rank == 0:
        print(json.dumps({"n_gpus": world, "views_rank0": len(s.views), "tmax": float(t.item()),
                          "grad_sum": g.tolist()}), flush=True)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-views", type=int, default=12)
    ap.add_argument("--views", type=int, default=None,
                    help="views per rank of the multiview (default 64) or large (default 8) workload")
    ap.add_argument("--tile", type=int, default=0, choices=[0, 16, 32],
                    help="screen tile edge in pixels (0: chosen by the autotuner)")
    ap.add_argument("--schedule", type=int, default=0, choices=[0, 1, 2],
                    help="per-tile kernel: 1 one CTA per tile, 2 persistent longest-first (0: autotuner)")
    ap.add_argument("--no-cached", action="store_true", help="skip the static-geometry (cached layers) step")
    ap.add_argument("--no-sub", action="store_true", help="skip the large / ragged / textured sub-records")
    ap.add_argument("--workload", default="multiview", choices=WORKLOADS)
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--texgrad", type=int, default=0, choices=[0, 1, 2],
                    help="texel gradient: 0 atomics, 1 deterministic texel gather, 2 inverse UV (approximate)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--backend", default="nccl", choices=["nccl", "gloo"],
                    help="process-group backend of a multi-rank run (gloo only checks the launch path on CPU)")
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)
    return args


def main():
    argv = sys.argv[1:]
    args = parse_args(argv)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # no launcher: start one rank per GPU here
        spawn_ranks(args.gpus, argv)
        return
    run_rank(args)


if __name__ == "__main__":
    main()
