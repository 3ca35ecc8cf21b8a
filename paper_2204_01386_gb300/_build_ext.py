"""Builds libdressi.so in-tree with nvcc for sm_103a (no torch extension machinery:
the library exposes a plain C ABI)."""
import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libdressi.so")
SOURCES = ["dressi_setup.cu", "dressi_tile_fwd.cu", "dressi_tile_bwd.cu", "dressi_tile_ids.cu", "dressi_tile_cached.cu",
           "dressi_tile_extra_ids.cu", "dressi_tile_extra_bwd.cu", "dressi_tile_nmap_fwd.cu",
           "dressi_tile_nmap_cached.cu", "dressi_texgather.cu", "dressi_peak.cu", "dressi_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _flags(extra=()):
    return ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
                   "-Xptxas", "-warn-spills"] + list(extra)


def _stale(obj, deps):
    return not os.path.exists(obj) or any(os.path.getmtime(d) > os.path.getmtime(obj) for d in deps)


def build(force=False, verbose=False, ptxas_v=False):
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "dressi.h"))
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        if force or _stale(o, [s] + headers):
            extra = ["-Xptxas", "-v"] if ptxas_v else []
            jobs.append(([nvcc()] + _flags(extra) + ["-c", s, "-o", o], o))
    outs = []
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = [ex.submit(subprocess.run, cmd, capture_output=True, text=True) for cmd, _ in jobs]
            for (cmd, o), f in zip(jobs, futs):
                r = f.result()
                outs.append(r.stderr)
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed for {o}:\n{r.stderr}")
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc()] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    if verbose:
        for o in outs:
            print(o)
    return LIB


if __name__ == "__main__":
    import sys
    build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv)
