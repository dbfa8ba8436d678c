"""Build libswccl.so (the CUDA kernels and the C ABI) in-tree for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel) with
one ``-gencode arch=compute_103a,code=sm_103a``; the objects are linked into
``paper_1105_5804_gb300/_build/libswccl.so`` with the static CUDA runtime, so
the library depends on the driver only.  No torch headers are involved.

The same sources built with narrower labeling tiles (-DSWCCL_TILE_W=64 and
128; without the simple-cubic kernels, whose bricks need the 256-wide tile)
give libswccl_w64.so and libswccl_w128.so: the batch autotuner times a batch
in each and keeps the fastest.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libswccl.so")
TILE_WIDTHS = (256, 128, 64)          # 256: libswccl.so; others: libswccl_w<width>.so
CUBIC_SOURCES = ("k_cubic.cu", "swccl_cubic.cu")


def lib_path(tile_w=256):
    return LIB if tile_w == 256 else os.path.join(OUT_DIR, "libswccl_w%d.so" % tile_w)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills"]


def _nvcc():
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libswccl")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Build every library variant; returns the path of libswccl.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    headers = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(HERE, "..", "include", "*.h"))
    plans = []          # (library, objects)
    jobs = []
    for tw in TILE_WIDTHS:
        obj_dir = OUT_DIR if tw == 256 else os.path.join(OUT_DIR, "w%d" % tw)
        os.makedirs(obj_dir, exist_ok=True)
        defs = [] if tw == 256 else ["-DSWCCL_TILE_W=%d" % tw]
        objs = []
        for src in sources():
            if tw != 256 and os.path.basename(src) in CUBIC_SOURCES:
                continue
            obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
            objs.append(obj)
            if force or _stale(obj, [src] + headers):
                jobs.append([nvcc] + ARCH + FLAGS + defs + list(extra_flags) + ["-c", src, "-o", obj])
        plans.append((lib_path(tw), objs))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or r.returncode != 0:
                print(" ".join(cmd))
                print(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed for %s" % cmd[-3])
    for lib, objs in plans:
        if force or jobs or _stale(lib, objs):
            tmp = lib + ".tmp.%d" % os.getpid()
            cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                print(" ".join(cmd))
                print(r.stdout + r.stderr)
                raise RuntimeError("link of %s failed" % os.path.basename(lib))
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
