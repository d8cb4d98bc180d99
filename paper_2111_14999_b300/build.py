"""Build libphoebe_gpu.so (sm_103a) in-tree with nvcc.

Each translation unit is compiled to an object under ``_build/`` (in parallel, only
when its source or a header is newer than the object), then the objects are linked
into the shared library next to this file.

Usage: python -m paper_2111_14999_b300.build [--force] [-v]
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(os.path.dirname(HERE), "_build")
LIB = os.path.join(HERE, "libphoebe_gpu.so")
SOURCES = ["api.cu", "pipeline.cu", "bands.cu", "couple_fp64.cu", "tc_gemm.cu", "noalloc.cu", "sampler.cu", "generic.cu",
           "batch.cu", "mlp_tc.cu", "transport.cu", "selftest.cu", "dft.cu", "dft_s1.cu", "dft64.cu", "threeph.cu"]
HEADERS = ["common.cuh", "kernels.cuh", "pipeline.h", "tc.h", "tc_ptx.cuh", "sampler.h", "generic.h", "mlp_tc.h", "dft.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _headers():
    hs = [os.path.join(CSRC, f) for f in HEADERS]
    hs.append(os.path.join(os.path.dirname(HERE), "include", "phoebe_gpu.h"))
    return [h for h in hs if os.path.exists(h)]


def _obj(src: str) -> str:
    return os.path.join(OBJ, os.path.splitext(src)[0] + ".o")


def _stale_obj(src: str, force: bool) -> bool:
    o = _obj(src)
    if force or not os.path.exists(o):
        return True
    t = os.path.getmtime(o)
    return any(os.path.getmtime(d) > t for d in [os.path.join(CSRC, src), *_headers()])


def _compile(src: str, verbose: bool):
    cmd = [nvcc(), *ARCH, *FLAGS, "-Xptxas", "-v" if verbose else "-O3", "-c", os.path.join(CSRC, src),
           "-o", _obj(src) + ".tmp"]
    proc = subprocess.run(cmd, capture_output=True, text=True)
    if proc.returncode == 0:
        os.replace(_obj(src) + ".tmp", _obj(src))
    return src, proc


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    todo = [s for s in SOURCES if _stale_obj(s, force)]
    if todo:
        with ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
            results = list(ex.map(lambda s: _compile(s, verbose), todo))
        bad = [(s, p) for s, p in results if p.returncode != 0]
        for s, p in results:
            if verbose or p.returncode != 0:
                sys.stderr.write(p.stdout + p.stderr)
        if bad:
            raise RuntimeError("nvcc failed on " + ", ".join(s for s, _ in bad))
    objs = [_obj(s) for s in SOURCES]
    if not todo and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(o) for o in objs):
        return LIB
    cmd = [nvcc(), *ARCH, "--shared", "-Xcompiler", "-fPIC", "-Xlinker", "--no-undefined", "-o", LIB + ".tmp",
           *objs]
    proc = subprocess.run(cmd, capture_output=True, text=True)
    if proc.returncode != 0:
        sys.stderr.write(proc.stdout + proc.stderr)
        raise RuntimeError("nvcc failed linking libphoebe_gpu.so")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
