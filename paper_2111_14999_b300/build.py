"""Build libphoebe_gpu.so (sm_103a) in-tree with nvcc.

Usage: python -m paper_2111_14999_b300.build [--force]
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libphoebe_gpu.so")
SOURCES = ["api.cu", "pipeline.cu", "bands.cu", "couple_fp64.cu", "tc_gemm.cu", "noalloc.cu", "sampler.cu", "generic.cu", "batch.cu", "mlp_tc.cu", "transport.cu", "selftest.cu", "dft.cu", "dft_s1.cu", "threeph.cu"]
HEADERS = ["common.cuh", "kernels.cuh", "pipeline.h", "tc.h", "tc_ptx.cuh", "sampler.h", "generic.h", "mlp_tc.h", "dft.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "phoebe_gpu.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    srcs = [os.path.join(CSRC, f) for f in SOURCES]
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "--shared", "-Xcompiler", "-fPIC", "-Xlinker", "--no-undefined",
           "-Xptxas", "-v" if verbose else "-O3", "-o", LIB + ".tmp", *srcs]
    proc = subprocess.run(cmd, capture_output=True, text=True)
    if proc.returncode != 0:
        sys.stderr.write(proc.stdout + proc.stderr)
        raise RuntimeError("nvcc failed building libphoebe_gpu.so")
    if verbose:
        sys.stderr.write(proc.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
