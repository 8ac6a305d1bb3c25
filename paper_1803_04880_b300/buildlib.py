"""Build libfrag.so in-tree with nvcc for sm_103a (no GPU needed to build)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libfrag.so")
SOURCES = ["frag_api.cu", "tile_kernels.cu", "stream_kernels.cu", "cipher_kernels.cu", "fused_kernels.cu", "block_kernels.cu", "noalloc.cu", "server.cu"]
HEADERS = [os.path.join(ROOT, "include", "frag.h"), os.path.join(CSRC, "frag_internal.cuh")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC,-O2,-Wall",
    "-Xptxas", "-v",
    "-cudart", "shared",
    "-shared",
    "-I", os.path.join(ROOT, "include"),
    "-Xlinker", "-rpath=/usr/local/cuda/lib64",
]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + HEADERS + [__file__]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, out: str = LIB, defines=()) -> str:
    """Compile libfrag.so (or `out`, with extra -D `defines`) for sm_103a."""
    if out == LIB and not defines and not force and not _stale():
        return LIB
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = [NVCC] + FLAGS + ["-D" + d for d in defines] + ["-o", tmp] + \
        [os.path.join(CSRC, s) for s in SOURCES]
    res = subprocess.run(cmd, capture_output=True, text=True)
    log = os.path.join(HERE, "build.log")
    with open(log, "w") as f:
        f.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed (see %s)" % log)
    if verbose:
        sys.stdout.write(res.stderr)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
