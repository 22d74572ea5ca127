"""Build of the CUDA C-ABI library ``libholo.so`` for sm_103a (GB300), in-tree.

Every ``csrc/*.cu`` translation unit is compiled by nvcc in parallel into ``_build/``
and linked into ``paper_2004_04049_gb300/libholo.so`` against the shared CUDA runtime
(the same ``libcudart.so.13`` PyTorch loads, so device pointers and streams are shared).
A unit is rebuilt only when it or a header is newer than its object file.
"""

import concurrent.futures
import glob
import os
import shutil
import subprocess
import sys

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG_DIR)
CSRC = os.path.join(PKG_DIR, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build", "holo")
LIB = os.path.join(PKG_DIR, "libholo.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I", INCLUDE, "-I", CSRC]


def nvcc_path():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libholo.so")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(src, obj, header_mtime):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return os.path.getmtime(src) > t or header_mtime > t


def build(verbose=False, extra_flags=(), jobs=None):
    """Compile and link libholo.so; returns its path. Raises RuntimeError on failure."""
    nvcc = nvcc_path()
    os.makedirs(BUILD, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    header_mtime = max([os.path.getmtime(h) for h in _headers()] + [0.0])
    objs = []
    todo = []
    for src in sources:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if _stale(src, obj, header_mtime) or extra_flags:
            todo.append((src, obj))

    def compile_one(item):
        src, obj = item
        cmd = [nvcc, "-c", src, "-o", obj] + ARCH + NVCC_FLAGS + list(extra_flags)
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r.returncode, r.stdout + r.stderr

    jobs = jobs or min(len(todo), os.cpu_count() or 4) or 1
    with concurrent.futures.ThreadPoolExecutor(max_workers=jobs) as ex:
        for src, rc, out in ex.map(compile_one, todo):
            if verbose and out.strip():
                print(out, flush=True)
            if rc != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{out}")
    newest = max(os.path.getmtime(o) for o in objs)
    if todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        # --no-undefined: a symbol one translation unit declares and no other defines
        # fails the build here rather than the dlopen
        cmd = [nvcc, "-shared", "-o", LIB] + objs + ARCH + ["-cudart", "shared",
                                                            "-Xlinker", "-rpath,/usr/local/cuda/lib64",
                                                            "-Xlinker", "--no-undefined"]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of libholo.so failed:\n{r.stdout}{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
