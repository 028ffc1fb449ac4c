"""Build libparamap.so (the C-ABI library) for sm_103a with nvcc, in-tree.

    python paper_2512_22575_b300/build.py [--force] [--checked]

(run by path: importing the package loads the library, which this builds).

Each .cu translation unit compiles in parallel into _build/, then the
objects link into paper_2512_22575_b300/libparamap.so (CUDA runtime linked
statically, so the library needs only the driver at run time).
"""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libparamap.so")
LIB_CHECKED = os.path.join(PKG, "libparamap_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                  f"-I{INCLUDE}", f"-I{CSRC}", "--expt-relaxed-constexpr"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, verbose, checked=False):
    bdir = os.path.join(BUILD, "checked") if checked else BUILD
    obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) \
        + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]
    if not _stale(obj, [src] + headers):
        return obj
    cmd = ["nvcc", *NVFLAGS, *(["-DPM_BOUNDS_CHECK=1"] if checked else []), "-c", src, "-o", obj + ".tmp"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build libparamap.so, or with checked the bounds-checked variant
    libparamap_checked.so (PM_BOUNDS_CHECK: every field gather, shared-memory
    slot and output write of the iteration kernels checked against its
    extent; see include/paramap.h)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib, _deps()):
        return lib
    os.makedirs(os.path.join(BUILD, "checked") if checked else BUILD, exist_ok=True)
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, checked), srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = ["nvcc", *ARCH, "-shared", "-o", tmp, *objs]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
