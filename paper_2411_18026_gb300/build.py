"""Compile the CUDA library ``libfds.so`` (sm_103a) in-tree.

Each ``csrc/*.cu`` translation unit is compiled in parallel with nvcc, then
linked into ``paper_2411_18026_gb300/libfds.so``.  Rebuilds only when a source
or header is newer than the library.  ``build(checked=True)`` builds the
bounds-checked variant ``libfds_checked.so`` (-DFDS_CHECKS: index-mapped
gathers and scatters check their indexes, fds_bounds_violations counts the
misses) from the same sources into its own object folder.
"""
import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfds.so")
OBJ_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libfds_checked.so")
ROOT = os.path.dirname(HERE)
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", os.path.join(ROOT, "include")]
# extra nvcc flags for experiments (e.g. -DFDS_FFP_TJ4=4); build(force=True) to rebuild
FLAGS += os.environ.get("FDS_NVCC_FLAGS", "").split()


def _deps():
    return (glob.glob(os.path.join(SRC, "*.cu")) + glob.glob(os.path.join(SRC, "*.cuh"))
            + [os.path.join(ROOT, "include", "fds.h"), os.path.abspath(__file__)])


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def _compile(cu, objdir=OBJ, extra=()):
    obj = os.path.join(objdir, os.path.basename(cu)[:-3] + ".o")
    cmd = [NVCC] + FLAGS + list(extra) + ["-c", cu, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (cu, r.stdout, r.stderr))
    return obj


def build(force=False, verbose=False, checked=False):
    lib, objdir = (LIB_CHECKED, OBJ_CHECKED) if checked else (LIB, OBJ)
    extra = ["-DFDS_CHECKS"] if checked else []
    if not force and not _stale(lib):
        return lib
    os.makedirs(objdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(SRC, "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda cu: _compile(cu, objdir, extra), srcs))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    if verbose:
        print("built", lib)
    return lib


if __name__ == "__main__":
    build(force=True, verbose=True)
