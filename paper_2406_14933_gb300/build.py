"""In-tree build of the CUDA library ``libasx.so`` for sm_103a (GB300).

Each ``csrc/*.cu`` is compiled by nvcc in parallel (one ``-gencode``), then linked into
``paper_2406_14933_gb300/_build/libasx.so`` with the static CUDA runtime.  Nothing is
installed outside the repository.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libasx.so")
ROOT = os.path.dirname(HERE)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
           "--expt-relaxed-constexpr", f"-I{os.path.join(ROOT, 'include')}"]
# per-file flags: the FP64 step rounds every multiply and add as written
FILE_FLAGS = {"step_fp64.cu": ["-fmad=false"]}


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libasx.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
        os.path.join(ROOT, "include", "asx.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link ``libasx.so``; returns its path.  Raises on any compiler error."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *NVFLAGS, *FILE_FLAGS.get(os.path.basename(src), []), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        with open(obj + ".log", "w") as f:
            f.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        for o in objs:
            print(open(o + ".log").read())
    return LIB


LIB_CHECKED = os.path.join(BUILD, "libasx_bounds.so")


def build_checked() -> str:
    """The bounds-checked debug build ``libasx_bounds.so``: the step kernel compiled with
    ``-DASX_BOUNDS_CHECK`` (every shared-memory ring index and global store of its tiles
    checked; a violation is reported as ASX_EBOUNDS and the access skipped), linked with
    the ordinary objects.  Builds the ordinary library first; returns the path."""
    build()
    src = os.path.join(CSRC, "step_strip.cu")
    obj = os.path.join(BUILD, "step_strip_bounds.cu.o")
    r = subprocess.run([_nvcc(), *ARCH, *NVFLAGS, "-DASX_BOUNDS_CHECK", "-c", src, "-o", obj],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src} (bounds-checked):\n{r.stderr}")
    objs = [obj] + [os.path.join(BUILD, os.path.basename(s) + ".o") for s in _sources()
                    if os.path.basename(s) != "step_strip.cu"]
    tmp = LIB_CHECKED + f".tmp{os.getpid()}"
    r = subprocess.run([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"], capture_output=True,
                       text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed (bounds-checked):\n{r.stderr}")
    os.replace(tmp, LIB_CHECKED)
    return LIB_CHECKED


if __name__ == "__main__":
    print(build(force=True, verbose=True))
