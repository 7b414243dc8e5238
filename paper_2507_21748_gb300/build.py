"""Build libevx.so (the CUDA library behind include/evx.h) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_2507_21748_gb300/_lib/libevx.so``. No cmake, no torch extension
machinery: the library is a plain C-ABI shared object.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libevx.so")
SOURCES = ["evx_kernels.cu", "evx_fast.cu", "evx_fused.cu", "evx_runtime.cu", "evx_adjoint.cu", "evx_static.cu",
           "evx_nn.cu", "evx_nn_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _flags(debug_bounds=False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]
    if debug_bounds:
        f.append("-DEVX_BOUNDS_CHECK")
    return f


def _deps_mtime():
    m = 0.0
    for fn in os.listdir(CSRC):
        m = max(m, os.path.getmtime(os.path.join(CSRC, fn)))
    for h in ("evx.h", "evx_nn.h"):
        m = max(m, os.path.getmtime(os.path.join(HERE, "..", "include", h)))
    return m


LIB_BOUNDS = os.path.join(OUT_DIR, "libevx_bounds.so")


def build_lib(force=False, verbose=False, jobs=None, debug_bounds=False):
    """Build libevx.so, or with debug_bounds=True the bounds-checked
    libevx_bounds.so (-DEVX_BOUNDS_CHECK; objects in _lib/bounds/)."""
    sources = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    lib_path = LIB_BOUNDS if debug_bounds else LIB
    obj_dir = os.path.join(OUT_DIR, "bounds") if debug_bounds else OUT_DIR
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= _deps_mtime():
        return lib_path
    os.makedirs(obj_dir, exist_ok=True)
    nvcc = _nvcc()
    flags = _flags(debug_bounds)

    def compile_one(src):
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        cmd = [nvcc] + flags + ["-I", os.path.join(HERE, "..", "include"), "-c",
                                os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=jobs or len(sources)) as ex:
        objs = list(ex.map(compile_one, sources))
    tmp = lib_path + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build_lib(force="-f" in sys.argv, verbose=True))
