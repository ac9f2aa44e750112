"""Build libmlq.so (the CUDA library behind include/mlq.h) in-tree.

Compiles for sm_103a only.  The two translation units are compiled in
parallel and linked with nvcc; the result lands in
``paper_2105_02007_gb300/lib/libmlq.so``.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libmlq.so")
INCLUDE = os.path.join(ROOT, "include")
# (source, extra flags, object name): the slab-solver kernels are compiled
# once per cluster size / inner precision so that the objects build in parallel
SOURCES = ([("mlq_api.cu", [], "mlq_api"), ("mlq_kl.cpp", [], "mlq_kl"), ("mlq_3d_inst.cu", ["-DMLQ_F64=0"], "mlq_3d_f32"),
            ("mlq_3d_inst.cu", ["-DMLQ_F64=1"], "mlq_3d_f64"),
            ("mlq_mesh.cu", [], "mlq_mesh"), ("mlq_estimator.cpp", [], "mlq_estimator"),
            ("mlq_locate.cu", [], "mlq_locate"), ("mlq_selftest.cu", [], "mlq_selftest")]
           + [("mlq_reg_inst.cu", [f"-DMLQ_CS={cs}"], f"mlq_reg_cs{cs}") for cs in (1, 2, 4, 8, 16)]
           + [("mlq_slab_inst.cu", [f"-DMLQ_F64={f}"], f"mlq_slab_f{64 if f else 32}") for f in (0, 1)])
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "mlq.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]

    def compile_one(item) -> str:
        src, flags, name = item
        obj = os.path.join(LIBDIR, name + ".o")
        cmd = [nvcc] + common + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd[1:1] = ARCH + ["-lineinfo", "-Xptxas", "-v" if verbose else "-O3"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose:
            sys.stderr.write(f"== {name}\n" + r.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
