"""Build the CUDA libraries in-tree with nvcc for sm_103a (GB300).

* ``libgf2.so``      -- the C ABI of ``include/gf2.h`` (all method kernels);
* ``libgf2synth.so`` -- the seeded input generator of ``include/gf2_synth.h``.

Translation units compile in parallel; the static CUDA runtime is linked in so
the libraries load next to any PyTorch build. Run ``python -m
paper_1006_1744_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
OBJ = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-I" + os.path.join(ROOT, "include")] + ARCH

LIBS = {
    "libgf2.so": ["gf2_api.cu", "gf2_pls.cu", "gf2_rref.cu", "gf2_mul.cu", "gf2_mul_tc.cu", "gf2_prof.cu", "gf2_noalloc.cu", "gf2_rec.cu", "gf2_status.cu", "gf2_batch.cu", "gf2_tune.cu", "gf2_graph.cu", "gf2_strassen.cu", "gf2_sweep.cu", "gf2_pair.cu"],
    "libgf2synth.so": ["gf2_synth.cu"],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the GF(2) library")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, obj: str, verbose: bool) -> None:
    cmd = [nvcc(), "-c", src, "-o", obj] + NVCC_FLAGS
    if verbose:
        cmd += ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{res.stderr}")
    if verbose and res.stderr:
        sys.stderr.write(res.stderr)


def build(force: bool = False, verbose: bool = False) -> dict[str, str]:
    os.makedirs(OBJ, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    headers += [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]
    jobs = []
    for lib, srcs in LIBS.items():
        for s in srcs:
            src = os.path.join(CSRC, s)
            obj = os.path.join(OBJ, s.replace(".cu", ".o"))
            if force or _stale(obj, [src] + headers):
                jobs.append((src, obj))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            for f in [ex.submit(_compile, s, o, verbose) for s, o in jobs]:
                f.result()
    out = {}
    for lib, srcs in LIBS.items():
        objs = [os.path.join(OBJ, s.replace(".cu", ".o")) for s in srcs]
        target = os.path.join(HERE, lib)
        if force or _stale(target, objs):
            tmp = target + ".tmp"
            cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static"]
            res = subprocess.run(cmd, capture_output=True, text=True)
            if res.returncode != 0:
                raise RuntimeError(f"link of {lib} failed:\n{res.stderr}")
            os.replace(tmp, target)
        out[lib] = target
    return out


if __name__ == "__main__":
    for k, v in build(force="--force" in sys.argv, verbose="-v" in sys.argv).items():
        print(k, "->", v)
