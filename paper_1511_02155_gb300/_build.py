"""In-tree build of ``libtlbm.so`` (the C ABI of include/tlbm.h) for sm_103a.

Each storage format and lattice is its own translation unit, so that the FP64
units can be compiled without fused multiply-add contraction (``-fmad=false``),
which keeps their arithmetic in the same rounding steps as a plain IEEE
evaluation, while the FP32 and 16-bit units keep FMA; no two units instantiate
the same kernel.  The units compile in parallel and link with the static CUDA
runtime into one shared library next to this file.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libtlbm.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = {
    "tlbm_api.cu": [],
    "tlbm_f64_q9.cu": ["-fmad=false"],
    "tlbm_f64_q19.cu": ["-fmad=false"],
    "tlbm_f32_q9.cu": [],
    "tlbm_f32_q19.cu": [],
    "tlbm_f16_q9.cu": [],
    "tlbm_f16_q19.cu": [],
    "tlbm_bf16_q9.cu": [],
    "tlbm_bf16_q19.cu": [],
    "tlbm_noalloc.cu": [],
    "tlbm_wetting.cpp": [],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtlbm.so")


def _sources_digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, os.path.join(ROOT, "include")):
        for name in sorted(os.listdir(d)):
            with open(os.path.join(d, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    h.update(repr(sorted(UNITS.items())).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile and link libtlbm.so unless an up-to-date one exists."""
    digest = _sources_digest()
    stamp = LIB + ".sha256"
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    common = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-I", os.path.join(ROOT, "include"), *ARCH, *extra_flags]
    if verbose:
        common += ["-Xptxas", "-v"]
    procs = []
    objs = []
    for unit, flags in UNITS.items():
        obj = os.path.join(BUILD, os.path.splitext(unit)[0] + ".o")
        objs.append(obj)
        cmd = [cc, "-c", os.path.join(CSRC, unit), "-o", obj, *common, *flags]
        procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for unit, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append(f"--- {unit}\n{text}")
        elif verbose and text:
            sys.stderr.write(f"--- {unit}\n{text}")
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([cc, "-shared", *ARCH, "-o", tmp, *objs, "-cudart", "static"], check=True)
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
