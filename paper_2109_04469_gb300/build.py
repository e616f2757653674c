"""Build libpic.so (sm_103a) in-tree with nvcc: one translation unit per precision path plus
the C-ABI, compiled in parallel and linked into paper_2109_04469_gb300/_lib/libpic.so."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libpic.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
          "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math", "--expt-relaxed-constexpr"]
# FP64 kernels and the host constants that feed them: no contraction into FMAs, so each
# product and sum rounds as the step contract writes it.
UNITS = {
    "pic_fp64.cu": ["-fmad=false"],
    "pic_capi.cu": ["-fmad=false"],
    # statistical FP32 path: contraction allowed (its FP64 field solve uses explicit
    # round-to-nearest intrinsics)
    "pic_fp32.cu": [],
    # allocation-free field solve: same rounded FP64 operations as the FP64 path
    "pic_static.cu": ["-fmad=false"],
    # surrogate network: tcgen05 BF16 GEMMs and FP32 elementwise kernels
    "pic_mlp.cu": [],
}


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found")
    return exe


def _sources_newer_than(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".h")) and os.path.getmtime(os.path.join(d, f)) > t:
                return True
    return os.path.getmtime(__file__) > t


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    if not force and not _sources_newer_than(LIB):
        return LIB
    exe = nvcc()
    extra_env = os.environ.get("PIC_NVCC_FLAGS", "").split()  # tuning sweeps only
    procs = []
    objs = []
    for src, extra in UNITS.items():
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        cmd = [exe, *ARCH, *COMMON, *extra, *extra_env, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{src}:\n{out.decode(errors='replace')}")
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.run([exe, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
