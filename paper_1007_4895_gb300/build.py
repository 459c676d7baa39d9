"""Builds liblbgb.so in-tree with nvcc for sm_103a (GB300).

The translation units compile in parallel, then link into one shared library next to
this file. Nothing is installed into site-packages.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbgb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["lb_api.cu", "lb_step.cu", "lb_step_st_f64.cu", "lb_step_st_f32.cu", "lb_step_st_f32dev.cu",
           "lb_step_st_f16.cu", "lb_step_st_bf16.cu", "lb_pair_f32.cu", "lb_pair_f32dev.cu", "lb_pair_f16.cu",
           "lb_pair_bf16.cu", "lb_ring_f32.cu", "lb_ring_f32dev.cu", "lb_ring_f16.cu", "lb_ring_bf16.cu",
           "lb_ring2_f32_q16.cu", "lb_ring2_f32_q36.cu", "lb_ring2_f32dev_q16.cu", "lb_ring2_f32dev_q36.cu", "lb_ring2_f16_q16.cu", "lb_ring2_f16_q36.cu", "lb_ring2_bf16_q16.cu", "lb_ring2_bf16_q36.cu",
           "lb_step3.cu", "lb_stream.cu", "lb_aux.cu", "lb_mlp.cu", "lb_noalloc.cu",
           "quadrature.cpp"]
# The paired-arithmetic layout (lb_pair.cuh) is held to the oracle's tolerance, not to
# the other layouts' bits, and is built with multiply-add contraction on.
CONTRACT = {"lb_pair_f32.cu", "lb_pair_f32dev.cu", "lb_pair_f16.cu", "lb_pair_bf16.cu", "lb_ring_f32.cu",
            "lb_ring_f32dev.cu", "lb_ring_f16.cu", "lb_ring_bf16.cu"} | {
                f"lb_ring2_{f}_q{q}.cu" for f in ("f32", "f32dev", "f16", "bf16") for q in (16, 36)}


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbgb.so")


def _deps() -> list[str]:
    out = []
    for d in (CSRC, os.path.join(os.path.dirname(HERE), "include")):
        for f in os.listdir(d):
            out.append(os.path.join(d, f))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps() + [os.path.abspath(__file__)])


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    # -fmad=false: no implicit multiply-add contraction. The step layouts evaluate the
    # same expressions in differently shaped code, and the compiler's choice of which
    # product to fuse depends on that shape; with contraction off every layout rounds
    # alike and the fused products are the explicit fma() calls of the source. The host
    # side likewise (-ffp-contract=off), so that host-computed constants are the same
    # on x86-64 and AArch64.
    common = ARCH + ["-O3", "-lineinfo", "-std=c++20", "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", CSRC,
                     "--expt-relaxed-constexpr", "-fmad=false"]
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        flags = [f for f in common if f != "-fmad=false"] + ["-fmad=true"] if src in CONTRACT else common
        cmd = [cc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    r = subprocess.run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
