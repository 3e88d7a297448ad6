"""Build the HFX CUDA library in-tree: generate the per-class ERI sources, compile
every translation unit for sm_103a in parallel with nvcc, link libhfx.so."""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
GEN = os.path.join(CSRC, "generated")
OBJ = os.path.join(HERE, "_build")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libhfx.so")
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", GEN, "-I", INCLUDE]
# HFX_CHECKED=1: a diagnostic build whose kernels test every global index of
# the exchange-build path and report (printf) and skip out-of-range accesses.
if os.environ.get("HFX_CHECKED", "0") not in ("", "0"):
    FLAGS = FLAGS + ["-DHFX_CHECKED"]
# HFX_NVCC_FLAGS: extra nvcc flags (e.g. -DHFX_SHFL_REDUCE for the butterfly
# chunk reduction, -DHFX_SPLIT_SMEM_ACC for every FP32 split class's
# accumulators in shared memory, -DHFX_LOCKSTEP_MIN_FLOPS=... for the lockstep
# threshold, -DHFX_PT_MINB=... for the per-thread launch bound,
# -DHFX_PT_PREFETCH=0|1 for the ket prefetch of every per-thread class instead
# of the per-class choice, -DHFX_SPLIT64_MAX_WARPS=4 for 4-warp FP64 split
# blocks, -DHFX_LOCKSTEP64=0 for FP64 split kernels without lockstep rounds,
# -DHFX_WIDE_WARPS=8|12|16 and -DHFX_MID_WARPS_F32=... for the warps per
# lockstep block of the FP32 split classes); part of every object's digest.
FLAGS = FLAGS + os.environ.get("HFX_NVCC_FLAGS", "").split()


def _sources():
    import importlib.util
    spec = importlib.util.spec_from_file_location("gen_eri", os.path.join(CSRC, "gen_eri.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    gen.generate(GEN)
    tus = sorted(os.path.join(GEN, f) for f in os.listdir(GEN) if f.endswith(".cu"))
    return [os.path.join(CSRC, f) for f in ("hfx_core.cu", "hfx_noalloc.cu", "hfx_server.cu", "hfx_periodic.cu")] + tus


def _digest(src, extra):
    h = hashlib.sha256()
    h.update(" ".join(FLAGS + extra).encode())
    h.update(os.environ.get("HFX_COOP_MIN_ACC", "").encode())  # generator switches
    h.update(os.environ.get("HFX_VRR_ORDER", "").encode())
    own = [os.path.join(GEN, os.path.basename(src).replace("tu_", "cls_").replace(".cu", ".cuh"))]
    own = [p for p in own if os.path.exists(p)]
    if os.path.basename(src) == "hfx_core.cu":
        own = sorted(os.path.join(GEN, f) for f in os.listdir(GEN) if f.endswith(".cuh"))
    for path in [src] + own + extra_headers():
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def extra_headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    hs += [os.path.join(GEN, f) for f in ("class_table.h", "class_dispatch.h")]
    return sorted(hs)


def _compile(src):
    base = os.path.splitext(os.path.basename(src))[0]
    extra = []
    tag = _digest(src, extra)
    obj = os.path.join(OBJ, f"{base}.{tag}.o")
    if os.path.exists(obj):
        return obj, None
    cmd = [NVCC] + FLAGS + extra + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        return None, f"{' '.join(cmd)}\n{r.stdout}\n{r.stderr}"
    os.replace(obj + ".tmp", obj)
    return obj, None


def build(verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    srcs = _sources()
    workers = max(1, min(len(srcs), os.cpu_count() or 1))
    objs, errs = [], []
    # the heaviest classes first so the pool's tail is short
    srcs.sort(key=lambda p: -os.path.getsize(p.replace("tu_", "cls_").replace(".cu", ".cuh"))
              if "tu_" in p else 0)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        for obj, err in ex.map(_compile, srcs):
            if err:
                errs.append(err)
            else:
                objs.append(obj)
    if errs:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + sorted(objs)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    keep = set(objs)
    for f in os.listdir(OBJ):  # objects of earlier source versions
        path = os.path.join(OBJ, f)
        if path not in keep and f.endswith(".o"):
            os.remove(path)
    if verbose:
        print(f"built {LIB} from {len(objs)} objects")
    return LIB


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
