"""Build libcluster.so (the C-ABI solver library) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libcluster.so")
PROBE_LIB = os.path.join(HERE, "libgather_probe.so")  # random-row gather probe (bench.py --workload rowrate)
SOURCES = ["solver.cu", "batch.cu", "server.cu", "objective_static.cu", "csr_build.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out.append(os.path.join(ROOT, "include", "cluster.h"))
    out.append(os.path.abspath(__file__))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False, out: str | None = None,
          defines: tuple = ()) -> str:
    """Compile every CUDA/C++ source of the library into one shared object.
    ``out``/``defines`` build a variant (e.g. ``("FC_MINB32=3",)``) elsewhere."""
    target = out or LIB
    if out is None and not defines and not force and up_to_date():
        return LIB
    cmd = [_nvcc(), "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-fvisibility=hidden", *ARCH, "-I", os.path.join(ROOT, "include")]
    if ptxas_v:
        cmd += ["-Xptxas", "-v"]
    cmd += [f"-D{d}" for d in defines]
    cmd += [os.path.join(CSRC, s) for s in SOURCES]
    cmd += ["-o", target + ".tmp", "-lcudart"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    if ptxas_v or verbose:
        sys.stderr.write(res.stderr)
    os.replace(target + ".tmp", target)
    return target


def build_probe(force: bool = False) -> str:
    """Compile the random-row gather probe (its own small library)."""
    src = os.path.join(CSRC, "probe_gather.cu")
    if not force and os.path.exists(PROBE_LIB) and os.path.getmtime(PROBE_LIB) >= os.path.getmtime(src):
        return PROBE_LIB
    cmd = [_nvcc(), "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-Xcompiler",
           "-fvisibility=hidden", *ARCH, src, "-o", PROBE_LIB + ".tmp", "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    os.replace(PROBE_LIB + ".tmp", PROBE_LIB)
    return PROBE_LIB


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas-v", action="store_true")
    ap.add_argument("--out", default=None)
    ap.add_argument("-D", dest="defines", action="append", default=[])
    a = ap.parse_args()
    print(build(force=a.force, verbose=True, ptxas_v=a.ptxas_v, out=a.out, defines=tuple(a.defines)))
    if a.out is None and not a.defines:
        print(build_probe(force=a.force))
