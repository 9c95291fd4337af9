"""Build librs.so in-tree with nvcc for sm_103a (translation units compiled in
parallel; objects under paper_1010_1386_gb300/_build/).

    python -m paper_1010_1386_gb300.build [--force] [--verbose]
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "librs.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]
EXTRA = os.environ.get("RS_NVCC_EXTRA", "").split()  # experiments only
G1_CAPS = (8, 16, 24, 32, 40, 48, 56, 64, 72)


def _units():
    units = []
    for cap in G1_CAPS:
        units.append(("kernels_g1.cu", f"g1_c{cap}.o", [f"-DRS_G1_CAP={cap}"]))
    for src in ("g1_dispatch.cu", "kernels_g23.cu", "kernels_g3.cu", "engine.cu", "server.cu", "noalloc.cu",
                "autotune.cu", "kernels_g2ntt.cu", "kernels_g2t.cu", "kernels_g3m.cu", "kernels_g3l.cu",
                "kernels_yun.cu", "kernels_schur.cu", "probe.cu"):
        units.append((src, src.rsplit(".", 1)[0] + ".o", []))
    units.append(("planner.cpp", "planner.o", ["-x", "cu"]))
    units.append(("squarefree.cpp", "squarefree.o", ["-x", "cu"]))
    return units


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(os.path.dirname(PKG), "include", "rs.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, jobs=None):
    os.makedirs(BUILD, exist_ok=True)
    deps = _deps()
    cmds = []
    objs = []
    for src, obj, extra in _units():
        out = os.path.join(BUILD, obj)
        objs.append(out)
        if force or _stale(out, deps):
            cmds.append([NVCC] + ARCH + FLAGS + EXTRA + extra + ["-c", os.path.join(CSRC, src), "-o", out])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r

    jobs = jobs or min(len(cmds) or 1, os.cpu_count() or 4)
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        list(ex.map(run, cmds))
    if force or cmds or _stale(LIB, objs):
        tmp = LIB + ".tmp"
        run([NVCC] + ARCH + ["-shared", "-Xlinker", "--no-undefined", "-o", tmp] + objs)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
