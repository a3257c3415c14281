"""Build libsgspm.so in-tree for sm_103a (B300) with nvcc.

    python -m paper_2606_28113_b300.build [--ptxas] [--force] [-j N]

The host code and small kernels (capi.cu) and the pass-kernel instantiations (k_*.cu) are
separate translation units, compiled in parallel and linked into one shared library written
next to this file and loaded by paper_2606_28113_b300.sgspm.  A unit is recompiled when any
source or header is newer than its object file.
"""
import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(HERE, "..", "include")
LIB = os.path.join(HERE, "libsgspm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]   # --ptxas adds -Xptxas -v


def sources():
    return ["capi.cu"] + sorted(os.path.basename(p) for p in glob.glob(os.path.join(CSRC, "k_*.cu")))


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _newest_input():
    files = glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]
    return max(os.path.getmtime(f) for f in files)


def build(verbose=False, ptxas_info=False, force=False, jobs=None):
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    newest = _newest_input()
    cmds, objs = [], []
    for src in sources():
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(obj)
        if not force and not ptxas_info and os.path.exists(obj) and os.path.getmtime(obj) >= newest:
            continue
        cmd = [nvcc(), *ARCH, *FLAGS, "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info:
            cmd[1:1] = ["-Xptxas", "-v"]
        cmds.append(cmd)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        return subprocess.run(cmd).returncode

    if cmds:
        with ThreadPoolExecutor(max_workers=jobs or os.cpu_count() or 4) as ex:
            codes = list(ex.map(run, cmds))
        if any(codes):
            raise RuntimeError("nvcc failed for: " + ", ".join(c[-3] for c, r in zip(cmds, codes) if r))
    if cmds or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc(), *ARCH, "-shared", "-o", LIB, *objs, "-lcudart"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    j = None
    if "-j" in sys.argv:
        j = int(sys.argv[sys.argv.index("-j") + 1])
    print(build(verbose=True, ptxas_info="--ptxas" in sys.argv, force="--force" in sys.argv, jobs=j))
