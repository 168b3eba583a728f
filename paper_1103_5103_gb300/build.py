"""Build libwilson.so (sm_103a) in-tree with nvcc: one translation unit per
csrc/*.cu file, compiled in parallel, linked against the shared CUDA runtime
so the library and PyTorch use the same runtime instance; and the
bounds-checked libwilson_checked.so from the same sources with WL_CHECKED."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libwilson.so")
OBJ = os.path.join(ROOT, "_build")
# the bounds-checked build: every internal site index tested (WL_CHECKED)
OUT_CHECKED = os.path.join(HERE, "libwilson_checked.so")
OBJ_CHECKED = os.path.join(ROOT, "_build", "checked")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"),
         "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(obj: str, deps: list[str]) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, checked: bool = True) -> str:
    """Compile every csrc/*.cu for sm_103a and link libwilson.so, and (checked)
    the bounds-checked libwilson_checked.so beside it, all translation units
    of both compiled in parallel; returns the path of libwilson.so."""
    nvcc = _nvcc()
    headers = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    variants = [(OBJ, OUT, [])] + ([(OBJ_CHECKED, OUT_CHECKED, ["-DWL_CHECKED"])] if checked else [])
    procs, links = [], []
    for objdir, out, defs in variants:
        os.makedirs(objdir, exist_ok=True)
        objs = []
        for src in sources():
            obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
            objs.append(obj)
            if not _stale(obj, [src] + headers):
                continue
            cmd = [nvcc] + ARCH + FLAGS + defs + ["-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        links.append((out, objs))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(f"{s}\n{o}" for s, o in failed))
    for out, objs in links:
        if _stale(out, objs):
            tmp = out + ".tmp%d" % os.getpid()
            cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
            subprocess.check_call(cmd)
            os.replace(tmp, out)
    return OUT


if __name__ == "__main__":
    print(build(verbose=True))
