"""Build the CUDA library libeapdtw.so in-tree for sm_103a (GB300).

Each .cu file under csrc/ is compiled by its own nvcc process (in parallel),
then linked into paper_2010_05371_gb300/_build/libeapdtw.so.  A rebuild is
skipped when the library is newer than every source and header.

    python -m paper_2010_05371_gb300.build [--force] [--verbose-ptxas]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
# Developer knobs for tuning experiments: an alternative build directory and
# extra nvcc flags (e.g. -D overrides of compile-time parameters).
BUILD = os.environ.get("EAPDTW_BUILD_DIR") or os.path.join(PKG, "_build")
EXTRA_FLAGS = os.environ.get("EAPDTW_NVCC_FLAGS", "").split()
LIB = os.path.join(BUILD, "libeapdtw.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libeapdtw.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


# Sources compiled more than once, with the defines of each unit: each large
# kernel instantiation gets its own nvcc process (see the files' headers).
SPLIT_UNITS = {
    "search_wide.cu": [[]] + [[f"-DEAPDTW_UNIT_BAND={b}", f"-DEAPDTW_UNIT_LB={lb}", f"-DEAPDTW_UNIT_COST={c}"]
                              for (lb, c) in ((0, 0), (1, 0), (0, 1)) for b in (0, 1, 2)],
    "batch_wide.cu": [[]] + [[f"-DEAPDTW_UNIT_LEVEL={lv}", f"-DEAPDTW_UNIT_BAND={b}"] for lv in (4, 5) for b in (0, 1, 2)],
    "pair_kernel.cu": [[], ["-DEAPDTW_UNIT_PAIR_WIDE"]],
    "search_elastic.cu": [[], ["-DEAPDTW_UNIT_EBAND=0"], ["-DEAPDTW_UNIT_EBAND=1"]],
    "search_k.cu": [[f"-DEAPDTW_UNIT_K={k}"] for k in (32, 16, 8, 4)],
    "batch_k.cu": [[f"-DEAPDTW_UNIT_K={k}"] for k in (32, 16, 8, 4)],
}


def units():
    """(source, extra nvcc flags, object name) of every compile unit."""
    out = []
    for src in sources():
        base = os.path.basename(src)[:-3]
        for i, defs in enumerate(SPLIT_UNITS.get(os.path.basename(src), [[]])):
            out.append((src, defs, base + (f".u{i}" if i else "") + ".o"))
    return out


def _inputs():
    files = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    files += glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    common = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr", *EXTRA_FLAGS]
    if verbose_ptxas:
        common += ["-Xptxas", "-v"]
    objs = []
    cmds = []
    for src, defs, name in units():
        obj = os.path.join(BUILD, name)
        objs.append(obj)
        cmds.append(common + defs + ["-c", src, "-o", obj])
    # the longest units first, so that they do not finish last
    order = {"search_wide": 0, "batch_wide": 1, "search_k": 2, "pair_kernel": 3, "search_elastic": 4, "batch_k": 5}
    cmds.sort(key=lambda c: order.get(os.path.basename(c[-1]).split(".")[0], 9))

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, p

    jobs = jobs or min(len(cmds), os.cpu_count() or 4)
    failed = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        for cmd, p in ex.map(run, cmds):
            out = (p.stdout + p.stderr).strip()
            if out and (verbose_ptxas or p.returncode != 0):
                print(out, file=sys.stderr)
            if p.returncode != 0:
                failed.append(cmd[-3])
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(failed))
    tmp = LIB + f".{os.getpid()}.tmp"
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    p = subprocess.run(link, capture_output=True, text=True)
    if p.returncode != 0:
        print(p.stdout + p.stderr, file=sys.stderr)
        raise RuntimeError("link of libeapdtw.so failed")
    os.replace(tmp, LIB)
    return LIB


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose-ptxas", action="store_true")
    args = ap.parse_args()
    print(build(force=args.force, verbose_ptxas=args.verbose_ptxas))


if __name__ == "__main__":
    main()
