"""Build ``libst.so`` (the C-ABI library) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
LIB = PKG / "libst.so"
SOURCES = ["st_api.cu", "st_cull.cu", "st_trace.cu", "st_prep.cpp", "st_noalloc.cu", "st_mlp.cu", "st_batch.cu",
           "st_dexel.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def needs_build() -> bool:
    if not LIB.exists():
        return True
    t = LIB.stat().st_mtime
    deps = list(CSRC.glob("*")) + [ROOT / "include" / "st.h"]
    return any(p.stat().st_mtime > t for p in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> Path:
    if not force and not needs_build():
        return LIB
    objs = []
    build_dir = ROOT / "_build"
    build_dir.mkdir(exist_ok=True)
    common = ["-O3", "-std=c++17", "-lineinfo", "-I", str(ROOT / "include"), "-I", str(CSRC),
              "-Xcompiler", "-fPIC,-ffp-contract=off", "--expt-relaxed-constexpr"]
    cmds = []
    for src in SOURCES:
        obj = build_dir / (src + ".o")
        cmd = [nvcc(), *ARCH, *common, "-c", str(CSRC / src), "-o", str(obj)]
        if ptxas_info and src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        cmds.append(cmd)
        objs.append(str(obj))
    # the sources compile independently: in parallel (the tracer's kernel
    # instances take most of the time)
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=min(len(cmds), os.cpu_count() or 1)) as ex:
        for r in ex.map(lambda c: subprocess.run(c, capture_output=ptxas_info), cmds):
            if ptxas_info:
                sys.stderr.write(r.stderr.decode(errors="replace"))
            if r.returncode != 0:
                raise subprocess.CalledProcessError(r.returncode, r.args)
    tmp = LIB.with_suffix(".so.tmp%d" % os.getpid())
    cmd = [nvcc(), *ARCH, "-shared", "-o", str(tmp), *objs]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
