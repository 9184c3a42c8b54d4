"""Builds libsdirt.so (sm_103a) in-tree with nvcc.

The translation units are compiled in parallel into paper_2503_11213_gb300/_build
and linked against the shared CUDA runtime (the one PyTorch also loads).
build(checked=True) builds libsdirt_checked.so in _build_checked with
-DSD_CHECKED: the kernels test the indices they compute before using them
and record failures (sd_check_status); the binding loads it when the
environment sets SDIRT_CHECKED=1.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = BUILD / "libsdirt.so"
BUILD_CHECKED = PKG / "_build_checked"
LIB_CHECKED = BUILD_CHECKED / "libsdirt_checked.so"
SOURCES = ["lens_trace.cu", "render.cu", "render_bwd.cu", "render_map.cu", "render_tc.cu",
           "mlp.cu", "tune.cu", "abi.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the sdirt CUDA library cannot be built")


def _stale(lib: Path) -> bool:
    if not lib.exists():
        return True
    t = lib.stat().st_mtime
    deps = [CSRC / s for s in SOURCES] + list(CSRC.glob("*.cuh")) + \
        [PKG.parent / "include" / "sdirt.h", Path(__file__)]
    return any(d.exists() and d.stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> Path:
    out_dir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    if not force and not _stale(lib):
        return lib
    out_dir.mkdir(parents=True, exist_ok=True)
    cc = nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = out_dir / (Path(src).stem + ".o")
        objs.append(obj)
        cmd = [cc, *ARCH, *FLAGS, *(["-DSD_CHECKED"] if checked else []),
               "-I", str(PKG.parent / "include"), "-c", str(CSRC / src), "-o", str(obj)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{src}:\n{out.decode(errors='replace')}")
        elif verbose:
            print(out.decode(errors="replace"))
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = lib.with_suffix(f".{os.getpid()}.tmp")
    link = [cc, *ARCH, "-shared", "-cudart", "shared", "-o", str(tmp), *map(str, objs),
            "-Xlinker", "-rpath=/usr/local/cuda/lib64"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
