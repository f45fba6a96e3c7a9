"""In-tree builds of the package's native libraries.

``libcc.so`` is the CUDA library behind the C-ABI in ``include/cc.h`` (sm_103a
only); ``inputs/libccgen.so`` is the host-side seeded input generator. Both are
compiled in place with nvcc / gcc, guarded by a file lock so that concurrent
test processes do not race, and rebuilt when a source is newer than the
library.
"""
from __future__ import annotations

import fcntl
import os
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
LIBCC = PKG / "libcc.so"
LIBGEN = PKG / "inputs" / "libccgen.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
              "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or Path(cand).exists()):
            return cand
    return "nvcc"


def _stale(target: Path, sources: list[Path]) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(s.stat().st_mtime > t for s in sources)


def _locked(fn):
    def wrapper(*a, **kw):
        lock = PKG / ".build.lock"
        with open(lock, "w") as fh:
            fcntl.flock(fh, fcntl.LOCK_EX)
            try:
                return fn(*a, **kw)
            finally:
                fcntl.flock(fh, fcntl.LOCK_UN)
    return wrapper


def _run(cmd: list[str]) -> None:
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")


def cc_sources() -> list[Path]:
    return sorted(CSRC.glob("*.cu")) + sorted(CSRC.glob("*.cuh")) + [INCLUDE / "cc.h"]


@_locked
def build_cc(force: bool = False) -> Path:
    """Compile every ``csrc/*.cu`` into ``libcc.so`` (one nvcc process per
    translation unit, run in parallel, then one link)."""
    srcs = cc_sources()
    if not force and not _stale(LIBCC, srcs):
        return LIBCC
    objdir = PKG / "_build"
    objdir.mkdir(exist_ok=True)
    procs, objs = [], []
    for cu in sorted(CSRC.glob("*.cu")):
        obj = objdir / (cu.stem + ".o")
        objs.append(obj)
        cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, "-I", str(INCLUDE), "-I", str(CSRC),
               "-c", str(cu), "-o", str(obj)]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                            stderr=subprocess.PIPE, text=True)))
    for cmd, p in procs:
        out, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(cmd)}\n{out}\n{err}")
    tmp = LIBCC.with_suffix(".so.tmp")
    _run([_nvcc(), *ARCH, "-shared", "-o", str(tmp), *map(str, objs)])
    os.replace(tmp, LIBCC)
    return LIBCC


@_locked
def build_gen(force: bool = False) -> Path:
    src = PKG / "inputs" / "gen.c"
    if not force and not _stale(LIBGEN, [src]):
        return LIBGEN
    tmp = LIBGEN.with_suffix(".so.tmp")
    _run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", str(src), "-o", str(tmp)])
    os.replace(tmp, LIBGEN)
    return LIBGEN
