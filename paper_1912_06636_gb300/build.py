"""Build libnao.so in-tree with nvcc for sm_103a (no torch involvement)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
SRC = PKG / "csrc"
LIBDIR = PKG / "lib"
LIB = LIBDIR / "libnao.so"
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2,-ffp-contract=off", f"-I{ROOT / 'include'}",
          f"-I{SRC}"]


def sources():
    return sorted(list(SRC.glob("*.cu")) + list(SRC.glob("*.cpp")))


def _compile(src: Path, obj: Path, extra):
    arch = ARCH if src.suffix == ".cu" else []  # .cpp files are host code compiled by nvcc's host compiler
    cmd = [NVCC, *arch, *COMMON, *extra, "-c", str(src), "-o", str(obj)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src.name}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(force: bool = False, verbose: bool = False, extra=None) -> Path:
    extra = list(extra or [])
    LIBDIR.mkdir(exist_ok=True)
    objdir = LIBDIR / "obj"
    objdir.mkdir(exist_ok=True)
    srcs = sources()
    headers = list(SRC.glob("*.h")) + list((ROOT / "include").glob("*.h"))
    newest = max(p.stat().st_mtime for p in srcs + headers + [Path(__file__)])
    if not force and LIB.exists() and LIB.stat().st_mtime >= newest:
        return LIB
    objs = [objdir / (s.stem + s.suffix.replace(".", "_") + ".o") for s in srcs]
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        logs = list(ex.map(lambda so: _compile(so[0], so[1], extra), zip(srcs, objs)))
    if verbose:
        for s, log in zip(srcs, logs):
            if log.strip():
                print(f"--- {s.name}\n{log}")
    tmp = str(LIB) + ".tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *map(str, objs), "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
