"""Build libstochq.so in-tree with nvcc for sm_103a (GB300).

Each translation unit under csrc/ is compiled in parallel, then linked into
``paper_1405_4524_gb300/libstochq.so``. A unit is recompiled only when its
source or a header changed. Usage: ``python -m paper_1405_4524_gb300.build``.

Build variants go to their own object folder and library:
``python -m paper_1405_4524_gb300.build --variant sums64`` builds
``libstochq_sums64.so``, in which the inner iteration's fused inner products
and norms accumulate in FP64 from the thread level up (SQ_INNER_SUMS_FP64);
the binding loads it when STOCHQ_LIBRARY names its path.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "libstochq.so")
BUILD = os.path.join(HERE, "_build")
VARIANTS = {"sums64": ["-DSQ_INNER_SUMS_FP64"]}

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libstochq")
    return p


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


def _compile(src: str, extra, bdir: str, cached: bool) -> str:
    obj = os.path.join(bdir, os.path.splitext(src)[0] + ".o")
    srcp = os.path.join(CSRC, src)
    newest = max([os.path.getmtime(srcp)] + [os.path.getmtime(h) for h in _headers()])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest and cached:
        return obj
    cmd = [nvcc(), "-c", srcp, "-o", obj, "-I", INCLUDE, *ARCH, *FLAGS, *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def library_path(variant: str | None = None) -> str:
    """Path of the default library, or of a named build variant."""
    return OUT if variant is None else os.path.join(HERE, f"libstochq_{variant}.so")


def build(verbose: bool = False, extra=(), variant: str | None = None) -> str:
    """Compile and link; extra flags always rebuild, a variant (a key of
    VARIANTS) builds in its own folder and is cached like the default."""
    if variant is not None and variant not in VARIANTS:
        raise ValueError(f"unknown build variant {variant!r}; known: {sorted(VARIANTS)}")
    flags = list(extra) + (VARIANTS[variant] if variant else [])
    bdir = BUILD if variant is None else f"{BUILD}_{variant}"
    out = library_path(variant)
    cached = not extra
    os.makedirs(bdir, exist_ok=True)
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, flags, bdir, cached), srcs))
    newest = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(out) or os.path.getmtime(out) < newest or not cached:
        cmd = [nvcc(), "-shared", *ARCH, "-o", out, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    if verbose:
        print(out)
    return out


if __name__ == "__main__":
    args = sys.argv[1:]
    variant = None
    if "--variant" in args:
        i = args.index("--variant")
        variant = args[i + 1]
        del args[i:i + 2]
    build(verbose=True, extra=args, variant=variant)
