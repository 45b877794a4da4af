"""Time the even-odd clover dslash on one lattice, for choosing and saving
launch shapes: ``python -m paper_1405_4524_gb300.dslash_bench --lattice
16x16x16x32 --prec f32 --n 16 [--shape tile:4,2,2,8,2 | site:64,2,0]
[--emulated] [--reps 10]``. Prints one JSON line: the shape used (the
autotuner's when none is given), microseconds per launch (CUDA events) and
the algorithmic GB/s (links and clover blocks once, every source's input
and output spinor once per launch). Synthetic inputs: the workload link
generator (eps 0.25) and Gaussian spinors.
"""

from __future__ import annotations

import argparse
import json

import numpy as np


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--lattice", default="16x16x16x32")
    p.add_argument("--prec", default="f32", choices=["f64", "f32", "f16"])
    p.add_argument("--n", type=int, default=16)
    p.add_argument("--shape", default="", help="tile:by,bz,bt,sg,nbuf or site:sx,ry,order")
    p.add_argument("--emulated", action="store_true", help="f64 fields in double-FP32 arithmetic")
    p.add_argument("--kappa", type=float, default=0.12)
    p.add_argument("--reps", type=int, default=10)
    a = p.parse_args(argv)
    import torch

    from . import inputs, stochq as sq

    dims = tuple(int(v) for v in a.lattice.split("x"))
    prec = {"f64": sq.SQ_F64, "f32": sq.SQ_F32, "f16": sq.SQ_F16}[a.prec]
    X, Y, Z, T = dims
    ctx = sq.sq_create(dims, -1)
    try:
        sq.sq_load_gauge(ctx, inputs.make_links(dims, 0.25, 1002), 12)
        sq.sq_build_clover(ctx, a.kappa, 1.0)
        if a.shape:
            kind, vals = a.shape.split(":")
            sq.sq_set_dslash_shape(ctx, prec, a.n, 1 if kind == "tile" else 0, [int(v) for v in vals.split(",")])
        fb = sq.sq_field_bytes(ctx, prec, a.n)
        bi, bo = (torch.zeros(fb, dtype=torch.uint8, device="cuda") for _ in range(2))
        g = torch.Generator(device="cuda").manual_seed(3)
        psi = torch.randn((a.n, T, Z, Y, X, 4, 3), dtype=torch.complex128, device="cuda", generator=g)
        sq.sq_pack_spinor(ctx, bi, psi, 1, prec, a.n)
        del psi
        flags = sq.SQ_DS_CLOVER_INV | (sq.SQ_DS_F64_EMULATED if a.emulated else 0)
        sq.sq_dslash_eo(ctx, bo, bi, None, 0, prec, a.n, flags | sq.SQ_DS_SYNC, 0.0)
        kind, shape = (None, None)
        if not a.emulated:
            kind, shape = sq.sq_get_dslash_shape(ctx, prec, a.n)
        for _ in range(2):
            sq.sq_dslash_eo(ctx, bo, bi, None, 0, prec, a.n, flags, 0.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(a.reps):
            sq.sq_dslash_eo(ctx, bo, bi, None, 0, prec, a.n, flags, 0.0)
        e1.record()
        torch.cuda.synchronize()
        us = 1000.0 * e0.elapsed_time(e1) / a.reps
    finally:
        sq.sq_destroy(ctx)
    vh = int(np.prod(dims)) // 2
    gauge = 8 * 144 + 576 if prec == sq.SQ_F64 else 8 * 48 + 288
    spin = {sq.SQ_F64: 384, sq.SQ_F32: 192, sq.SQ_F16: 104}[prec]
    byt = vh * (gauge + a.n * spin)
    out = {"lattice": a.lattice, "prec": a.prec, "emulated": a.emulated, "n": a.n,
           "kind": {0: "site", 1: "tile", None: "emulated"}[kind], "shape": list(shape) if shape else None,
           "us_per_launch": round(us, 2), "algorithmic_bytes": byt, "GB_per_s": round(byt / us / 1e3, 1)}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
