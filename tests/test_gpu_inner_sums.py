"""FP32 inner-iteration sums against FP64 ones, on the 4^3x8 and 16^3x32
solves.

The default library sums the inner iteration's BiCGStab inner products and
norms over FP32 and FP16 fields in FP32 per thread (12 complex terms) and per
warp (32 sites), then in FP64 across warps. The build variant
libstochq_sums64.so (SQ_INNER_SUMS_FP64) sums them in FP64 from the thread
level up. Both builds solve the same sources in a child process each
(STOCHQ_LIBRARY selects the variant); the test checks that

* each library reports the precision it was built with (sq_inner_sum_bits);
* every source converges to 1e-10 in both, with iteration counts that agree
  to within 2 iterations or 5% (FP32 inner) / 10% (FP16 inner);
* the solutions agree with each other to 1e-9 (relative L2) and with the FP64
  oracle: every 4^3x8 source against the oracle's solution, and at 16^3x32
  the oracle's operator residual on two sources and one source against the
  oracle's solution, all to 1e-9.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from gpu_helpers import rel
from paper_1405_4524_gb300 import build as sqbuild
from paper_1405_4524_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
from paper_1405_4524_gb300 import inputs
from paper_1405_4524_gb300 import stochq as sq
out = sys.argv[1]
res = {"bits": sq.sq_inner_sum_bits()}
arrays = {}
for name in ("4x4x4x8", "16x16x16x32"):
    spec = inputs.WORKLOADS[name]
    U = inputs.make_links(spec["dims"], spec["eps"], spec["link_seed"])
    eta = inputs.make_z4(spec["dims"], spec["n_rhs"], spec["src_seed"])
    ctx = sq.sq_create(spec["dims"], -1)
    try:
        sq.sq_load_gauge(ctx, U, 12)
        for prec in (sq.SQ_F32, sq.SQ_F16):
            sol = np.zeros_like(eta)
            st, stats = sq.sq_solve(ctx, spec["kappa"], spec["csw"], eta, sol, spec["n_rhs"], 1e-10,
                                    sq.sq_default_params(inner_prec=prec))
            key = f"{name}_{prec}"
            res[key] = [dict(status=s["status"], iterations=s["iterations"], updates=s["updates"],
                             true_residual=s["true_residual"]) for s in stats]
            arrays[key] = sol
    finally:
        sq.sq_destroy(ctx)
np.savez(out + ".npz", **arrays)
with open(out + ".json", "w") as f:
    json.dump(res, f)
"""


def run_child(tmp_path, tag, library):
    env = dict(os.environ)
    env.pop("STOCHQ_LIBRARY", None)
    if library is not None:
        env["STOCHQ_LIBRARY"] = library
    out = str(tmp_path / tag)
    r = subprocess.run([sys.executable, "-c", CHILD, out], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    with open(out + ".json") as f:
        meta = json.load(f)
    return meta, dict(np.load(out + ".npz"))


@pytest.fixture(scope="module")
def runs(tmp_path_factory):
    tmp = tmp_path_factory.mktemp("sums")
    variant = sqbuild.build(variant="sums64")
    return run_child(tmp, "fp32sums", None), run_child(tmp, "fp64sums", variant)


def test_builds_report_their_sum_precision(runs):
    (m32, _), (m64, _) = runs
    assert m32["bits"] == 32 and m64["bits"] == 64


@pytest.mark.parametrize("name", ["4x4x4x8", "16x16x16x32"])
@pytest.mark.parametrize("prec", [1, 2])
def test_iterations_and_solutions_agree(runs, name, prec):
    (m32, s32), (m64, s64) = runs
    key = f"{name}_{prec}"
    a, b = m32[key], m64[key]
    for k, (x, y) in enumerate(zip(a, b)):
        assert x["status"] == 0 and y["status"] == 0, (k, x, y)
        assert x["true_residual"] <= 1e-10 and y["true_residual"] <= 1e-10, (k, x, y)
        # FP16 fields round the recurrence at 2^-11, and a source whose final
        # check misses 1e-10 is resumed with a tighter target: wider bound
        frac = 0.05 if prec == 1 else 0.10
        assert abs(x["iterations"] - y["iterations"]) <= max(2, frac * y["iterations"]), (k, x, y)
        assert rel(s32[key][k], s64[key][k]) <= 1e-9, k
    print(key, "iterations FP32 sums", [x["iterations"] for x in a], "FP64 sums", [y["iterations"] for y in b])


@pytest.mark.parametrize("prec", [1, 2])
def test_small_solutions_match_oracle(runs, prec):
    (_, s32), (_, s64) = runs
    spec = inputs.WORKLOADS["4x4x4x8"]
    U = inputs.make_links(spec["dims"], spec["eps"], spec["link_seed"])
    F = oracle.field_strength(U)
    eta = inputs.make_z4(spec["dims"], spec["n_rhs"], spec["src_seed"])
    key = f"4x4x4x8_{prec}"
    for k in range(spec["n_rhs"]):
        ref, _, res = oracle.solve(U, eta[k], spec["kappa"], spec["csw"], -1.0, tol=1e-13, F=F)
        assert res <= 1e-13
        assert rel(s32[key][k], ref) <= 1e-9 and rel(s64[key][k], ref) <= 1e-9, k


def test_large_solutions_match_oracle(runs):
    (_, s32), (_, s64) = runs
    spec = inputs.WORKLOADS["16x16x16x32"]
    U = inputs.make_links(spec["dims"], spec["eps"], spec["link_seed"])
    F = oracle.field_strength(U)
    eta = inputs.make_z4(spec["dims"], spec["n_rhs"], spec["src_seed"])
    kappa, csw = spec["kappa"], spec["csw"]
    for prec in (1, 2):
        key = f"16x16x16x32_{prec}"
        for k in (0, 9):
            for s in (s32, s64):
                r = eta[k] - oracle.apply_M(U, F, s[key][k], kappa, csw, -1.0)
                assert np.linalg.norm(r) / np.linalg.norm(eta[k]) <= 1e-10, (key, k)
    ref, _, res = oracle.solve(U, eta[5], kappa, csw, -1.0, tol=1e-12, F=F)
    assert res <= 1e-12
    for prec in (1, 2):
        key = f"16x16x16x32_{prec}"
        assert rel(s32[key][5], ref) <= 1e-9 and rel(s64[key][5], ref) <= 1e-9, key
