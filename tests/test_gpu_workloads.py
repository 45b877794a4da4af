"""Full-size workloads on the GPU, in the configuration the benchmark runs
(autotuned dslash shape, CUDA graphs, default precision policy), checked on
outputs the FP64 oracle can compute:

* one dslash application (FP32 and FP16 fields, clover inverse + xpay) on
  the three large lattices, element by element against the oracle;
* 16^3x32, kappa 0.120, 16 Z4 sources, FP32 inner + FP64 reliable updates:
  every source reaches 1e-10 (the library's FP64 residual), the oracle's own
  M confirms it on sampled sources, and one source matches the oracle's
  solution to 1e-9;
* 24^3x48, kappa 0.122, 64 time-diluted sources, FP16 inner: residuals,
  oracle residual and pion correlator on sampled sources;
* 32^3x64, kappa 0.122, 24 sources, FP16-inner / FP64-outer defect
  correction: residuals, oracle residual on a sampled source;
* the heterogeneous batch: 96 sources on 16^3x32 and 24^3x48 at kappa
  0.118, 0.121, 0.124 in one batch.
"""

import numpy as np
import pytest

import oracle
from gpu_helpers import device_buffer, random_spinors, rel
from paper_1405_4524_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

_cache = {}


def lattice(name):
    if name not in _cache:
        spec = dict(inputs.WORKLOADS[name])
        U = inputs.make_links(spec["dims"], spec["eps"], spec["link_seed"])
        _cache[name] = (spec, U, oracle.field_strength(U), oracle.parity_field(spec["dims"]))
    return _cache[name]


def context(dims, U):
    from paper_1405_4524_gb300 import stochq as sq

    ctx = sq.sq_create(dims, -1)
    sq.sq_load_gauge(ctx, U, 12)
    return sq, ctx


def oracle_residual(U, F, psi, eta, kappa, csw):
    r = eta - oracle.apply_M(U, F, psi, kappa, csw, -1.0)
    return float(np.linalg.norm(r) / np.linalg.norm(eta))


@pytest.mark.parametrize("name", ["16x16x16x32", "24x24x24x48", "32x32x32x64"])
@pytest.mark.parametrize("prec,tol", [(1, 1e-6), (2, 5e-3)])
def test_dslash_full_size(name, prec, tol):
    spec, U, F, par = lattice(name)
    sq, ctx = context(spec["dims"], U)
    try:
        kappa, csw, a = spec["kappa"], spec["csw"], -spec["kappa"] ** 2
        sq.sq_build_clover(ctx, kappa, csw)
        n = 2
        psi = random_spinors(spec["dims"], n, 61)
        x = random_spinors(spec["dims"], n, 62)
        fb = sq.sq_field_bytes(ctx, prec, n)
        bin_, bx, bout = device_buffer(fb), device_buffer(fb), device_buffer(fb)
        sq.sq_pack_spinor(ctx, bin_, psi, 1, prec, n)
        sq.sq_pack_spinor(ctx, bx, x, 0, prec, n)
        Ainv = np.linalg.inv(oracle.clover_matrices(F, kappa, csw))
        want = [oracle.restrict(x[k] + a * oracle.site_apply(Ainv, oracle.hopping_eo(U, psi[k], 0, par, -1.0)),
                                par, 0) for k in range(n)]
        del Ainv
        # the autotuned shape, then each kernel forced: per-site and halo-tiled
        for force in [None, (0, (64, 2, 0)), (1, (4, 2, 2, 2, 2))]:
            if force is not None:
                sq.sq_set_dslash_shape(ctx, prec, n, *force)
            sq.sq_dslash_eo(ctx, bout, bin_, bx, 0, prec, n,
                            sq.SQ_DS_CLOVER_INV | sq.SQ_DS_XPAY | sq.SQ_DS_SYNC, a)
            got = np.zeros_like(psi)
            sq.sq_unpack_spinor(ctx, got, bout, 0, prec, n)
            for k in range(n):
                assert rel(got[k], want[k]) < tol, (force, k)
    finally:
        sq.sq_destroy(ctx)


def test_solve_16x16x16x32_fp32_reliable():
    name = "16x16x16x32"
    spec, U, F, par = lattice(name)
    sq, ctx = context(spec["dims"], U)
    try:
        eta = inputs.make_z4(spec["dims"], spec["n_rhs"], spec["src_seed"])
        sol = np.zeros_like(eta)
        st, stats = sq.sq_solve(ctx, spec["kappa"], spec["csw"], eta, sol, spec["n_rhs"], 1e-10,
                                sq.sq_default_params(inner_prec=sq.SQ_F32))
        assert st == 0
        assert all(s["status"] == 0 and s["true_residual"] <= 1e-10 for s in stats)
        for k in (0, 9):
            assert oracle_residual(U, F, sol[k], eta[k], spec["kappa"], spec["csw"]) <= 1e-10
        ref, it, res = oracle.solve(U, eta[5], spec["kappa"], spec["csw"], -1.0, tol=1e-13, F=F)
        assert res <= 1e-13
        assert rel(sol[5], ref) <= 1e-9
        # the plain FP64 solver reaches the same solution
        sol64 = np.zeros_like(eta[:2])
        sq.sq_solve(ctx, spec["kappa"], spec["csw"], eta[4:6], sol64, 2, 1e-10,
                    sq.sq_default_params(inner_prec=sq.SQ_F64))
        assert rel(sol64[1], ref) <= 1e-9
    finally:
        sq.sq_destroy(ctx)


def test_solve_24x24x24x48_fp16_time_diluted():
    name = "24x24x24x48"
    spec, U, F, par = lattice(name)
    sq, ctx = context(spec["dims"], U)
    try:
        n, T = spec["n_rhs"], spec["dims"][3]
        ts = [k % T for k in range(n)]
        eta = inputs.make_z4(spec["dims"], n, spec["src_seed"], ts)
        sol = np.zeros_like(eta)
        st, stats = sq.sq_solve(ctx, spec["kappa"], spec["csw"], eta, sol, n, 1e-10,
                                sq.sq_default_params(inner_prec=sq.SQ_F16))
        assert st == 0
        assert all(s["status"] == 0 and s["true_residual"] <= 1e-10 for s in stats)
        C = sq.sq_contract_pion(ctx, sol, n, ts)
        for k in (3, 50):
            assert oracle_residual(U, F, sol[k], eta[k], spec["kappa"], spec["csw"]) <= 1e-10
            assert np.allclose(C[k], oracle.pion_correlator(sol[k], ts[k]), rtol=1e-13)
    finally:
        sq.sq_destroy(ctx)


def test_solve_32x32x32x64_fp16_defect_correction():
    name = "32x32x32x64"
    spec, U, F, par = lattice(name)
    sq, ctx = context(spec["dims"], U)
    try:
        n = spec["n_rhs"]
        eta = inputs.make_z4(spec["dims"], n, spec["src_seed"])
        sol = np.zeros_like(eta)
        prm = sq.sq_default_params(inner_prec=sq.SQ_F16, outer=sq.SQ_OUTER_DEFECT, delta=1e-3)
        st, stats = sq.sq_solve(ctx, spec["kappa"], spec["csw"], eta, sol, n, 1e-10, prm)
        assert st == 0
        assert all(s["status"] == 0 and s["true_residual"] <= 1e-10 for s in stats)
        assert all(s["restarts"] >= 2 for s in stats)  # defect-correction cycles
        k = 17
        assert oracle_residual(U, F, sol[k], eta[k], spec["kappa"], spec["csw"]) <= 1e-10
    finally:
        sq.sq_destroy(ctx)


def test_batch_96_sources_two_lattices_three_kappas():
    from paper_1405_4524_gb300 import stochq as sq

    specA, UA, FA, _ = lattice("16x16x16x32")
    specB, UB, FB, _ = lattice("24x24x24x48")
    ctxA = sq.sq_create(specA["dims"], -1)
    ctxB = sq.sq_create(specB["dims"], -1)
    try:
        sq.sq_load_gauge(ctxA, UA, 12)
        sq.sq_load_gauge(ctxB, UB, 12)
        groups = []
        for gi, (ctx, spec) in enumerate([(ctxA, specA), (ctxB, specB)]):
            for ki, kappa in enumerate([0.118, 0.121, 0.124]):
                eta = inputs.make_z4(spec["dims"], 16, 3000 + 10 * gi + ki)
                groups.append(dict(ctx=ctx, kappa=kappa, c_sw=1.0, sources=eta,
                                   solutions=np.zeros_like(eta), n_rhs=16, tol=1e-10))
        st, stats = sq.sq_solve_batch(groups, sq.sq_default_params(inner_prec=sq.SQ_F16))
        assert st == 0 and len(stats) == 96
        assert all(s["status"] == 0 and s["true_residual"] <= 1e-10 for s in stats)
        its = [s["iterations"] for s in stats]
        # heavier kappa needs more iterations: retirement happens per source
        assert np.mean(its[32:48]) > np.mean(its[0:16])
        for gi, (U, F) in enumerate([(UA, FA), (UB, FB)]):
            g = groups[3 * gi + 2]
            assert oracle_residual(U, F, g["solutions"][7], g["sources"][7], g["kappa"], 1.0) <= 1e-10
    finally:
        sq.sq_destroy(ctxA)
        sq.sq_destroy(ctxB)
