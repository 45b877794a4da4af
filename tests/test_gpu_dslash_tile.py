"""GPU parity of the halo-tiled dslash (csrc/sq_dslash_tile.cu) against the
FP64 oracle, through the C ABI, with every tile shape forced by
sq_set_dslash_shape: FP32 and FP16 fields, with and without A^-1 and xpay,
both output parities, ragged source groups, ring depths 2 and 3, both time
boundary conditions; solves whose inner dslash is the tiled kernel; the
full-size FP16 lattice against the per-site kernel; and the bounded wait
running out.

Tolerances (relative L2 per source): FP32 1e-6, FP16 5e-3.
"""

import numpy as np
import pytest

import oracle
from gpu_helpers import Setup, device_buffer, random_spinors, rel
from test_tile_plan_model import shapes

pytestmark = pytest.mark.gpu

TOL = {1: 1e-6, 2: 5e-3}

# (dims, t_bc): X/2 = 2, 4, 8; a 2-wide y and z (halo rows that wrap onto
# the tile itself); periodic time
LATTICES = [((4, 4, 4, 8), -1), ((8, 4, 4, 8), -1), ((16, 4, 2, 4), 1), ((8, 2, 2, 16), -1)]


@pytest.fixture(scope="module", params=LATTICES, ids=lambda d: "x".join(map(str, d[0])) + f"_bc{d[1]}")
def setup(request):
    dims, t_bc = request.param
    s = Setup(dims, eps=0.4, seed=13, t_bc=t_bc)
    yield s
    s.close()


def oracle_dslash(s, psi_in, x, p_out, kappa, csw, clover, xpay, a):
    w = oracle.hopping_eo(s.U, psi_in, p_out, s.par, s.t_bc)
    if clover:
        w = oracle.site_apply(s.Ainv(kappa, csw), w)
    if xpay:
        w = x + a * w
    return oracle.restrict(w, s.par, p_out)


def run_dslash(s, prec, n, psi, x, p_out, flags, a):
    sq = s.sq
    fb = sq.sq_field_bytes(s.ctx, prec, n)
    bin_, bx, bout = device_buffer(fb), device_buffer(fb), device_buffer(fb)
    sq.sq_pack_spinor(s.ctx, bin_, psi, 1 - p_out, prec, n)
    sq.sq_pack_spinor(s.ctx, bx, x, p_out, prec, n)
    sq.sq_dslash_eo(s.ctx, bout, bin_, bx if flags & sq.SQ_DS_XPAY else None, p_out, prec, n,
                    flags | sq.SQ_DS_SYNC, a)
    got = np.zeros_like(psi)
    sq.sq_unpack_spinor(s.ctx, got, bout, p_out, prec, n)
    return got


def tile_shapes(dims, prec, limit=None):
    out = shapes(dims, "f16" if prec == 2 else "f32")
    return out if limit is None else out[:: max(1, len(out) // limit)][:limit]


@pytest.mark.parametrize("prec", [1, 2])
def test_every_tile_shape(setup, prec):
    s = setup
    sq = s.sq
    sh = tile_shapes(s.dims, prec)
    if prec == 2 and (s.dims[0] // 2) % 4:
        assert sh == []
        with pytest.raises(sq.StochqError):
            sq.sq_set_dslash_shape(s.ctx, prec, 5, 1, (1, 1, 1, 2, 2))
        return
    assert sh
    kappa, csw, a = 0.121, 1.0, -0.37
    sq.sq_build_clover(s.ctx, kappa, csw)
    n = 5  # ragged source groups for sg = 2 and 4
    psi = random_spinors(s.dims, n, 41)
    x = random_spinors(s.dims, n, 42)
    want = {}
    for p_out in (0, 1):
        for clover, xpay in [(0, 0), (1, 1)]:
            want[p_out, clover, xpay] = [oracle_dslash(s, psi[k], x[k], p_out, kappa, csw, clover, xpay, a)
                                         for k in range(n)]
    for i, (by, bz, bt) in enumerate(sh):
        sg = (2, 4, 8)[i % 3]
        nbuf = 2 + (i % 2)
        try:
            sq.sq_set_dslash_shape(s.ctx, prec, n, 1, (by, bz, bt, sg, nbuf))
        except sq.StochqError:
            continue  # shared memory: a 3-deep ring may not fit
        assert sq.sq_get_dslash_shape(s.ctx, prec, n) == (1, (by, bz, bt, sg, nbuf))
        for (p_out, clover, xpay), w in want.items():
            flags = (sq.SQ_DS_CLOVER_INV if clover else 0) | (sq.SQ_DS_XPAY if xpay else 0)
            got = run_dslash(s, prec, n, psi, x, p_out, flags, a)
            for k in range(n):
                assert rel(got[k], w[k]) < TOL[prec], ((by, bz, bt, sg, nbuf), p_out, clover, xpay, k)


@pytest.mark.parametrize("prec", [1, 2])
def test_xpay_and_clover_alone(setup, prec):
    """The two other fused variants (A^-1 only, xpay only) on one shape."""
    s = setup
    sq = s.sq
    sh = tile_shapes(s.dims, prec)
    if not sh:
        pytest.skip("no tiled shape for this lattice and precision")
    kappa, csw, a = 0.118, 1.0, 0.53
    sq.sq_build_clover(s.ctx, kappa, csw)
    n = 3
    psi = random_spinors(s.dims, n, 51)
    x = random_spinors(s.dims, n, 52)
    sq.sq_set_dslash_shape(s.ctx, prec, n, 1, sh[0] + (2, 2))
    for clover, xpay in [(1, 0), (0, 1)]:
        flags = (sq.SQ_DS_CLOVER_INV if clover else 0) | (sq.SQ_DS_XPAY if xpay else 0)
        for p_out in (0, 1):
            got = run_dslash(s, prec, n, psi, x, p_out, flags, a)
            for k in range(n):
                w = oracle_dslash(s, psi[k], x[k], p_out, kappa, csw, clover, xpay, a)
                assert rel(got[k], w) < TOL[prec]


def test_tiled_and_per_site_kernels_agree_fp32():
    """Same inputs through both kernels: equal up to FP32 rounding order."""
    from paper_1405_4524_gb300 import stochq as sq

    dims = (8, 4, 4, 8)
    s = Setup(dims, eps=0.3, seed=17)
    try:
        sq.sq_build_clover(s.ctx, 0.12, 1.0)
        n = 6
        psi = random_spinors(dims, n, 61)
        x = random_spinors(dims, n, 62)
        flags = sq.SQ_DS_CLOVER_INV | sq.SQ_DS_XPAY
        sq.sq_set_dslash_shape(s.ctx, 1, n, 0, (64, 2, 0))
        a0 = run_dslash(s, 1, n, psi, x, 0, flags, -0.0144)
        sq.sq_set_dslash_shape(s.ctx, 1, n, 1, (4, 2, 2, 4, 2))
        a1 = run_dslash(s, 1, n, psi, x, 0, flags, -0.0144)
        for k in range(n):
            assert rel(a1[k], a0[k]) < 2e-7
    finally:
        s.close()


@pytest.mark.parametrize("inner", [1, 2])
def test_solve_through_tiled_kernel(inner):
    """A mixed-precision solve whose inner dslash (fused reductions included)
    is the tiled kernel: every source within 1e-9 of the oracle's solution."""
    from paper_1405_4524_gb300 import inputs, stochq as sq

    dims = (8, 4, 4, 8)
    kappa, csw = 0.12, 1.0
    U = inputs.make_links(dims, 0.25, 1007)
    eta = inputs.make_z4(dims, 4, 2007)
    ctx = sq.sq_create(dims, -1)
    try:
        sq.sq_load_gauge(ctx, U, 12)
        sq.sq_set_dslash_shape(ctx, inner, 4, 1, (2, 2, 2, 2, 2))
        sol = np.zeros_like(eta)
        _, stats = sq.sq_solve(ctx, kappa, csw, eta, sol, 4, 1e-10, sq.sq_default_params(inner_prec=inner))
        assert sq.sq_get_dslash_shape(ctx, inner, 4)[0] == 1
        F = oracle.field_strength(U)
        for k in range(4):
            ref, _, _ = oracle.solve(U, eta[k], kappa, csw, -1.0, tol=1e-13, F=F)
            assert stats[k]["true_residual"] <= 1e-10
            assert rel(sol[k], ref) <= 1e-9
    finally:
        sq.sq_destroy(ctx)


def test_full_size_fp16_tiled_vs_per_site():
    """32^3 x 64 with 24 FP16 sources (the defect-correction workload's size
    and source count): every site through the tiled kernel (the tuner's
    shape if it is a tiled one) against the per-site kernel. Both store FP16
    with per-site norms, so they differ by FP16 roundings only. The oracle
    comparison at this size is test_gpu_workloads.test_dslash_full_size."""
    import torch

    from paper_1405_4524_gb300 import inputs, stochq as sq

    dims = (32, 32, 32, 64)
    n = 24
    U = inputs.make_links(dims, 0.25, 1004)
    ctx = sq.sq_create(dims, -1)
    try:
        sq.sq_load_gauge(ctx, U, 12)
        sq.sq_build_clover(ctx, 0.122, 1.0)
        X, Y, Z, T = dims
        g = torch.Generator(device="cuda").manual_seed(71)
        psi = torch.randn((n, T, Z, Y, X, 4, 3), dtype=torch.complex128, device="cuda", generator=g)
        fb = sq.sq_field_bytes(ctx, 2, n)
        bin_, bt_, bp = device_buffer(fb), device_buffer(fb), device_buffer(fb)
        sq.sq_pack_spinor(ctx, bin_, psi, 1, 2, n)
        flags = sq.SQ_DS_CLOVER_INV | sq.SQ_DS_SYNC
        sq.sq_dslash_eo(ctx, bt_, bin_, None, 0, 2, n, flags, 0.0)  # autotuned
        kind, shape = sq.sq_get_dslash_shape(ctx, 2, n)
        if kind != 1:
            sq.sq_set_dslash_shape(ctx, 2, n, 1, (4, 2, 2, 2, 2))
            sq.sq_dslash_eo(ctx, bt_, bin_, None, 0, 2, n, flags, 0.0)
        sq.sq_set_dslash_shape(ctx, 2, n, 0, (64, 2, 0))
        sq.sq_dslash_eo(ctx, bp, bin_, None, 0, 2, n, flags, 0.0)
        out_t = torch.zeros_like(psi)
        sq.sq_unpack_spinor(ctx, out_t, bt_, 0, 2, n)
        out_p = torch.zeros_like(psi)
        sq.sq_unpack_spinor(ctx, out_p, bp, 0, 2, n)
        for k in range(n):
            d = float(torch.linalg.norm(out_t[k] - out_p[k]) / torch.linalg.norm(out_p[k]))
            assert d < 2e-3, (k, d)
    finally:
        sq.sq_destroy(ctx)


def test_bounded_wait_runs_out():
    """The stall test: every CTA first waits, with a limit of 2000 cycles, on a
    barrier that nothing completes; the wait runs out, the CTA lets its
    issued copies land and returns, and the call reports SQ_ERR_TIMEOUT.
    With normal waits restored the same context gives the oracle's result."""
    from paper_1405_4524_gb300 import stochq as sq

    dims = (8, 4, 4, 8)
    s = Setup(dims, eps=0.3, seed=19)
    try:
        n = 8
        psi = random_spinors(dims, n, 81)
        x = random_spinors(dims, n, 82)
        sq.sq_set_dslash_shape(s.ctx, 1, n, 1, (4, 2, 2, 8, 2))
        sq.sq_set_wait_cycles(s.ctx, 2000, True)
        with pytest.raises(sq.StochqError) as e:
            run_dslash(s, 1, n, psi, x, 1, 0, 0.0)
        assert e.value.status == sq.SQ_ERR_TIMEOUT
        sq.sq_set_wait_cycles(s.ctx, 0, False)
        got = run_dslash(s, 1, n, psi, x, 1, 0, 0.0)
        for k in range(n):
            assert rel(got[k], oracle_dslash(s, psi[k], x[k], 1, 0, 0, 0, 0, 0)) < 1e-6
    finally:
        s.close()


def test_solve_reports_timeout():
    """A solve whose tiled dslash waits run out returns SQ_ERR_TIMEOUT; the
    context then solves normally."""
    from paper_1405_4524_gb300 import inputs, stochq as sq

    dims = (8, 4, 4, 8)
    U = inputs.make_links(dims, 0.25, 1007)
    eta = inputs.make_z4(dims, 2, 2008)
    ctx = sq.sq_create(dims, -1)
    try:
        sq.sq_load_gauge(ctx, U, 12)
        sq.sq_set_dslash_shape(ctx, 1, 2, 1, (2, 2, 2, 2, 2))
        sq.sq_set_wait_cycles(ctx, 2000, True)
        sol = np.zeros_like(eta)
        st, _ = sq.sq_solve(ctx, 0.12, 1.0, eta, sol, 2, 1e-10, sq.sq_default_params(max_iter=40),
                            raise_on_error=False)
        assert st == sq.SQ_ERR_TIMEOUT
        sq.sq_set_wait_cycles(ctx, 0, False)
        sol[...] = 0
        st, stats = sq.sq_solve(ctx, 0.12, 1.0, eta, sol, 2, 1e-10)
        assert st == 0 and all(x["true_residual"] <= 1e-10 for x in stats)
    finally:
        sq.sq_destroy(ctx)


def test_tuned_shapes_persist(tmp_path):
    """Shapes tuned in one context, saved to a file and loaded into a fresh
    context of the same lattice, are the ones that context then uses; lines
    of another lattice, another GPU or an inadmissible shape are skipped."""
    from paper_1405_4524_gb300 import stochq as sq

    dims = (8, 4, 4, 8)
    path = str(tmp_path / "shapes.txt")
    s = Setup(dims, eps=0.3, seed=23)
    try:
        n = 4
        psi = random_spinors(dims, n, 91)
        run_dslash(s, 1, n, psi, psi, 0, 0, 0.0)  # the tuner's pick
        sq.sq_set_dslash_shape(s.ctx, 2, n, 1, (4, 2, 2, 2, 3))     # a set one
        want = {1: sq.sq_get_dslash_shape(s.ctx, 1, n), 2: sq.sq_get_dslash_shape(s.ctx, 2, n)}
        sq.sq_tune_save(s.ctx, path)
    finally:
        s.close()
    with open(path, "a") as f:
        f.write("stochq-shape some_other_gpu 8 4 4 8 1 12 4 0 64 2 0 0 0 0 0 2\n")
        f.write("garbage line\n")
    lines = open(path).read().splitlines()
    gpu = lines[0].split()[1]
    with open(path, "a") as f:
        f.write(f"stochq-shape {gpu} 16 4 4 8 1 12 4 0 64 2 0 0 0 0 0 2\n")   # another lattice
        f.write(f"stochq-shape {gpu} 8 4 4 8 1 12 9 1 3 3 3 2 2 0 0 0\n")      # inadmissible tile
    s2 = Setup(dims, eps=0.3, seed=23)
    try:
        with pytest.raises(sq.StochqError):
            sq.sq_get_dslash_shape(s2.ctx, 1, n)
        assert sq.sq_tune_load(s2.ctx, path) == 2
        assert sq.sq_get_dslash_shape(s2.ctx, 1, n) == want[1]
        assert sq.sq_get_dslash_shape(s2.ctx, 2, n) == want[2]
        got = run_dslash(s2, 2, n, psi, psi, 1, 0, 0.0)  # runs at the loaded tiled shape
        for k in range(n):
            assert rel(got[k], oracle_dslash(s2, psi[k], psi[k], 1, 0, 0, 0, 0, 0)) < 5e-3
    finally:
        s2.close()
