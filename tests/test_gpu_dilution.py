"""GPU parity of the dilution kernel and of diluted / point-source solves
(Sec. "Stochastic propagators": time-spin-colour dilution; the point
propagators of the exact comparison), through the C ABI.

Bars: diluted sources bitwise equal to the oracle's (the kernel copies
values); every diluted source solved to a true FP64 residual <= 1e-10 and
within 1e-9 of the oracle's solution; the point propagator within 1e-9 of
the dense LU inverse's columns.
"""

import numpy as np
import pytest

import oracle
from gpu_helpers import Setup, rel
from paper_1405_4524_gb300 import inputs

pytestmark = pytest.mark.gpu

SCHEMES = [("time", 1), ("spin_colour", 2), ("full", 3)]


@pytest.mark.parametrize("name,scheme", SCHEMES)
def test_dilute_matches_oracle(name, scheme):
    import torch
    from paper_1405_4524_gb300 import stochq as sq

    dims = (4, 4, 2, 6)
    ctx = sq.sq_create(dims, -1)
    try:
        noise = inputs.make_z4(dims, 2, 7101)
        want = oracle.dilute(noise, name)
        got = sq.sq_dilute(ctx, noise, 2, scheme)
        assert got.shape == want.shape and np.array_equal(got, want)
        gd = sq.sq_dilute(ctx, torch.from_numpy(noise).cuda(), 2, scheme)
        assert np.array_equal(gd.cpu().numpy(), want)
    finally:
        sq.sq_destroy(ctx)


def test_full_dilution_solve():
    """One Z4 noise vector on 4^3 x 8 fully diluted into 96 sources, solved in
    one batch: every source to 1e-10, sampled solutions against the oracle,
    and the diluted solutions sum to the solution of the noise vector
    (linearity)."""
    spec = inputs.WORKLOADS["4x4x4x8"]
    dims = spec["dims"]
    s = Setup(dims, spec["eps"], spec["link_seed"])
    sq = s.sq
    try:
        noise = inputs.make_z4(dims, 1, 7201)
        src = sq.sq_dilute(s.ctx, noise, 1, sq.SQ_DILUTE_FULL)
        n = src.shape[0]
        assert n == 96
        sol = np.zeros_like(src)
        st, stats = sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], src, sol, n, 1e-10)
        assert st == 0 and all(x["status"] == 0 and x["true_residual"] <= 1e-10 for x in stats)
        for d in (0, 13, 50, 95):
            ref, _, res = oracle.solve(s.U, src[d], spec["kappa"], spec["csw"], -1.0, tol=1e-13, F=s.F)
            assert rel(sol[d], ref) <= 1e-9
        whole = np.zeros_like(noise)
        sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], noise, whole, 1, 1e-12)
        assert rel(sol.sum(axis=0), whole[0]) <= 1e-9
    finally:
        s.close()


def test_point_propagator():
    """Twelve point sources at one site (spin-colour dilution of a one-site
    noise vector): the solutions are the dense inverse's columns, and their
    pion contractions add up to sum_y tr S_p S_p^dag per timeslice."""
    from test_oracle_pins import dense_M

    dims = (4, 2, 2, 4)
    X, Y, Z, T = dims
    s = Setup(dims, 0.25, 7301)
    sq = s.sq
    kappa, csw = 0.12, 1.0
    try:
        y0 = (1, 1, 0, 3)  # t, z, y, x
        noise = np.zeros((1, T, Z, Y, X, 4, 3), dtype=np.complex128)
        noise[(0,) + y0] = 1.0
        src = sq.sq_dilute(s.ctx, noise, 1, sq.SQ_DILUTE_SPIN_COLOUR)
        sol = np.zeros_like(src)
        st, stats = sq.sq_solve(s.ctx, kappa, csw, src, sol, 12, 1e-12)
        assert st == 0
        S = np.linalg.inv(dense_M(s.U, s.F, kappa, csw, -1.0, dims))
        site = ((y0[0] * Z + y0[1]) * Y + y0[2]) * X + y0[3]
        for a in range(12):
            col = S[:, 12 * site + a].reshape(src[a].shape)
            assert rel(sol[a], col) <= 1e-9
        C = sq.sq_contract_pion(s.ctx, sol, 12, [y0[0]] * 12).sum(axis=0)
        Sp = S[:, 12 * site:12 * site + 12].reshape(T, Z * Y * X * 12, 12)
        want = np.array([np.sum(np.abs(Sp[(y0[0] + dt) % T]) ** 2) for dt in range(T)])
        assert np.allclose(C, want, rtol=1e-9, atol=0)
    finally:
        s.close()


def test_dilute_errors():
    from paper_1405_4524_gb300 import stochq as sq

    dims = (2, 2, 2, 4)
    ctx = sq.sq_create(dims, -1)
    try:
        noise = inputs.make_z4(dims, 1, 7401)
        out = np.zeros((48,) + noise.shape[1:], dtype=np.complex128)
        with pytest.raises(sq.StochqError):
            sq.sq_dilute(ctx, noise, 1, 7, out=out)
        with pytest.raises(sq.StochqError):
            sq.sq_dilute(ctx, noise, 0, sq.SQ_DILUTE_TIME)
        assert np.array_equal(sq.sq_dilute(ctx, noise, 1, sq.SQ_DILUTE_TIME), oracle.dilute(noise, "time"))
    finally:
        sq.sq_destroy(ctx)
