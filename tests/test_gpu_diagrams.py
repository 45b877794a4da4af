"""GPU parity of the diagram contractions (sq_contract_diagrams, Sec.
"Stochastic propagators" and Sec. "Correlation function") and their
vacuum-subtracted ensemble combination (sq_diagrams_ensemble) against the
oracle (oracle.diagrams), through the C ABI.

Bar: every one of the seven quantities within 1e-12 of its largest magnitude
over t (FP64, different summation orders: the oracle fills S literally, the
GPU contracts Gram matrices). The end-to-end case (point and noise solutions
from the library's own solver) is within the solutions' 1e-9 accuracy.
"""

import numpy as np
import pytest

import oracle
from oracle import diagrams as dg
from gpu_helpers import random_spinors
from paper_1405_4524_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sq():
    from paper_1405_4524_gb300 import stochq

    return stochq


def close_rows(got, want, bar):
    for q in range(want.shape[0]):
        scale = float(np.max(np.abs(want[q])))
        assert float(np.max(np.abs(got[q] - want[q]))) <= bar * scale, (dg.NAMES[q], got[q], want[q])


@pytest.mark.parametrize("dims,n", [((2, 2, 2, 2), 3), ((4, 2, 2, 4), 19), ((4, 4, 4, 4), 6)])
@pytest.mark.parametrize("two_sets", [False, True])
def test_diagrams_match_oracle(sq, dims, n, two_sets):
    """Random point and noise fields (the contraction is linear in each
    input, so any fields test it), one CTA, ragged 16-source tiles, two sets
    or one."""
    Xp = random_spinors(dims, 12, 101)
    eA, xA = inputs.make_z4(dims, n, 102), random_spinors(dims, n, 103)
    eB, xB = (inputs.make_z4(dims, n, 104), random_spinors(dims, n, 105)) if two_sets else (None, None)
    ctx = sq.sq_create(dims, -1)
    try:
        got = sq.sq_contract_diagrams(ctx, Xp, eA, xA, n, eB, xB)
    finally:
        sq.sq_destroy(ctx)
    want = dg.diagrams_stochastic(Xp, eA, xA, eB, xB)
    close_rows(got, want, 1e-12)
    assert np.array_equal(got[6], np.conj(got[5]))
    assert np.all(got[0].imag == 0)


def test_complete_basis_gives_the_exact_diagrams(sq):
    """2^4 lattice, dense inverse: 192 sources sqrt(N) e_i (every unit vector)
    for both sets make the stochastic route exact, so the GPU result equals
    the exact diagrams of the inverse."""
    from test_oracle_pins import dense_M

    dims = (2, 2, 2, 2)
    X, Y, Z, T = dims
    U = inputs.make_links(dims, 0.25, 61)
    F = oracle.field_strength(U)
    Minv = np.linalg.inv(dense_M(U, F, 0.12, 1.0, -1.0, dims))
    N = 12 * X * Y * Z * T
    eta = (np.sqrt(N) * np.eye(N, dtype=np.complex128)).reshape(N, T, Z, Y, X, 4, 3)
    Xs = np.ascontiguousarray((Minv @ eta.reshape(N, -1).T).T).reshape(eta.shape)
    Xp = Minv[:, :12].T.reshape(12, T, Z, Y, X, 4, 3).copy()
    ctx = sq.sq_create(dims, -1)
    try:
        got = sq.sq_contract_diagrams(ctx, Xp, eta, Xs, N, eta, Xs)
    finally:
        sq.sq_destroy(ctx)
    close_rows(got, dg.diagrams_exact(Minv, dims), 1e-11)


def test_end_to_end_with_the_solver(sq):
    """4^4 lattice: the twelve point sources from sq_dilute (spin-colour
    dilution of a noise vector that is 1 on the origin's twelve components),
    two Z4 sets, all solved by sq_solve to 1e-11, contracted on the device;
    against the oracle's diagrams of the oracle's own solutions (dense
    inverse)."""
    import torch

    from test_oracle_pins import dense_M

    dims = (4, 4, 4, 4)
    X, Y, Z, T = dims
    kappa, csw = 0.12, 1.0
    U = inputs.make_links(dims, 0.25, 1011)
    F = oracle.field_strength(U)
    Minv = np.linalg.inv(dense_M(U, F, kappa, csw, -1.0, dims))
    n = 8
    one = np.zeros((1, T, Z, Y, X, 4, 3), dtype=np.complex128)
    one[0, 0, 0, 0, 0] = 1.0
    eA, eB = inputs.make_z4(dims, n, 1012), inputs.make_z4(dims, n, 1013)
    ctx = sq.sq_create(dims, -1)
    try:
        sq.sq_load_gauge(ctx, U, 12)
        prm = sq.sq_default_params(io=sq.SQ_DEVICE)
        src_p = sq.sq_dilute(ctx, torch.from_numpy(one).cuda(), 1, sq.SQ_DILUTE_SPIN_COLOUR)
        Xp = torch.zeros_like(src_p)
        sq.sq_solve(ctx, kappa, csw, src_p, Xp, 12, 1e-11, prm)
        dA, dB = torch.from_numpy(eA).cuda(), torch.from_numpy(eB).cuda()
        xA, xB = torch.zeros_like(dA), torch.zeros_like(dB)
        sq.sq_solve(ctx, kappa, csw, dA, xA, n, 1e-11, prm)
        sq.sq_solve(ctx, kappa, csw, dB, xB, n, 1e-11, prm)
        got = sq.sq_contract_diagrams(ctx, Xp, dA, xA, n, dB, xB).cpu().numpy()
    finally:
        sq.sq_destroy(ctx)
    solve = lambda e: (Minv @ e.reshape(e.shape[0], -1).T).T.reshape(e.shape)
    Xp_o = Minv[:, :12].T.reshape(12, T, Z, Y, X, 4, 3).copy()
    want = dg.diagrams_stochastic(Xp_o, eA, solve(eA), eB, solve(eB))
    close_rows(got, want, 1e-8)


def test_host_and_device_io_are_bitwise_equal(sq):
    import torch

    dims, n = (4, 2, 2, 4), 5
    Xp = random_spinors(dims, 12, 201)
    eA, xA = inputs.make_z4(dims, n, 202), random_spinors(dims, n, 203)
    eB, xB = inputs.make_z4(dims, n, 204), random_spinors(dims, n, 205)
    ctx = sq.sq_create(dims, -1)
    try:
        h = sq.sq_contract_diagrams(ctx, Xp, eA, xA, n, eB, xB)
        cu = lambda a: torch.from_numpy(a).cuda()
        d = sq.sq_contract_diagrams(ctx, cu(Xp), cu(eA), cu(xA), n, cu(eB), cu(xB)).cpu().numpy()
        again = sq.sq_contract_diagrams(ctx, Xp, eA, xA, n, eB, xB)
    finally:
        sq.sq_destroy(ctx)
    assert np.array_equal(h, d) and np.array_equal(h, again)


def test_ensemble_matches_oracle(sq):
    """Per-configuration records of several configurations (from the GPU
    contraction of independent noise sets) through sq_diagrams_ensemble and
    through oracle.diagrams.ensemble."""
    import torch

    dims, n = (2, 2, 2, 4), 4
    ctx = sq.sq_create(dims, -1)
    try:
        recs = []
        for c in range(6):
            Xp = random_spinors(dims, 12, 300 + c)
            eA, xA = inputs.make_z4(dims, n, 310 + c), random_spinors(dims, n, 320 + c)
            eB, xB = inputs.make_z4(dims, n, 330 + c), random_spinors(dims, n, 340 + c)
            recs.append(sq.sq_contract_diagrams(ctx, Xp, eA, xA, n, eB, xB))
        rec = np.array(recs)
        got = sq.sq_diagrams_ensemble(ctx, rec)
        got_d = sq.sq_diagrams_ensemble(ctx, torch.from_numpy(rec).cuda()).cpu().numpy()
    finally:
        sq.sq_destroy(ctx)
    want = dg.ensemble(rec)
    assert np.allclose(got, want, rtol=1e-13, atol=1e-13 * np.max(np.abs(want)))
    assert np.array_equal(got, got_d)


def test_errors(sq):
    dims, n = (2, 2, 2, 2), 2
    Xp = random_spinors(dims, 12, 401)
    eA, xA = inputs.make_z4(dims, n, 402), random_spinors(dims, n, 403)
    ctx = sq.sq_create(dims, -1)
    try:
        with pytest.raises(sq.StochqError) as e:
            sq.sq_contract_diagrams(ctx, Xp, eA, xA, 0)
        assert e.value.status == sq.SQ_ERR_ARG
        with pytest.raises(ValueError):
            sq.sq_contract_diagrams(ctx, Xp, eA, xA, n, eA, None)
        with pytest.raises(sq.StochqError) as e:
            sq.sq_contract_diagrams(ctx, None, eA, xA, n)
        assert e.value.status == sq.SQ_ERR_ARG
        with pytest.raises(sq.StochqError) as e:
            sq.sq_diagrams_ensemble(ctx, np.zeros((0, 7, 2), dtype=np.complex128))
        assert e.value.status == sq.SQ_ERR_ARG
    finally:
        sq.sq_destroy(ctx)
