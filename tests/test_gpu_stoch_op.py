"""GPU parity of the stochastic-operator contraction (Eq. stoop) and its
correlator, through the C ABI, against the FP64 oracle.

Bar: every element of O and C within 1e-12 of the largest element's
magnitude (both sides sum the same products in FP64, in different orders;
K = X*Y*Z*12 terms per element give a rounding spread of order
K * 2^-53 * max|term|, far below the bar), and bitwise equality between
host and device I/O (same kernels, same order).
"""

import numpy as np
import pytest

import oracle
from gpu_helpers import random_spinors
from paper_1405_4524_gb300 import inputs

pytestmark = pytest.mark.gpu

BAR = 1e-12


def close(got, want):
    scale = float(np.max(np.abs(want)))
    return float(np.max(np.abs(got - want))) <= BAR * scale


@pytest.fixture(scope="module")
def sq():
    from paper_1405_4524_gb300 import stochq

    return stochq


@pytest.mark.parametrize("dims,n", [((4, 4, 4, 8), 4), ((6, 4, 4, 8), 19), ((2, 2, 2, 4), 1),
                                    ((8, 6, 4, 6), 33)])
def test_operator_and_correlator_match_oracle(sq, dims, n):
    """Several pair tiles with a ragged last one (19, 33), one source, a
    slice of two K-chunks, T not a power of two."""
    ctx = sq.sq_create(dims, -1)
    try:
        eta = inputs.make_z4(dims, n, 4101 + n)
        X = random_spinors(dims, n, 4201 + n)
        O, C = sq.sq_contract_stoch_op(ctx, eta, X, n)
        Ow = oracle.stochastic_operator(eta, X)
        assert O.shape == Ow.shape
        assert close(O, Ow)
        assert close(C, oracle.stochastic_operator_correlator(Ow))
    finally:
        sq.sq_destroy(ctx)


def test_device_io_is_bitwise_host_io(sq):
    import torch

    dims, n = (4, 4, 4, 8), 5
    ctx = sq.sq_create(dims, -1)
    try:
        eta = inputs.make_z4(dims, n, 4301)
        X = random_spinors(dims, n, 4302)
        O, C = sq.sq_contract_stoch_op(ctx, eta, X, n)
        Od, Cd = sq.sq_contract_stoch_op(ctx, torch.from_numpy(eta).cuda(), torch.from_numpy(X).cuda(), n)
        assert Od.is_cuda and Cd.is_cuda
        assert np.array_equal(Od.cpu().numpy(), O)
        assert np.array_equal(Cd.cpu().numpy(), C)
        # repeated call: same bits
        O2, C2 = sq.sq_contract_stoch_op(ctx, eta, X, n)
        assert np.array_equal(O2, O) and np.array_equal(C2, C)
        # no correlator requested: O unchanged, C not written
        O3, C3 = sq.sq_contract_stoch_op(ctx, eta, X, n, correlator=False)
        assert C3 is None and np.array_equal(O3, O)
    finally:
        sq.sq_destroy(ctx)


def test_solutions_of_the_solver(sq):
    """O built from the solver's own solutions (tol 1e-12) agrees with O
    built by the oracle from the oracle's solutions (tol 1e-13)."""
    spec = inputs.WORKLOADS["4x4x4x8"]
    dims, n = spec["dims"], spec["n_rhs"]
    from gpu_helpers import Setup

    s = Setup(dims, spec["eps"], spec["link_seed"])
    try:
        eta = inputs.make_z4(dims, n, spec["src_seed"])
        sol = np.zeros_like(eta)
        s.sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], eta, sol, n, 1e-12)
        ref = np.array([oracle.solve(s.U, eta[k], spec["kappa"], spec["csw"], -1.0, tol=1e-13, F=s.F)[0]
                        for k in range(n)])
        O, C = sq.sq_contract_stoch_op(s.ctx, eta, sol, n)
        Ow = oracle.stochastic_operator(eta, ref)
        scale = float(np.max(np.abs(Ow)))
        assert float(np.max(np.abs(O - Ow))) <= 1e-9 * scale
        Cw = oracle.stochastic_operator_correlator(Ow)
        assert float(np.max(np.abs(C - Cw))) <= 1e-8 * float(np.max(np.abs(Cw)))
    finally:
        s.close()


def test_full_size_workload(sq):
    """The 16^3 x 32 lattice with 16 sources (the size the benchmark
    contracts): every element against the oracle."""
    dims, n = (16, 16, 16, 32), 16
    ctx = sq.sq_create(dims, -1)
    try:
        eta = inputs.make_z4(dims, n, 4401)
        X = random_spinors(dims, n, 4402)
        O, C = sq.sq_contract_stoch_op(ctx, eta, X, n)
        Ow = oracle.stochastic_operator(eta, X)
        assert close(O, Ow)
        assert close(C, oracle.stochastic_operator_correlator(Ow))
    finally:
        sq.sq_destroy(ctx)


def test_errors(sq):
    dims = (4, 4, 4, 8)
    ctx = sq.sq_create(dims, -1)
    try:
        eta = inputs.make_z4(dims, 2, 4501)
        with pytest.raises(sq.StochqError):
            sq.sq_contract_stoch_op(ctx, eta, eta, 0)
        with pytest.raises(ValueError):
            import torch

            sq.sq_contract_stoch_op(ctx, eta, torch.from_numpy(eta).cuda(), 2)
        # the context still works after the errors
        O, _ = sq.sq_contract_stoch_op(ctx, eta, eta, 2)
        assert close(O, oracle.stochastic_operator(eta, eta))
    finally:
        sq.sq_destroy(ctx)


# ---------------------------------------------------------------------------
# traces of filled stochastic propagators (Eq. Sfill) without the fill
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,n,two", [((4, 4, 4, 8), 4, True), ((4, 4, 4, 8), 4, False),
                                        ((2, 2, 4, 6), 19, True), ((2, 2, 2, 4), 1, False)])
def test_prop_trace_matches_oracle_fill(sq, dims, n, two):
    """Against the oracle's explicit fill of S for every source timeslice."""
    ctx = sq.sq_create(dims, -1)
    try:
        eA = inputs.make_z4(dims, n, 5101)
        xA = random_spinors(dims, n, 5102)
        eB = inputs.make_z4(dims, n, 5201 + 100) if two else None
        xB = random_spinors(dims, n, 5202) if two else None
        C = sq.sq_contract_prop_trace(ctx, eA, xA, n, eB, xB)
        want = oracle.stochastic_propagator_trace(eA, xA, eB, xB)
        assert C.shape == want.shape
        assert close(C, want)
    finally:
        sq.sq_destroy(ctx)


def gram_form(eA, xA, eB, xB):
    """(1/n^2) tr[P(t) Q(t0)] in numpy: the identity pinned against the
    oracle's fill in the oracle pins, for sizes where the fill cannot be
    stored."""
    n = eA.shape[0]
    P = np.einsum("jtzyxsc,itzyxsc->tji", np.conj(xB), xA)
    Q = np.einsum("itzyxsc,jtzyxsc->tij", np.conj(eA), eB)
    return np.einsum("tji,sij->st", P, Q) / n**2


def test_prop_trace_full_size(sq):
    dims, n = (16, 16, 16, 32), 16
    ctx = sq.sq_create(dims, -1)
    try:
        eA = inputs.make_z4(dims, n, 5301)
        xA = random_spinors(dims, n, 5302)
        eB = inputs.make_z4(dims, n, 5401)
        xB = random_spinors(dims, n, 5402)
        C = sq.sq_contract_prop_trace(ctx, eA, xA, n, eB, xB)
        assert close(C, gram_form(eA, xA, eB, xB))
    finally:
        sq.sq_destroy(ctx)


def test_prop_trace_device_io_and_errors(sq):
    import torch

    dims, n = (4, 4, 4, 8), 3
    ctx = sq.sq_create(dims, -1)
    try:
        eA = inputs.make_z4(dims, n, 5501)
        xA = random_spinors(dims, n, 5502)
        C = sq.sq_contract_prop_trace(ctx, eA, xA, n)
        Cd = sq.sq_contract_prop_trace(ctx, torch.from_numpy(eA).cuda(), torch.from_numpy(xA).cuda(), n)
        assert Cd.is_cuda and np.array_equal(Cd.cpu().numpy(), C)
        # one set: C[t0, t] is a sum of |.|^2, real and non-negative
        assert np.all(np.abs(C.imag) <= 1e-12 * np.abs(C).max()) and np.all(C.real >= 0)
        with pytest.raises(ValueError):
            sq.sq_contract_prop_trace(ctx, eA, xA, n, eA, None)
        out = np.zeros((8, 8), dtype=np.complex128)
        st = sq._lib.sq_contract_prop_trace(ctx, eA.ctypes.data, xA.ctypes.data, eA.ctypes.data, None, n,
                                            out.ctypes.data, sq.SQ_HOST)
        assert st == sq.SQ_ERR_ARG
        with pytest.raises(sq.StochqError):
            sq.sq_contract_prop_trace(ctx, eA, xA, 0)
        assert np.array_equal(sq.sq_contract_prop_trace(ctx, eA, xA, n), C)
    finally:
        sq.sq_destroy(ctx)
