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
