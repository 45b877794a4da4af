"""GPU parity of the tensor-core stochastic operators (sq_contract_stoch_op_z4,
Eq. stoop) against the FP64 oracle, through the C ABI.

Bar: every element of O and C within 1e-12 of the largest element's
magnitude, as for the FP64 route. The route is exact up to the truncation
of gamma5 X to 55 bits below each 4096-row block's largest component and
FP64 rounding, so the bar holds with a wide margin even when the sources'
magnitudes differ by e^16 (the inputs below scale each source and
timeslice by a random factor in [e^-8, e^8]).
"""

import numpy as np
import pytest

import oracle
from gpu_helpers import random_spinors
from paper_1405_4524_gb300 import inputs

pytestmark = pytest.mark.gpu

BAR = 1e-12


def close(got, want, bar=BAR):
    return float(np.max(np.abs(got - want))) <= bar * float(np.max(np.abs(want)))


@pytest.fixture(scope="module")
def sq():
    from paper_1405_4524_gb300 import stochq

    return stochq


def scaled_spinors(dims, n, seed):
    X = random_spinors(dims, n, seed)
    rng = np.random.default_rng(seed + 1)
    f = np.exp(rng.uniform(-8.0, 8.0, (n, dims[3])))
    return X * f[:, :, None, None, None, None, None]


@pytest.mark.parametrize("dims,n", [((2, 2, 2, 2), 3), ((4, 4, 4, 8), 20), ((8, 8, 8, 2), 5),
                                    ((2, 2, 2, 4), 130)])
def test_tensor_core_operators_match_oracle(sq, dims, n):
    """One CTA; two j tiles; two exact chunks of 8192 columns (8^3 slice);
    two i tiles and nine j tiles with ragged edges (130 sources)."""
    ctx = sq.sq_create(dims, -1)
    try:
        eta = inputs.make_z4(dims, n, 6101 + n)
        X = scaled_spinors(dims, n, 6201 + n)
        O, C = sq.sq_contract_stoch_op(ctx, eta, X, n, tensor_cores=True)
        Ow = oracle.stochastic_operator(eta, X)
        assert close(O, Ow), float(np.max(np.abs(O - Ow)) / np.max(np.abs(Ow)))
        assert close(C, oracle.stochastic_operator_correlator(Ow))
    finally:
        sq.sq_destroy(ctx)


def test_tensor_core_full_size_and_fp64_route(sq):
    """16^3 x 32 with 16 sources (twelve exact chunks per slice): against the
    oracle and against the FP64-pipe route."""
    dims, n = (16, 16, 16, 32), 16
    ctx = sq.sq_create(dims, -1)
    try:
        eta = inputs.make_z4(dims, n, 6301)
        X = scaled_spinors(dims, n, 6302)
        O, C = sq.sq_contract_stoch_op(ctx, eta, X, n, tensor_cores=True)
        Ow = oracle.stochastic_operator(eta, X)
        assert close(O, Ow)
        assert close(C, oracle.stochastic_operator_correlator(Ow))
        O64, _ = sq.sq_contract_stoch_op(ctx, eta, X, n)
        assert close(O, O64, 1e-13)
    finally:
        sq.sq_destroy(ctx)


def test_tensor_core_diluted_sources_device_io(sq):
    """Time-diluted Z4 sources (zero off their timeslice), device I/O equal
    bitwise to host I/O, repeated calls equal bitwise."""
    import torch

    dims, n = (4, 4, 4, 8), 8
    ctx = sq.sq_create(dims, -1)
    try:
        eta = inputs.make_z4(dims, n, 6401, [k % 8 for k in range(n)])
        X = scaled_spinors(dims, n, 6402)
        O, C = sq.sq_contract_stoch_op(ctx, eta, X, n, tensor_cores=True)
        Ow = oracle.stochastic_operator(eta, X)
        assert close(O, Ow)
        Od, Cd = sq.sq_contract_stoch_op(ctx, torch.from_numpy(eta).cuda(), torch.from_numpy(X).cuda(), n,
                                         tensor_cores=True)
        assert np.array_equal(Od.cpu().numpy(), O) and np.array_equal(Cd.cpu().numpy(), C)
        O2, _ = sq.sq_contract_stoch_op(ctx, eta, X, n, tensor_cores=True)
        assert np.array_equal(O2, O)
    finally:
        sq.sq_destroy(ctx)


def test_tensor_core_rejects_general_sources(sq):
    dims, n = (2, 2, 2, 4), 2
    ctx = sq.sq_create(dims, -1)
    try:
        X = random_spinors(dims, n, 6501)
        eta = inputs.make_z4(dims, n, 6502)
        eta[1, 2, 0, 1, 1, 3, 2] = 0.5
        with pytest.raises(sq.StochqError) as ex:
            sq.sq_contract_stoch_op(ctx, eta, X, n, tensor_cores=True)
        assert ex.value.status == sq.SQ_ERR_ARG
        X[0, 0, 0, 0, 0, 0, 0] = np.inf
        with pytest.raises(sq.StochqError) as ex:
            sq.sq_contract_stoch_op(ctx, inputs.make_z4(dims, n, 6502), X, n, tensor_cores=True)
        assert ex.value.status == sq.SQ_ERR_NONFINITE
        # the context still works
        X = random_spinors(dims, n, 6503)
        eta = inputs.make_z4(dims, n, 6504)
        O, _ = sq.sq_contract_stoch_op(ctx, eta, X, n, tensor_cores=True)
        assert close(O, oracle.stochastic_operator(eta, X))
    finally:
        sq.sq_destroy(ctx)


def test_tensor_core_many_sources(sq):
    """256 sources on 8^3 x 16 (2 i tiles x 16 j tiles per timeslice, two
    exact chunks): sampled pairs against the oracle, every element against
    the FP64-pipe route."""
    dims, n = (8, 8, 8, 16), 256
    ctx = sq.sq_create(dims, -1)
    try:
        eta = inputs.make_z4(dims, n, 6601)
        X = inputs.make_gaussian_spinors(dims, n, 6701)
        O, C = sq.sq_contract_stoch_op(ctx, eta, X, n, tensor_cores=True)
        rng = np.random.default_rng(6801)
        scale = float(np.max(np.abs(O)))
        for i, j in zip(rng.integers(0, n, 12), rng.integers(0, n, 12)):
            want = oracle.stochastic_operator(eta[[i]], X[[j]])[:, 0, 0]
            assert float(np.max(np.abs(O[:, i, j] - want))) <= BAR * scale
        O64, C64 = sq.sq_contract_stoch_op(ctx, eta, X, n)
        assert close(O, O64, 1e-13)
        assert close(C, C64, 1e-12)
    finally:
        sq.sq_destroy(ctx)


def test_tensor_core_timeslice_batches(sq):
    """32^3 x 64 with 16 sources: the packed operands of all 64 timeslices
    exceed the 8 GiB workspace, so the call runs in four batches of 16
    timeslices. Inputs made on the device (seeded); every element
    against the FP64-pipe route and sampled pairs against the oracle."""
    import torch

    dims, n = (32, 32, 32, 64), 16
    X_, Y, Z, T = dims
    g = torch.Generator(device="cuda")
    g.manual_seed(6901)
    k = torch.randint(0, 4, (n, T, Z, Y, X_, 4, 3), generator=g, device="cuda")
    eta = torch.tensor([1, 1j, -1, -1j], dtype=torch.complex128, device="cuda")[k]
    del k
    X = torch.randn(eta.shape, dtype=torch.complex128, device="cuda", generator=g)
    ctx = sq.sq_create(dims, -1)
    try:
        O, C = sq.sq_contract_stoch_op(ctx, eta, X, n, tensor_cores=True)
        O64, C64 = sq.sq_contract_stoch_op(ctx, eta, X, n)
        O, O64 = O.cpu().numpy(), O64.cpu().numpy()
        assert close(O, O64, 1e-13)
        assert close(C.cpu().numpy(), C64.cpu().numpy(), 1e-12)
        for i, j in [(0, 15), (7, 7), (12, 3)]:
            want = oracle.stochastic_operator(eta[[i]].cpu().numpy(), X[[j]].cpu().numpy())[:, 0, 0]
            assert float(np.max(np.abs(O[:, i, j] - want))) <= BAR * float(np.max(np.abs(O)))
    finally:
        sq.sq_destroy(ctx)
        del eta, X
        torch.cuda.empty_cache()


def test_tensor_core_bounded_wait_runs_out(sq):
    """The stall test: the product warp first waits, with a limit of 2000
    cycles, on a barrier that nothing completes; the call reports
    SQ_ERR_TIMEOUT after the issued copies and products have drained and the
    tensor memory is freed. Normal waits then give the oracle's operators."""
    dims, n = (4, 4, 4, 8), 20
    eta = inputs.make_z4(dims, n, 7301)
    X = scaled_spinors(dims, n, 7302)
    ctx = sq.sq_create(dims, -1)
    try:
        sq.sq_set_wait_cycles(ctx, 2000, True)
        with pytest.raises(sq.StochqError) as e:
            sq.sq_contract_stoch_op(ctx, eta, X, n, tensor_cores=True)
        assert e.value.status == sq.SQ_ERR_TIMEOUT
        sq.sq_set_wait_cycles(ctx, 0, False)
        O, C = sq.sq_contract_stoch_op(ctx, eta, X, n, tensor_cores=True)
        assert close(O, oracle.stochastic_operator(eta, X))
    finally:
        sq.sq_destroy(ctx)


def test_tensor_core_tiny_magnitudes(sq):
    """Sources whose chunks' largest component sits near the bottom of the
    FP64 normal range: the exact digit weights become subnormal powers of
    two and the operators still match the oracle (relative to their size)."""
    dims, n = (2, 2, 2, 4), 3
    eta = inputs.make_z4(dims, n, 7401)
    X = random_spinors(dims, n, 7402) * 2.0 ** -1000
    ctx = sq.sq_create(dims, -1)
    try:
        O, _ = sq.sq_contract_stoch_op(ctx, eta, X, n, tensor_cores=True)
        want = oracle.stochastic_operator(eta, X)
        assert float(np.max(np.abs(O - want))) <= 1e-10 * float(np.max(np.abs(want)))
    finally:
        sq.sq_destroy(ctx)
