"""Caller-supplied device memory (sq_set_allocator): the context's persistent
buffers come from the callbacks, every one is released through them with its
size, and the results are bitwise those of the default allocator."""

import numpy as np
import pytest

from paper_1405_4524_gb300 import inputs

pytestmark = pytest.mark.gpu


def run(sq, ctx, spec, U, eta):
    sq.sq_load_gauge(ctx, U, 12)
    sol = np.zeros_like(eta)
    sq.sq_solve(ctx, spec["kappa"], spec["csw"], eta, sol, eta.shape[0], 1e-10)
    O, C = sq.sq_contract_stoch_op(ctx, eta, sol, eta.shape[0])
    return sol, O, C


def test_callbacks_own_every_persistent_buffer():
    import torch
    from paper_1405_4524_gb300 import stochq as sq

    spec, U, eta = inputs.workload("4x4x4x8", n_rhs=3)
    live = {}
    log = {"alloc": 0, "free": 0}

    def alloc(nbytes, stream):
        p = torch.cuda.caching_allocator_alloc(nbytes, torch.cuda.current_device(), stream or 0)
        live[p] = nbytes
        log["alloc"] += 1
        return p

    def free(ptr, nbytes, stream):
        assert live.pop(ptr) == nbytes
        torch.cuda.caching_allocator_delete(ptr)
        log["free"] += 1

    ref_ctx = sq.sq_create(spec["dims"], -1)
    try:
        ref = run(sq, ref_ctx, spec, U, eta)
    finally:
        sq.sq_destroy(ref_ctx)
    ctx = sq.sq_create(spec["dims"], -1)
    try:
        sq.sq_set_allocator(ctx, alloc, free)
        got = run(sq, ctx, spec, U, eta)
        assert log["alloc"] >= 6  # two gauge copies, three clover arrays, a workspace, scratch
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        with pytest.raises(sq.StochqError) as ex:
            sq.sq_set_allocator(ctx, None, None)
        assert ex.value.status == sq.SQ_ERR_STATE
    finally:
        sq.sq_destroy(ctx)
    assert not live and log["free"] == log["alloc"]


def test_torch_allocator_and_argument_errors():
    import torch
    from paper_1405_4524_gb300 import stochq as sq

    spec, U, eta = inputs.workload("4x4x4x8", n_rhs=2)
    ctx = sq.sq_create(spec["dims"], -1)
    try:
        assert sq._lib.sq_set_allocator(ctx, 1, None, None) == sq.SQ_ERR_ARG
        with pytest.raises(ValueError):
            sq.sq_set_allocator(ctx, lambda n, s: 0, None)
        before = torch.cuda.memory_allocated()
        sq.use_torch_allocator(ctx)
        sq.sq_load_gauge(ctx, U, 12)
        assert torch.cuda.memory_allocated() > before
        sol = np.zeros_like(eta)
        st, stats = sq.sq_solve(ctx, spec["kappa"], spec["csw"], eta, sol, 2, 1e-10)
        assert st == 0 and max(s["true_residual"] for s in stats) <= 1e-10
    finally:
        sq.sq_destroy(ctx)
