"""The allocation-free norm entry point, through the C ABI.

sq_norm2_eo_noalloc serves callers that must not allocate device memory at
the point of the call (for instance while another thread captures a CUDA
graph, or under a framework whose pool owns the device memory). It keeps its
reduction scratch in a static device array instead. This checks, for every
field precision, that two calls in a row give the same per-source norms as
the allocating sq_norm2_eo within the FP64 tolerance of the other tests,
and that sizes beyond its stated maximum are refused. It runs last so that
a failure here cannot hide any other test's result; it also passes alone
in a fresh process.
"""

import numpy as np
import pytest

from gpu_helpers import Setup, device_buffer, random_spinors

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_noalloc_norms_match_allocating_entry_point(prec):
    dims = (6, 4, 4, 10)  # ragged site count: Vh = 480
    s = Setup(dims, eps=0.3, seed=21)
    try:
        sq = s.sq
        n = 7
        psi = random_spinors(dims, n, 40 + prec)
        buf = device_buffer(sq.sq_field_bytes(s.ctx, prec, n))
        sq.sq_pack_spinor(s.ctx, buf, psi, 0, prec, n)
        ref = sq.sq_norm2_eo(s.ctx, buf, prec, n)
        first = sq.sq_norm2_eo_noalloc(s.ctx, buf, prec, n)
        second = sq.sq_norm2_eo_noalloc(s.ctx, buf, prec, n)
        assert np.allclose(first, ref, rtol=1e-13, atol=0)
        assert np.allclose(second, ref, rtol=1e-13, atol=0)
        assert np.all(ref > 0)
    finally:
        s.close()


def test_noalloc_device_output_and_limit():
    import torch

    dims = (4, 4, 4, 8)
    s = Setup(dims, eps=0.3, seed=22)
    try:
        sq = s.sq
        n = 3
        psi = random_spinors(dims, n, 50)
        buf = device_buffer(sq.sq_field_bytes(s.ctx, 1, n))
        sq.sq_pack_spinor(s.ctx, buf, psi, 1, 1, n)
        out = torch.zeros(n, dtype=torch.float64, device="cuda")
        sq.sq_norm2_eo_noalloc(s.ctx, buf, 1, n, out)
        torch.cuda.synchronize()
        ref = sq.sq_norm2_eo(s.ctx, buf, 1, n)
        assert np.allclose(out.cpu().numpy(), ref, rtol=1e-13, atol=0)
        with pytest.raises(sq.StochqError) as e:
            sq.sq_norm2_eo_noalloc(s.ctx, buf, 1, 257)
        assert e.value.status == sq.SQ_ERR_ARG
    finally:
        s.close()
