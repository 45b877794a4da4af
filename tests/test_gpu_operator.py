"""GPU parity of the layout conversion (G0), the even-odd hopping kernels
(G1, every precision and fused variant), the clover build (G2) and the
full FP64 operator (G8), against the FP64 oracle, through the C ABI.

Tolerances (relative L2 per source over the output parity's sites):
FP64 1e-13, FP32 1e-6, FP16 (per-site norm) 5e-3.
"""

import numpy as np
import pytest

import oracle
from gpu_helpers import Setup, device_buffer, random_spinors, rel

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 1e-6, 2: 5e-3}

# several CTA tiles, ragged tails (Vh not a multiple of 32/64/128), odd
# half-extents, and a 2-wide direction
LATTICES = [(4, 4, 4, 8), (6, 4, 2, 10), (8, 6, 4, 6), (2, 2, 2, 4)]


@pytest.fixture(scope="module", params=LATTICES, ids=lambda d: "x".join(map(str, d)))
def setup(request):
    s = Setup(request.param, eps=0.4, seed=11)
    yield s
    s.close()


def roundtrip(s, psi, parity, prec):
    sq = s.sq
    n = psi.shape[0]
    buf = device_buffer(sq.sq_field_bytes(s.ctx, prec, n))
    sq.sq_pack_spinor(s.ctx, buf, psi, parity, prec, n)
    out = np.zeros_like(psi)
    sq.sq_unpack_spinor(s.ctx, out, buf, parity, prec, n)
    return out


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_pack_unpack_roundtrip(setup, prec):
    s = setup
    psi = random_spinors(s.dims, 3, 5)
    for p in (0, 1):
        got = roundtrip(s, psi, p, prec)
        want = oracle.restrict(psi, s.par, p)
        if prec == 0:
            assert np.array_equal(got, want)
        else:
            # FP32: round to nearest; FP16: per-site norm, 11-bit mantissa
            bound = 2.0 ** -24 if prec == 1 else 2.0 ** -11
            site_max = np.max(np.abs(np.stack([want.real, want.imag])), axis=(0, -1, -2),
                              keepdims=True)[0]
            err = np.abs(got - want)
            assert np.all(err <= 2 * bound * np.maximum(site_max, np.abs(want)) + 1e-300)
        # the other parity is untouched (zero here)
        assert np.all(oracle.restrict(got, s.par, 1 - p) == 0)


def oracle_dslash(s, psi_in, x, p_out, kappa, csw, clover, xpay, a):
    w = oracle.hopping_eo(s.U, psi_in, p_out, s.par, s.t_bc)
    if clover:
        w = oracle.site_apply(s.Ainv(kappa, csw), w)
    if xpay:
        w = x + a * w
    return oracle.restrict(w, s.par, p_out)


@pytest.mark.parametrize("prec,recon", [(0, 18), (1, 12), (1, 18), (2, 12), ("f64_emulated", 18)])
@pytest.mark.parametrize("clover,xpay", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_dslash_eo(setup, prec, recon, clover, xpay):
    """FP64, FP32 and FP16 fields; "f64_emulated": FP64 fields through the
    double-FP32 kernel the mixed solvers use for their FP64 steps (same
    tolerance as FP64)."""
    s = setup
    emul = 0
    if prec == "f64_emulated":
        prec, emul = 0, s.sq.SQ_DS_F64_EMULATED
    sq = s.sq
    if recon == 18:
        sq.sq_load_gauge(s.ctx, s.U, 18)
    kappa, csw, a = 0.121, 1.0, -0.37
    if clover:
        sq.sq_build_clover(s.ctx, kappa, csw)
    n = 3
    psi = random_spinors(s.dims, n, 21)
    x = random_spinors(s.dims, n, 22)
    for p_out in (0, 1):
        fb = sq.sq_field_bytes(s.ctx, prec, n)
        bin_, bx, bout = device_buffer(fb), device_buffer(fb), device_buffer(fb)
        sq.sq_pack_spinor(s.ctx, bin_, psi, 1 - p_out, prec, n)
        sq.sq_pack_spinor(s.ctx, bx, x, p_out, prec, n)
        flags = (sq.SQ_DS_CLOVER_INV if clover else 0) | (sq.SQ_DS_XPAY if xpay else 0) | emul
        sq.sq_dslash_eo(s.ctx, bout, bin_, bx if xpay else None, p_out, prec, n,
                        flags | sq.SQ_DS_SYNC, a)
        got = np.zeros_like(psi)
        sq.sq_unpack_spinor(s.ctx, got, bout, p_out, prec, n)
        for k in range(n):
            want = oracle_dslash(s, psi[k], x[k], p_out, kappa, csw, clover, xpay, a)
            assert rel(got[k], want) < TOL[prec], (k, p_out)
    if recon == 18:
        sq.sq_load_gauge(s.ctx, s.U, 12)


@pytest.mark.parametrize("t_bc", [-1, 1])
def test_full_operator_fp64(t_bc):
    dims = (4, 4, 4, 8)
    s = Setup(dims, eps=0.5, seed=3, t_bc=t_bc)
    try:
        psi = random_spinors(dims, 2, 8)
        for kappa, csw in [(0.115, 1.0), (0.13, 1.7)]:
            out = np.zeros_like(psi)
            s.sq.sq_apply_M(s.ctx, out, psi, 2, kappa, csw)
            for k in range(2):
                want = oracle.apply_M(s.U, s.F, psi[k], kappa, csw, float(t_bc))
                assert rel(out[k], want) < 1e-13
    finally:
        s.close()


def test_singular_clover_is_reported():
    """Constant abelian background: A has eigenvalues 1 -+ kappa c_sw sin(th);
    kappa c_sw = 1/sin(th) makes a block exactly singular."""
    dims = (4, 4, 4, 4)
    X, Y, Z, T = dims
    U = np.zeros((T, Z, Y, X, 4, 3, 3), dtype=np.complex128)
    U[...] = np.eye(3)
    th = 2 * np.pi / 4
    xs = np.broadcast_to(np.arange(X)[None, None, None, :], (T, Z, Y, X))
    ys = np.broadcast_to(np.arange(Y)[None, None, :, None], (T, Z, Y, X))
    U[..., 0, 0, 0] = np.exp(1j * th * ys)  # U_x depends on y: F_xy != 0
    U[..., 0, 1, 1] = np.exp(-1j * th * ys)
    del xs
    from paper_1405_4524_gb300 import stochq as sq

    ctx = sq.sq_create(dims, -1)
    try:
        sq.sq_load_gauge(ctx, U, 12)
        sq.sq_build_clover(ctx, 0.1, 1.0)  # regular
        with pytest.raises(sq.StochqError) as e:
            sq.sq_build_clover(ctx, 0.25, 1.0 / (0.25 * np.sin(th)))
        assert e.value.status == sq.SQ_ERR_CLOVER
    finally:
        sq.sq_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_norm2_eo(setup, prec):
    """Per-source squared norms of a device field against numpy on the
    unpacked (stored) values; bitwise reproducible on a second call."""
    s = setup
    sq = s.sq
    n = 5
    psi = random_spinors(s.dims, n, 31)
    buf = device_buffer(sq.sq_field_bytes(s.ctx, prec, n))
    sq.sq_pack_spinor(s.ctx, buf, psi, 1, prec, n)
    stored = np.zeros_like(psi)
    sq.sq_unpack_spinor(s.ctx, stored, buf, 1, prec, n)
    want = np.sum(np.abs(stored.reshape(n, -1)) ** 2, axis=1)
    got = sq.sq_norm2_eo(s.ctx, buf, prec, n)
    assert np.allclose(got, want, rtol=1e-13, atol=0)
    again = sq.sq_norm2_eo(s.ctx, buf, prec, n)
    assert np.array_equal(got, again)
