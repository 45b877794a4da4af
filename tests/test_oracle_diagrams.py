"""Pins of the diagram-contraction oracle (oracle/diagrams.py) against things
other than itself: explicit site loops, the gamma5-hermiticity form of
Diagram 2 from other blocks of the same inverse, a complete basis of scaled
unit sources (for which the stochastic route of Eq. Sfill is exact), the
statistical unbiasedness of two independent Z4 sets, the pion contraction of
the point solutions, the sample-covariance form of the vacuum subtraction,
and the Gram rearrangement of Diagram 2 that the GPU path evaluates.
"""

import numpy as np
import pytest

import oracle
from oracle import diagrams as dg
from paper_1405_4524_gb300 import inputs
from test_oracle_pins import dense_M

KAPPA, CSW = 0.12, 1.0


def setup(dims, seed):
    U = inputs.make_links(dims, 0.25, seed)
    F = oracle.field_strength(U)
    Minv = np.linalg.inv(dense_M(U, F, KAPPA, CSW, -1.0, dims))
    return U, Minv


def point_solutions(Minv, dims):
    """Xp[a] = M^{-1} e_a, e_a the unit source of spin-colour a at the origin."""
    X, Y, Z, T = dims
    return Minv[:, :12].T.reshape(12, T, Z, Y, X, 4, 3).copy()


def solve_all(Minv, eta):
    n = eta.shape[0]
    return (Minv @ eta.reshape(n, -1).T).T.reshape(eta.shape)


@pytest.fixture(scope="module")
def tiny():
    dims = (2, 2, 2, 2)
    U, Minv = setup(dims, 61)
    return dims, Minv


@pytest.fixture(scope="module")
def small():
    dims = (4, 2, 2, 4)
    U, Minv = setup(dims, 62)
    return dims, Minv


def test_exact_diagrams_site_loops(tiny):
    """Every formula of the module docstring with explicit loops over sites
    and 12 x 12 matrix products."""
    dims, Minv = tiny
    X, Y, Z, T = dims
    V3 = X * Y * Z
    S = Minv.reshape(T, V3, 12, T, V3, 12)

    def blk(t, i, t0, j):
        return S[t, i, :, t0, j, :]

    got = dg.diagrams_exact(Minv, dims)
    for t in range(T):
        P = sum(np.trace(blk(t, y, 0, 0) @ blk(t, y, 0, 0).conj().T) for y in range(V3))
        Q0 = sum(np.trace(blk(t, z, 0, x) @ blk(t, z, 0, x).conj().T) for x in range(V3) for z in range(V3))
        Qtt = sum(np.trace(blk(t, z, t, y) @ blk(t, z, t, y).conj().T) for y in range(V3) for z in range(V3))
        C2 = 0j
        for x in range(V3):
            for y in range(V3):
                for z in range(V3):
                    C2 += np.trace(blk(0, x, 0, 0).conj().T @ blk(0, x, t, z) @ blk(t, y, t, z).conj().T
                                   @ blk(t, y, 0, 0))
        assert np.allclose(got[0, t], P, rtol=1e-13, atol=0)
        assert np.allclose(got[1, t], Q0, rtol=1e-13, atol=0)
        assert np.allclose(got[2, t], Qtt, rtol=1e-13, atol=0)
        assert np.allclose(got[5, t], C2, rtol=1e-12, atol=1e-16)
    P0 = got[0, 0]
    assert np.allclose(got[3], got[0] * got[1])
    assert np.allclose(got[4], got[2] * P0)
    assert np.array_equal(got[6], np.conj(got[5]))
    # P, Q0, Qtt are real and positive; P(0) > 0
    assert np.all(np.abs(got[:3].imag) <= 1e-15 * np.abs(got[:3].real)) and np.all(got[:3].real > 0)


@pytest.mark.parametrize("which", ["tiny", "small"])
def test_diagram2_gamma5_hermiticity(which, tiny, small):
    """S(w;w')^+ = g5 S(w';w) g5 turns Diagram 2 into a product of four
    propagators read from other blocks of the inverse (a quark loop through
    the origin, (0,x), (t,z) and (t,y)): the same number."""
    dims, Minv = tiny if which == "tiny" else small
    got = dg.diagrams_exact(Minv, dims)
    for t in ([0, 1] if which == "tiny" else [0, 2]):
        alt = dg.c2_gamma5_form(Minv, dims, t)
        assert abs(got[5, t] - alt) <= 1e-12 * abs(alt)


def test_complete_basis_is_exact(tiny):
    """With N = 12V sources eta_i = sqrt(N) e_i (every unit vector), the filled
    propagator (1/N) sum_i X_i eta_i^+ is M^{-1} itself, so the stochastic
    route gives the exact diagrams (to rounding), for one set and two."""
    dims, Minv = tiny
    X, Y, Z, T = dims
    N = 12 * X * Y * Z * T
    eta = (np.sqrt(N) * np.eye(N, dtype=np.complex128)).reshape(N, T, Z, Y, X, 4, 3)
    Xs = solve_all(Minv, eta)
    Xp = point_solutions(Minv, dims)
    exact = dg.diagrams_exact(Minv, dims)
    for got in (dg.diagrams_stochastic(Xp, eta, Xs), dg.diagrams_stochastic(Xp, eta, Xs, eta, Xs)):
        assert np.allclose(got, exact, rtol=1e-11, atol=1e-13 * np.max(np.abs(exact)))


def test_stochastic_estimates_are_unbiased(small):
    """Two independent Z4 sets: the mean of 24 independent estimates of each
    diagram lies within 5 standard errors of the exact value (real and
    imaginary parts of C2)."""
    dims, Minv = small
    exact = dg.diagrams_exact(Minv, dims)
    Xp = point_solutions(Minv, dims)
    n = 6
    est = []
    for r in range(24):
        eA = inputs.make_z4(dims, n, 11000 + 100 * r)
        eB = inputs.make_z4(dims, n, 11050 + 100 * r)
        est.append(dg.diagrams_stochastic(Xp, eA, solve_all(Minv, eA), eB, solve_all(Minv, eB)))
    est = np.array(est)
    for q in (1, 2, 3, 4, 5):
        for part in (np.real, np.imag):
            v = part(est[:, q])
            err = v.std(axis=0, ddof=1) / np.sqrt(len(v))
            dev = np.abs(v.mean(axis=0) - part(exact[q]))
            ok = (dev < 5.0 * err) | (dev <= 1e-12 * np.max(np.abs(exact[q])))
            assert np.all(ok), (dg.NAMES[q], part.__name__, dev / np.maximum(err, 1e-300))
    # P uses the exact point propagator: no noise at all
    assert np.allclose(est[:, 0], exact[0], rtol=1e-12)


def test_point_factor_is_the_pion_contraction(small):
    dims, Minv = small
    Xp = point_solutions(Minv, dims)
    eta = inputs.make_z4(dims, 2, 11900)
    got = dg.diagrams_stochastic(Xp, eta, solve_all(Minv, eta))
    P = sum(oracle.pion_correlator(Xp[a]) for a in range(12))
    assert np.allclose(got[0].real, P, rtol=1e-13)


def test_two_sets_trace_factors_match_the_filled_trace(small):
    """Q0 and Qtt are the t0 = 0 row and the diagonal of the (separately
    pinned) trace of filled propagators."""
    dims, Minv = small
    T = dims[3]
    Xp = point_solutions(Minv, dims)
    eA, eB = inputs.make_z4(dims, 4, 11700), inputs.make_z4(dims, 4, 11701)
    xA, xB = solve_all(Minv, eA), solve_all(Minv, eB)
    got = dg.diagrams_stochastic(Xp, eA, xA, eB, xB)
    Ct = oracle.stochastic_propagator_trace(eA, xA, eB, xB)
    assert np.allclose(got[1], Ct[0], rtol=1e-12)
    assert np.allclose(got[2], np.array([Ct[t, t] for t in range(T)]), rtol=1e-12)


def gram_c2(Xp, eA, xA, eB, xB):
    """Diagram 2 rearranged (the route of the GPU path):
    C2(t) = (1/N^2) sum_ij Q_ij(t) W_ji(t), Q_ij(t) = sum_{z in t} eA_i^+ eB_j,
    W_ji(t) = sum_a conj(GB(t)_aj) GA(0)_ai, G(t)_ai = sum_{x in t} Xp_a^+ X_i."""
    n = eA.shape[0]
    Q = np.einsum("itzyxsc,jtzyxsc->tij", np.conj(eA), eB)
    GA = np.einsum("atzyxsc,itzyxsc->tai", np.conj(Xp), xA)
    GB = np.einsum("atzyxsc,itzyxsc->tai", np.conj(Xp), xB)
    W = np.einsum("taj,ai->tji", np.conj(GB), GA[0])
    return np.einsum("tij,tji->t", Q, W) / (n * n)


def test_gram_rearrangement_of_diagram2(small):
    dims, Minv = small
    Xp = point_solutions(Minv, dims)
    eA, eB = inputs.make_z4(dims, 5, 11800), inputs.make_z4(dims, 5, 11801)
    xA, xB = solve_all(Minv, eA), solve_all(Minv, eB)
    lit = dg.diagrams_stochastic(Xp, eA, xA, eB, xB)[5]
    assert np.allclose(gram_c2(Xp, eA, xA, eB, xB), lit, rtol=1e-12, atol=1e-14 * np.max(np.abs(lit)))


def test_ensemble_subtraction_is_a_covariance():
    """<AB> - <A><B> is the biased sample covariance of A and B."""
    rng = np.random.default_rng(5)
    ncfg, T = 40, 6
    rec = np.zeros((ncfg, 7, T), dtype=np.complex128)
    rec[:, 0] = 1 + rng.random((ncfg, T))
    rec[:, 1] = 2 + rng.random((ncfg, T)) + 0.3 * rec[:, 0]
    rec[:, 2] = 3 + rng.random((ncfg, T))
    rec[:, 3] = rec[:, 0] * rec[:, 1]
    rec[:, 4] = rec[:, 2] * rec[:, 0, :1]
    rec[:, 5] = rng.random((ncfg, T)) + 1j * rng.random((ncfg, T))
    rec[:, 6] = np.conj(rec[:, 5])
    out = dg.ensemble(rec)
    for t in range(T):
        c0 = np.cov(rec[:, 0, t].real, rec[:, 1, t].real, bias=True)[0, 1]
        c1 = np.cov(rec[:, 2, t].real, rec[:, 0, 0].real, bias=True)[0, 1]
        assert np.isclose(out[0, t], c0, rtol=1e-12)
        assert np.isclose(out[1, t], c1, rtol=1e-12)
    assert np.allclose(out[2], rec[:, 5].mean(axis=0))
    assert np.allclose(out[4], out[0] + out[1] - out[2] - out[3])
    assert np.allclose(out[4].imag, 0, atol=1e-15)
