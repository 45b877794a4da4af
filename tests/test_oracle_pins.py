"""Pins of the FP64 oracle against things other than itself.

Each check below is chosen so that a plausible mistake in the oracle (a
dropped term, a wrong sign, a wrong neighbour index, a transposed or
un-daggered link, a wrong clover normalisation or leaf orientation, a broken
Krylov step) fails at least one of them:

* Dirac algebra of the gamma basis (Clifford relations, gamma5).
* Free field (all links 1): the momentum-space closed form of M and of
  M^{-1}, with antiperiodic time momenta.
* gamma5-hermiticity  <phi, g5 M g5 chi> = <M phi, chi>.
* gauge covariance   M[U^g] (g psi) = g M[U] psi.
* constant abelian background: closed-form clover term.
* dense LU on tiny lattices for BiCGStab and the even-odd formulas.
* the pion contraction against brute-force loops and against its exact
  expectation value from the dense inverse.
"""

import numpy as np
import pytest

import oracle
from oracle import dirac
from paper_1405_4524_gb300 import inputs


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def unit_links(dims):
    X, Y, Z, T = dims
    U = np.zeros((T, Z, Y, X, 4, 3, 3), dtype=np.complex128)
    U[...] = np.eye(3)
    return U


def random_spinor(dims, rng, n=None):
    X, Y, Z, T = dims
    sh = (T, Z, Y, X, 4, 3) if n is None else (n, T, Z, Y, X, 4, 3)
    return rng.standard_normal(sh) + 1j * rng.standard_normal(sh)


def random_su3(shape, rng):
    g = rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))
    q, r = np.linalg.qr(g)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[..., None, None]


# ---------------------------------------------------------------------------
# Dirac algebra
# ---------------------------------------------------------------------------

def test_gamma_clifford_and_gamma5():
    G = oracle.GAMMA
    for mu in range(4):
        assert np.allclose(G[mu], G[mu].conj().T)
        for nu in range(4):
            anti = G[mu] @ G[nu] + G[nu] @ G[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4))
    assert np.allclose(oracle.GAMMA5, np.diag([1, 1, -1, -1]))
    for mu in range(4):
        assert np.allclose(oracle.GAMMA5 @ G[mu], -G[mu] @ oracle.GAMMA5)


def test_sigma_block_diagonal_in_chirality():
    for mu, nu in oracle.PLANES:
        s = oracle.sigma(mu, nu)
        assert np.allclose(s, s.conj().T)
        assert np.allclose(s[:2, 2:], 0) and np.allclose(s[2:, :2], 0)


# ---------------------------------------------------------------------------
# Free field: closed-form momentum space
# ---------------------------------------------------------------------------

def free_M_of_p(p, kappa):
    """M(p) = (1 - 2 k sum cos p) + 2 i k sum g_mu sin p_mu (U = 1)."""
    a = 1.0 - 2.0 * kappa * np.sum(np.cos(p))
    return a * np.eye(4) + 2j * kappa * sum(
        oracle.GAMMA[mu] * np.sin(p[mu]) for mu in range(4))


@pytest.mark.parametrize("t_bc", [-1.0, 1.0])
def test_free_field_plane_waves(t_bc):
    dims = (4, 6, 4, 8)
    X, Y, Z, T = dims
    kappa, csw = 0.13, 1.0
    U = unit_links(dims)
    F = oracle.field_strength(U)
    assert np.allclose(F, 0)
    rng = np.random.default_rng(5)
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y),
                             np.arange(X), indexing="ij")
    shift4 = 0.5 if t_bc < 0 else 0.0
    for n in [(0, 0, 0, 0), (1, 2, 3, 5), (3, 5, 1, 7), (2, 0, 1, 2)]:
        p = np.array([2 * np.pi * n[0] / X, 2 * np.pi * n[1] / Y,
                      2 * np.pi * n[2] / Z, 2 * np.pi * (n[3] + shift4) / T])
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        psi = phase[..., None, None] * u
        got = oracle.apply_M(U, F, psi, kappa, csw, t_bc)
        want = phase[..., None, None] * (free_M_of_p(p, kappa) @ u)
        assert rel(got, want) < 1e-13


def free_propagator_fft(eta, dims, kappa):
    """psi = M^{-1} eta at U = 1, antiperiodic time, by FFT.

    Momenta p_i = 2 pi k_i / L_i, p_4 = (2 k_4 + 1) pi / T; the half-integer
    time momentum is carried by the twist exp(-i pi t / T). With
    a = 1 - 2k sum cos p and s_mu = sin p_mu:
    M(p)^{-1} = (a - 2 i k g.s) / (a^2 + 4 k^2 s.s).
    """
    X, Y, Z, T = dims
    tw = np.exp(1j * np.pi * np.arange(T) / T)[:, None, None, None, None, None]
    eh = np.fft.fftn(eta / tw, axes=(0, 1, 2, 3))
    kt, kz, ky, kx = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y),
                                 np.arange(X), indexing="ij")
    p = [2 * np.pi * kx / X, 2 * np.pi * ky / Y, 2 * np.pi * kz / Z,
         2 * np.pi * (kt + 0.5) / T]
    a = 1.0 - 2.0 * kappa * sum(np.cos(q) for q in p)
    s = [np.sin(q) for q in p]
    den = a ** 2 + 4 * kappa ** 2 * sum(q ** 2 for q in s)
    Minv = a[..., None, None] * np.eye(4) - 2j * kappa * sum(
        oracle.GAMMA[mu] * s[mu][..., None, None] for mu in range(4))
    Minv = Minv / den[..., None, None]
    ph = Minv @ eh
    return np.fft.ifftn(ph, axes=(0, 1, 2, 3)) * tw


def test_free_field_propagator_closed_form():
    dims = (4, 4, 6, 8)
    kappa = 0.124
    U = unit_links(dims)
    rng = np.random.default_rng(7)
    eta = random_spinor(dims, rng)
    want = free_propagator_fft(eta, dims, kappa)
    F = oracle.field_strength(U)
    # apply_M of the closed-form solution gives back the source
    assert rel(oracle.apply_M(U, F, want, kappa, 1.0, -1.0), eta) < 1e-13
    # and the oracle's BiCGStab finds the same solution
    got, it, res = oracle.solve(U, eta, kappa, 1.0, -1.0, tol=1e-13)
    assert res <= 1e-13
    assert rel(got, want) < 1e-11


# ---------------------------------------------------------------------------
# Invariants on random gauge fields (with the clover term)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def rough_field():
    dims = (4, 4, 4, 6)
    U = inputs.make_links(dims, 0.8, 77)
    return dims, U, oracle.field_strength(U)


def test_gamma5_hermiticity(rough_field):
    dims, U, F = rough_field
    rng = np.random.default_rng(11)
    phi, chi = random_spinor(dims, rng), random_spinor(dims, rng)
    g5 = lambda v: oracle.GAMMA5 @ v
    for kappa, csw in [(0.12, 1.0), (0.2, 2.5)]:
        lhs = oracle.inner(phi, g5(oracle.apply_M(U, F, g5(chi), kappa, csw)))
        rhs = oracle.inner(oracle.apply_M(U, F, phi, kappa, csw), chi)
        assert abs(lhs - rhs) / abs(rhs) < 1e-13


def test_gauge_covariance(rough_field):
    dims, U, F = rough_field
    X, Y, Z, T = dims
    rng = np.random.default_rng(12)
    g = random_su3((T, Z, Y, X), rng)
    Ug = np.empty_like(U)
    for mu in range(4):
        g_fwd = oracle.shift(g, mu, +1, 2, 1.0)
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ oracle.dagger(g_fwd)
    Fg = oracle.field_strength(Ug)
    psi = random_spinor(dims, rng)
    gpsi = psi @ np.swapaxes(g, -1, -2)  # colour rotation at every site
    kappa, csw = 0.125, 1.3
    lhs = oracle.apply_M(Ug, Fg, gpsi, kappa, csw)
    rhs = oracle.apply_M(U, F, psi, kappa, csw) @ np.swapaxes(g, -1, -2)
    assert rel(lhs, rhs) < 1e-13


def test_clover_structure(rough_field):
    dims, U, F = rough_field
    assert np.allclose(np.trace(F, axis1=-2, axis2=-1), 0, atol=1e-14)
    assert np.allclose(F, -oracle.dagger(F), atol=1e-14)
    A = oracle.clover_matrices(F, 0.12, 1.0)
    assert np.allclose(A, oracle.dagger(A), atol=1e-14)
    assert np.allclose(A[..., :6, 6:], 0, atol=1e-15)
    assert np.allclose(A[..., 6:, :6], 0, atol=1e-15)
    # the explicit matrices and the operator form agree
    rng = np.random.default_rng(3)
    psi = random_spinor(dims, rng)
    assert rel(oracle.site_apply(A, psi),
               oracle.clover_apply(F, psi, 0.12, 1.0)) < 1e-14


@pytest.mark.parametrize("mu,nu,n", [(0, 2, 1), (3, 1, 1), (1, 3, 2)])
def test_constant_abelian_background(mu, nu, n):
    """U_mu(x) = diag(e^{i th x_nu}, e^{-i th x_nu}, 1), th = 2 pi n / L_nu,
    all other links 1. Every mu-nu leaf is diag(e^{-i th}, e^{i th}, 1), so
    Fhat_mu_nu = i diag(-sin th, sin th, 0) and all other planes vanish."""
    dims = (4, 4, 6, 8)
    X, Y, Z, T = dims
    U = unit_links(dims)
    coord = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y),
                        np.arange(X), indexing="ij")[::-1]  # x, y, z, t
    th = 2 * np.pi * n / dims[nu]
    phi = th * coord[nu]
    U[..., mu, 0, 0] = np.exp(1j * phi)
    U[..., mu, 1, 1] = np.exp(-1j * phi)
    F = oracle.field_strength(U)
    f = 1j * np.diag([-np.sin(th), np.sin(th), 0.0])
    kappa, csw = 0.11, 1.7
    for p, (a, b) in enumerate(oracle.PLANES):
        if (a, b) == (mu, nu):
            want = f
        elif (a, b) == (nu, mu):
            want = -f
        else:
            want = np.zeros((3, 3))
        assert np.allclose(F[..., p, :, :], want, atol=1e-14)
    s = oracle.sigma(mu, nu)
    A_want = np.eye(12) + 1j * kappa * csw * np.kron(s, f)
    A = oracle.clover_matrices(F, kappa, csw)
    assert np.allclose(A, A_want, atol=1e-14)


# ---------------------------------------------------------------------------
# Dense linear algebra on tiny lattices
# ---------------------------------------------------------------------------

def dense_M(U, F, kappa, csw, t_bc, dims):
    X, Y, Z, T = dims
    n = X * Y * Z * T * 12
    basis = np.eye(n, dtype=np.complex128).reshape(n, T, Z, Y, X, 4, 3)
    cols = oracle.apply_M(U, F, basis, kappa, csw, t_bc)
    return cols.reshape(n, n).T


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4)])
def test_dense_lu_vs_bicgstab(dims):
    U = inputs.make_links(dims, 0.25, 31)
    F = oracle.field_strength(U)
    kappa, csw = 0.12, 1.0
    M = dense_M(U, F, kappa, csw, -1.0, dims)
    # gamma5-hermiticity at the matrix level: g5 M g5 = M^dag
    V = np.prod(dims)
    G5 = np.kron(np.eye(V), np.kron(oracle.GAMMA5, np.eye(3)))
    assert np.allclose(G5 @ M @ G5, M.conj().T, atol=1e-14)
    eta = inputs.make_z4(dims, 1, 99)[0]
    exact = np.linalg.solve(M, eta.reshape(-1)).reshape(eta.shape)
    got, it, res = oracle.solve(U, eta, kappa, csw, -1.0, tol=1e-13)
    assert res <= 1e-13
    assert rel(got, exact) < 1e-12


def test_schur_formulas_vs_dense():
    dims = (4, 2, 2, 4)
    U = inputs.make_links(dims, 0.5, 41)
    F = oracle.field_strength(U)
    kappa, csw = 0.13, 1.0
    par = oracle.parity_field(dims)
    A = oracle.clover_matrices(F, kappa, csw)
    Ainv = np.linalg.inv(A)
    eta = inputs.make_z4(dims, 1, 7)[0]
    M = dense_M(U, F, kappa, csw, -1.0, dims)
    exact = np.linalg.solve(M, eta.reshape(-1)).reshape(eta.shape)
    # the exact solution's even part solves the Schur system
    b = oracle.schur_source(U, Ainv, eta, kappa, par)
    lhs = oracle.schur_apply(U, Ainv, oracle.restrict(exact, par, 0), kappa, par)
    assert rel(lhs, b) < 1e-13
    # and the reconstruction gives back the full solution
    psi = oracle.schur_reconstruct(U, Ainv, eta, oracle.restrict(exact, par, 0),
                                   kappa, par)
    assert rel(psi, exact) < 1e-13
    # BiCGStab on the Schur system, reconstructed
    xe, it, res = oracle.bicgstab(
        lambda v: oracle.schur_apply(U, Ainv, v, kappa, par), b, tol=1e-13)
    psi2 = oracle.schur_reconstruct(U, Ainv, eta, xe, kappa, par)
    assert rel(psi2, exact) < 1e-12


def test_bicgstab_on_a_random_matrix():
    rng = np.random.default_rng(2)
    n = 300
    A = np.eye(n) * 4 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, it, res = oracle.bicgstab(lambda v: A @ v, b, tol=1e-13)
    assert res <= 1e-13
    assert rel(x, np.linalg.solve(A, b)) < 1e-12


# ---------------------------------------------------------------------------
# Pion contraction
# ---------------------------------------------------------------------------

def test_pion_correlator_brute_force():
    dims = (2, 2, 2, 4)
    X, Y, Z, T = dims
    rng = np.random.default_rng(9)
    psi = random_spinor(dims, rng)
    for t0 in [0, 3]:
        C = oracle.pion_correlator(psi, t0)
        for dt in range(T):
            acc = 0.0
            for z in range(Z):
                for y in range(Y):
                    for x in range(X):
                        for s in range(4):
                            for c in range(3):
                                v = psi[(t0 + dt) % T, z, y, x, s, c]
                                acc += v.real ** 2 + v.imag ** 2
            assert abs(C[dt] - acc) <= 1e-13 * acc


def test_pion_stochastic_estimate_matches_exact():
    """E_eta[C(t)] = sum_{x in t} sum_y tr[S(x,y) S(x,y)^dag] for Z4 eta,
    where S = M^{-1} comes from the dense LU inverse."""
    dims = (4, 2, 2, 4)
    X, Y, Z, T = dims
    U = inputs.make_links(dims, 0.25, 51)
    F = oracle.field_strength(U)
    kappa, csw = 0.12, 1.0
    M = dense_M(U, F, kappa, csw, -1.0, dims)
    S = np.linalg.inv(M)
    per_row = np.sum(np.abs(S) ** 2, axis=1).reshape(T, Z, Y, X, 4, 3)
    exact = per_row.sum(axis=(1, 2, 3, 4, 5))
    n = 48
    eta = inputs.make_z4(dims, n, 500)
    psi = (S @ eta.reshape(n, -1).T).T.reshape(eta.shape)
    Cs = np.array([oracle.pion_correlator(psi[k]) for k in range(n)])
    mean = Cs.mean(axis=0)
    err = Cs.std(axis=0, ddof=1) / np.sqrt(n)
    z = np.abs(mean - exact) / err
    assert np.all(z < 4.0), z


# ---------------------------------------------------------------------------
# Stochastic-operator contraction (Eq. stoop)
# ---------------------------------------------------------------------------

def test_stochastic_operator_brute_force():
    """O_ij(t) and its correlator against explicit loops, with gamma5 of the
    DeGrand-Rossi basis written out as diag(1, 1, -1, -1)."""
    dims = (2, 2, 2, 4)
    X, Y, Z, T = dims
    rng = np.random.default_rng(21)
    n = 3
    eta = np.stack([random_spinor(dims, rng) for _ in range(n)])
    sol = np.stack([random_spinor(dims, rng) for _ in range(n)])
    O = oracle.stochastic_operator(eta, sol)
    g5 = [1.0, 1.0, -1.0, -1.0]
    ref = np.zeros((T, n, n), dtype=np.complex128)
    for t in range(T):
        for i in range(n):
            for j in range(n):
                acc = 0j
                for z in range(Z):
                    for y in range(Y):
                        for x in range(X):
                            for s in range(4):
                                for c in range(3):
                                    acc += np.conj(eta[i, t, z, y, x, s, c]) * g5[s] * sol[j, t, z, y, x, s, c]
                ref[t, i, j] = acc
    assert np.max(np.abs(O - ref)) <= 1e-13 * np.max(np.abs(ref))
    C = oracle.stochastic_operator_correlator(O)
    for dt in range(T):
        acc = 0j
        for t0 in range(T):
            for i in range(n):
                for j in range(n):
                    acc += ref[(t0 + dt) % T, i, j] * ref[t0, j, i]
        assert abs(C[dt] - acc / (n * n * T)) <= 1e-13 * abs(acc / (n * n * T))


def test_stochastic_operator_of_the_noise_itself():
    """With X_j = eta_j and Z4 noise the diagonal O_ii(t) vanishes exactly
    (|eta| = 1 everywhere and gamma5 is traceless over spin), and
    O_ji(t) = conj(O_ij(t)) (gamma5 is Hermitian)."""
    dims = (2, 2, 2, 4)
    eta = inputs.make_z4(dims, 4, 33)
    O = oracle.stochastic_operator(eta, eta)
    assert np.all(np.abs(np.einsum("tii->ti", O)) == 0.0)
    assert np.allclose(O, np.conj(np.transpose(O, (0, 2, 1))), rtol=0, atol=1e-14)


def test_stochastic_operator_estimate_matches_exact():
    """For Z4 noise the i != j terms of O_ij(t0 + dt) O_ji(t0) estimate
    sum_{x in t0, y in t0+dt} |S(x, y)|_F^2 (gamma5-hermiticity), S = M^{-1}
    from the dense LU inverse; averaged over t0."""
    dims = (4, 2, 2, 4)
    X, Y, Z, T = dims
    U = inputs.make_links(dims, 0.25, 52)
    F = oracle.field_strength(U)
    kappa, csw = 0.12, 1.0
    M = dense_M(U, F, kappa, csw, -1.0, dims)
    S = np.linalg.inv(M)
    nsite = T * Z * Y * X
    B = np.abs(S.reshape(nsite, 12, nsite, 12)) ** 2
    blk = B.sum(axis=(1, 3)).reshape(T, Z * Y * X, T, Z * Y * X).sum(axis=(1, 3))  # [t_x, t_y]
    exact = np.array([np.mean([blk[t0, (t0 + dt) % T] for t0 in range(T)]) for dt in range(T)])
    n = 40
    eta = inputs.make_z4(dims, n, 600)
    sol = (S @ eta.reshape(n, -1).T).T.reshape(eta.shape)
    O = oracle.stochastic_operator(eta, sol)
    # per pair (i < j) estimates, symmetrised, averaged over t0
    est = []
    for i in range(n):
        for j in range(i + 1, n):
            e = [np.mean([O[(t0 + dt) % T, i, j] * O[t0, j, i] + O[(t0 + dt) % T, j, i] * O[t0, i, j]
                          for t0 in range(T)]) / 2 for dt in range(T)]
            est.append(np.real(e))
    est = np.array(est)
    mean = est.mean(axis=0)
    err = est.std(axis=0, ddof=1) / np.sqrt(len(est))
    z = np.abs(mean - exact) / err
    assert np.all(z < 5.0), (z, mean, exact)
    # the correlator function (all pairs, i = j included as in the paper's
    # sum) is the off-diagonal estimate plus the diagonal terms
    C = oracle.stochastic_operator_correlator(O)
    off = np.zeros(T, dtype=np.complex128)
    diag = np.zeros(T, dtype=np.complex128)
    for dt in range(T):
        for t0 in range(T):
            P = O[(t0 + dt) % T] * O[t0].T  # P_ij = O_ij(t0 + dt) O_ji(t0)
            diag[dt] += np.trace(P) / T
            off[dt] += (P.sum() - np.trace(P)) / T
    assert np.allclose(np.real(off) / (n * (n - 1)), mean, rtol=1e-10, atol=0)
    assert np.allclose(C * n * n, off + diag, rtol=1e-10, atol=0)


# ---------------------------------------------------------------------------
# traces of filled stochastic propagators (Eq. Sfill, Table Lcomp)
# ---------------------------------------------------------------------------

def test_propagator_trace_brute_force():
    """Eq. Sfill filled site pair by site pair with outer products of the
    12-component site vectors, and tr[S_A S_B^dag] summed over every source
    site on t0 and sink site on t, for two sets on a 2^4 lattice; one set
    is the two-set formula with B = A."""
    dims = (2, 2, 2, 2)
    X, Y, Z, T = dims
    n = 2
    rng = np.random.default_rng(41)
    eA, xA, eB, xB = (random_spinor(dims, rng, n) for _ in range(4))
    C = oracle.stochastic_propagator_trace(eA, xA, eB, xB)
    sites = [(z, y, x) for z in range(Z) for y in range(Y) for x in range(X)]
    for t0 in range(T):
        for t in range(T):
            acc = 0j
            for src in sites:
                for snk in sites:
                    SA = np.zeros((12, 12), dtype=np.complex128)
                    SB = np.zeros((12, 12), dtype=np.complex128)
                    for i in range(n):
                        SA += np.outer(xA[i][(t,) + snk].reshape(12), np.conj(eA[i][(t0,) + src].reshape(12))) / n
                        SB += np.outer(xB[i][(t,) + snk].reshape(12), np.conj(eB[i][(t0,) + src].reshape(12))) / n
                    acc += np.trace(SA @ SB.conj().T)
            assert abs(C[t0, t] - acc) <= 1e-12 * abs(acc)
    assert np.allclose(oracle.stochastic_propagator_trace(eA, xA), oracle.stochastic_propagator_trace(eA, xA, eA, xA),
                       rtol=1e-14, atol=0)


def test_propagator_trace_point_source_limit():
    """Twelve spin-colour point sources at one site of timeslice t0 in place
    of noise: the fill is the point propagator from that site divided by
    N_r = 12, so C[t0, t] = (1/144) sum_k sum_{z in t} |X_k(z)|^2, the pion
    contraction of the twelve columns (pinned separately), and every other
    source timeslice gives zero."""
    dims = (2, 2, 2, 4)
    T = dims[3]
    t0, site = 1, (1, 0, 1)
    eta = np.zeros((12, T, 2, 2, 2, 4, 3), dtype=np.complex128)
    for k in range(12):
        eta[k][(t0,) + site].reshape(12)[k] = 1.0
    Xk = random_spinor(dims, np.random.default_rng(43), 12)
    C = oracle.stochastic_propagator_trace(eta, Xk)
    want = sum(oracle.pion_correlator(Xk[k], t0) for k in range(12)) / 144.0
    for t in range(T):
        assert abs(C[t0, t] - want[(t - t0) % T]) <= 1e-13 * abs(want[(t - t0) % T])
    assert np.all(C[[t for t in range(T) if t != t0]] == 0)


def test_propagator_trace_estimate_matches_exact():
    """Two independent Z4 sets with X = M^{-1} eta: the expectation of C[t0, t]
    is sum over x on t0 and z on t of ||M^{-1}(z, x)||_F^2 (E[eta eta^dag] = 1
    per set, the sets independent), from the dense LU inverse on 4x2x2x4; the
    mean of 24 independent estimates agrees within 5 standard errors."""
    dims = (4, 2, 2, 4)
    X, Y, Z, T = dims
    U = inputs.make_links(dims, 0.25, 52)
    F = oracle.field_strength(U)
    M = dense_M(U, F, 0.12, 1.0, -1.0, dims)
    S = np.linalg.inv(M)
    nsite = T * Z * Y * X
    B = np.abs(S.reshape(nsite, 12, nsite, 12)) ** 2
    blk = B.sum(axis=(1, 3)).reshape(T, Z * Y * X, T, Z * Y * X).sum(axis=(1, 3))  # [t_sink, t_source]
    n = 8
    est = []
    for r in range(24):
        eA = inputs.make_z4(dims, n, 9000 + 100 * r)
        eB = inputs.make_z4(dims, n, 9050 + 100 * r)
        xA = (S @ eA.reshape(n, -1).T).T.reshape(eA.shape)
        xB = (S @ eB.reshape(n, -1).T).T.reshape(eB.shape)
        est.append(oracle.stochastic_propagator_trace(eA, xA, eB, xB))
    est = np.array(est)
    mean = np.real(est.mean(axis=0))
    err = np.real(est).std(axis=0, ddof=1) / np.sqrt(len(est))
    exact = blk.T  # [t0, t]
    z = np.abs(mean - exact) / err
    assert np.all(z < 5.0), (z, mean, exact)


def test_propagator_trace_gram_identity():
    """The fill route equals the Gram-matrix form used without the fill:
    C[t0, t] = (1/N_r^2) sum_ij P_ji(t) Q_ij(t0), P_ji(t) = sum_{z in t}
    XB_j^dag XA_i, Q_ij(t0) = sum_{x in t0} etaA_i^dag etaB_j; the identity
    is then checked at sizes where the fill cannot be stored."""
    dims = (2, 2, 4, 4)
    T = dims[3]
    n = 5
    rng = np.random.default_rng(47)
    eA, xA, eB, xB = (random_spinor(dims, rng, n) for _ in range(4))
    C = oracle.stochastic_propagator_trace(eA, xA, eB, xB)
    G = np.zeros((T, T), dtype=np.complex128)
    for t0 in range(T):
        for t in range(T):
            for i in range(n):
                for j in range(n):
                    P = np.vdot(xB[j, t], xA[i, t])
                    Q = np.vdot(eA[i, t0], eB[j, t0])
                    G[t0, t] += P * Q
    assert np.allclose(C, G / n**2, rtol=1e-12, atol=0)


# ---------------------------------------------------------------------------
# dilution (time, spin-colour, full) and point sources
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("scheme,D", [("time", 4), ("spin_colour", 12), ("full", 48)])
def test_dilution_completeness_and_supports(scheme, D):
    """The D sources of a noise vector sum to it, their supports are
    disjoint, and each keeps exactly its timeslice / component (explicit
    loops over the index space)."""
    dims = (2, 2, 2, 4)
    noise = inputs.make_z4(dims, 2, 81)
    out = oracle.dilute(noise, scheme)
    assert out.shape == (2 * D,) + noise.shape[1:]
    for k in range(2):
        blk = out[k * D:(k + 1) * D]
        assert np.array_equal(blk.sum(axis=0), noise[k])
        assert np.all(np.count_nonzero(blk, axis=0) == 1)  # Z4 noise is nowhere zero
        for d in range(D):
            for t in range(4):
                for s in range(4):
                    for c in range(3):
                        a = 3 * s + c
                        keep = {"time": t == d, "spin_colour": a == d,
                                "full": (t == d // 12 and a == d % 12)}[scheme]
                        got = blk[d][t, :, :, :, s, c]
                        assert np.array_equal(got, noise[k][t, :, :, :, s, c] if keep else 0 * got)


def test_full_dilution_of_a_one_site_noise_is_the_point_propagator():
    """A noise vector that is 1 on the twelve components of one site: its
    twelve spin-colour diluted sources are the point sources there, and the
    estimate sum_a X_a eta_a^dag (Eq. Sfill with N_r = 1) is the column block
    M^{-1}(., y0) of the dense inverse exactly."""
    dims = (4, 2, 2, 4)
    X, Y, Z, T = dims
    U = inputs.make_links(dims, 0.25, 61)
    F = oracle.field_strength(U)
    M = dense_M(U, F, 0.12, 1.0, -1.0, dims)
    S = np.linalg.inv(M)
    y0 = (2, 1, 0, 1)  # t, z, y, x
    noise = np.zeros((1, T, Z, Y, X, 4, 3), dtype=np.complex128)
    noise[(0,) + y0] = 1.0
    src = oracle.dilute(noise, "spin_colour")
    sol = np.array([np.linalg.solve(M, src[a].reshape(-1)) for a in range(12)])
    est = np.einsum("ai,ab->ib", sol, np.conj(src.reshape(12, -1))[:, :])  # (V*12, V*12)
    site = ((y0[0] * Z + y0[1]) * Y + y0[2]) * X + y0[3]
    cols = slice(12 * site, 12 * site + 12)
    assert np.allclose(est[:, cols], S[:, cols], rtol=0, atol=1e-12)
