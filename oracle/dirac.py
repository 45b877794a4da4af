"""Plain FP64 CPU oracle: clover-Wilson operator, BiCGStab, pion correlator.

TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
CPU-baseline / reference leg may import this module. The library's product
path never calls it, and it shares no code with the CUDA kernels.

What it computes. The paper needs the quark propagator S = M^{-1}, the
inverse of the lattice fermion matrix in the background gauge field
(Sec. "Stochastic propagators", the definition above Eq. Sfill), applied to
random sources eta_i to give solution vectors X_i = M^{-1} eta_i (Eq. Sfill).
The fermions are clover fermions with the tree-level coefficient c_SW = 1.0
(Sec. "Correlation function"). The paper never writes M out; this module
takes the standard kappa-normalised Sheikholeslami-Wohlert operator

    M = A - kappa D,
    D psi(x) = sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu)
                        + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ],
    A(x) = 1 + i kappa c_sw sum_{mu<nu} sigma_mu_nu (x) Fhat_mu_nu(x),
    sigma_mu_nu = (i/2)[g_mu, g_nu],
    Fhat_mu_nu = (Q_mu_nu - Q_mu_nu^dag)/8 with its trace removed,

where Q_mu_nu(x) is the sum of the four plaquette leaves in the mu-nu plane
that start and end at x, and g_mu are the DeGrand-Rossi gamma matrices.
The fermion field is periodic in space and carries the factor ``t_bc`` on the
hop across the time boundary (-1: antiperiodic).

Array conventions: gauge field ``U`` has shape (T, Z, Y, X, 4, 3, 3)
([.., mu, row, col]); a spinor field has shape (..., T, Z, Y, X, 4, 3)
([.., spin, colour]) with any number of leading batch axes. Direction
mu = 0, 1, 2, 3 is x, y, z, t, stored on array axes -3, -4, -5, -6 of a
spinor (axes 3, 2, 1, 0 of the lattice block).

Every function is written for clarity, not speed: whole-lattice numpy
shifts, per-site 3x3 and 4x4 products, no even-odd blocking unless the
function is the even-odd formula itself.

Pins (tests/test_oracle_pins.py; tests/test_oracle_mutations.py plants
mistakes and checks that a pin catches each): free-field closed form of M
and M^{-1} with antiperiodic time momenta, gamma5-hermiticity, gauge
covariance, a constant abelian background (clover normalisation 1/8, leaf
orientation, mu<nu bookkeeping), dense LU on tiny lattices (BiCGStab and the
even-odd formulas), brute-force loops and the exact expectation value for
the pion contraction and for the stochastic-operator contraction O_ij(t)
(with O_ii = 0 for X = eta as a special case); brute-force loops, the
point-source limit and the exact expectation value for the traces of
filled stochastic propagators; completeness, disjoint supports and the
exact point propagator from a one-site noise vector for the dilution. Parity unpinned: the overall sign of the clover term
(+i kappa c_sw) is the Sheikholeslami-Wohlert / Luscher-Sint-Sommer-Weisz
convention and is fixed by that citation only; no invariant above changes
when it flips.
"""

from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# Dirac algebra (DeGrand-Rossi basis)
# ---------------------------------------------------------------------------

_I = 1j
GAMMA = np.array(
    [
        [[0, 0, 0, _I], [0, 0, _I, 0], [0, -_I, 0, 0], [-_I, 0, 0, 0]],  # g_1 (x)
        [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],  # g_2 (y)
        [[0, 0, _I, 0], [0, 0, 0, -_I], [-_I, 0, 0, 0], [0, _I, 0, 0]],  # g_3 (z)
        [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],  # g_4 (t)
    ],
    dtype=np.complex128,
)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
EYE4 = np.eye(4, dtype=np.complex128)

# The six planes mu < nu, in the order used for field-strength arrays.
PLANES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def sigma(mu: int, nu: int) -> np.ndarray:
    """sigma_mu_nu = (i/2) [g_mu, g_nu]."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


def dagger(m: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(m, -1, -2))


# ---------------------------------------------------------------------------
# Lattice shifts
# ---------------------------------------------------------------------------

def _lattice_axis(mu: int, nd_site: int) -> int:
    """Array axis of direction mu for an array whose last nd_site axes are
    per-site (spin/colour) axes, so the lattice block is (T, Z, Y, X)."""
    return -(nd_site + 1 + mu)


def shift(f: np.ndarray, mu: int, step: int, nd_site: int, t_bc: float = 1.0):
    """g(x) = f(x + step * mu_hat) for step = +1 or -1, periodic wrap.

    For mu = 3 (time) the value that wraps across the boundary is multiplied
    by ``t_bc``. ``nd_site`` is the number of trailing per-site axes of f.
    """
    ax = _lattice_axis(mu, nd_site)
    g = np.roll(f, -step, axis=ax)
    if mu == 3 and t_bc != 1.0:
        n = f.shape[ax]
        idx = [slice(None)] * f.ndim
        # step=+1: site t = T-1 reads t = 0;  step=-1: site t = 0 reads t = T-1
        idx[ax] = n - 1 if step == 1 else 0
        g[tuple(idx)] *= t_bc
    return g


def _colour(U_mu: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(U psi)[s, a] = sum_b U[a, b] psi[s, b] at every site."""
    return psi @ np.swapaxes(U_mu, -1, -2)


def _colour_dag(U_mu: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(U^dag psi)[s, a] = sum_b conj(U[b, a]) psi[s, b] at every site."""
    return psi @ np.conj(U_mu)


def _spin(G: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(G psi)[s, c] = sum_s' G[s, s'] psi[s', c] at every site."""
    return G @ psi


# ---------------------------------------------------------------------------
# Wilson hopping term
# ---------------------------------------------------------------------------

def hopping(U: np.ndarray, psi: np.ndarray, t_bc: float = -1.0) -> np.ndarray:
    """D psi(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu)
                        + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu)."""
    out = np.zeros_like(psi)
    for mu in range(4):
        U_mu = U[..., mu, :, :]
        fwd = _colour(U_mu, shift(psi, mu, +1, 2, t_bc))
        out += _spin(EYE4 - GAMMA[mu], fwd)
        bwd = shift(_colour_dag(U_mu, psi), mu, -1, 2, t_bc)
        out += _spin(EYE4 + GAMMA[mu], bwd)
    return out


# ---------------------------------------------------------------------------
# Clover term
# ---------------------------------------------------------------------------

def _link_shift(U_nu: np.ndarray, mu: int, step: int) -> np.ndarray:
    """Gauge links carry no boundary phase: plain periodic shift."""
    return shift(U_nu, mu, step, 2, 1.0)


def plaquette_leaves(U: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """Q_mu_nu(x): sum of the four mu-nu plaquettes that start and end at x,
    all traversed in the same (mu then nu) orientation."""
    Um, Un = U[..., mu, :, :], U[..., nu, :, :]
    sm = lambda A, s: _link_shift(A, mu, s)  # A(x + s mu)
    sn = lambda A, s: _link_shift(A, nu, s)  # A(x + s nu)
    # U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
    l1 = Um @ sm(Un, +1) @ dagger(sn(Um, +1)) @ dagger(Un)
    # U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
    l2 = Un @ dagger(sn(sm(Um, -1), +1)) @ dagger(sm(Un, -1)) @ sm(Um, -1)
    # U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
    l3 = (dagger(sm(Um, -1)) @ dagger(sn(sm(Un, -1), -1))
          @ sn(sm(Um, -1), -1) @ sn(Un, -1))
    # U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag
    l4 = dagger(sn(Un, -1)) @ sn(Um, -1) @ sm(sn(Un, -1), +1) @ dagger(Um)
    return l1 + l2 + l3 + l4


def field_strength(U: np.ndarray) -> np.ndarray:
    """Fhat_mu_nu(x) = (Q - Q^dag)/8 minus its trace/3; shape (..., 6, 3, 3)
    in the plane order of PLANES. Each Fhat is traceless anti-Hermitian."""
    out = []
    for mu, nu in PLANES:
        Q = plaquette_leaves(U, mu, nu)
        F = (Q - dagger(Q)) / 8.0
        tr = np.trace(F, axis1=-2, axis2=-1)
        F = F - (tr / 3.0)[..., None, None] * np.eye(3)
        out.append(F)
    return np.stack(out, axis=-3)


def clover_apply(F: np.ndarray, psi: np.ndarray, kappa: float, csw: float):
    """A psi = psi + i kappa c_sw sum_{mu<nu} (sigma_mu_nu (x) Fhat_mu_nu) psi."""
    out = psi.copy()
    for p, (mu, nu) in enumerate(PLANES):
        term = _colour(F[..., p, :, :], _spin(sigma(mu, nu), psi))
        out += 1j * kappa * csw * term
    return out


def clover_matrices(F: np.ndarray, kappa: float, csw: float) -> np.ndarray:
    """A(x) as an explicit 12x12 matrix per site, index 3*spin + colour."""
    lat = F.shape[:-3]
    A = np.zeros(lat + (4, 3, 4, 3), dtype=np.complex128)
    for p, (mu, nu) in enumerate(PLANES):
        A += np.einsum("st,...ab->...satb", sigma(mu, nu), F[..., p, :, :])
    A = 1j * kappa * csw * A.reshape(lat + (12, 12))
    return A + np.eye(12)


def site_apply(Mx: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a per-site 12x12 matrix field to a spinor field."""
    sh = psi.shape
    v = psi.reshape(sh[:-2] + (12, 1))
    return (Mx @ v).reshape(sh)


# ---------------------------------------------------------------------------
# The fermion matrix and its even-odd (Schur) blocks
# ---------------------------------------------------------------------------

def apply_M(U, F, psi, kappa, csw, t_bc=-1.0):
    """M psi = A psi - kappa D psi on the full lattice."""
    return clover_apply(F, psi, kappa, csw) - kappa * hopping(U, psi, t_bc)


def parity_field(dims) -> np.ndarray:
    """p(x) = (x + y + z + t) mod 2 as an int array of shape (T, Z, Y, X)."""
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y),
                             np.arange(X), indexing="ij")
    return (x + y + z + t) % 2


def restrict(psi: np.ndarray, par: np.ndarray, p: int) -> np.ndarray:
    """Zero psi on sites whose parity is not p."""
    return psi * (par == p)[..., None, None]


def hopping_eo(U, psi, p_out, par, t_bc=-1.0):
    """D_{p,1-p}: hop from sites of parity 1-p onto sites of parity p."""
    return restrict(hopping(U, restrict(psi, par, 1 - p_out), t_bc), par, p_out)


def schur_apply(U, Ainv, x_e, kappa, par, t_bc=-1.0):
    """Mhat x_e = x_e - kappa^2 A_ee^{-1} D_eo A_oo^{-1} D_oe x_e (even sites).

    From M = [[A_ee, -k D_eo], [-k D_oe, A_oo]]: eliminating the odd sites
    gives (A_ee - k^2 D_eo A_oo^{-1} D_oe) x_e = eta_e + k D_eo A_oo^{-1} eta_o,
    left-multiplied here by A_ee^{-1}.
    """
    t_o = site_apply(Ainv, hopping_eo(U, x_e, 1, par, t_bc))
    t_e = site_apply(Ainv, hopping_eo(U, t_o, 0, par, t_bc))
    return restrict(x_e, par, 0) - kappa * kappa * t_e


def schur_source(U, Ainv, eta, kappa, par, t_bc=-1.0):
    """bhat_e = A_ee^{-1} (eta_e + kappa D_eo A_oo^{-1} eta_o)."""
    t_o = site_apply(Ainv, restrict(eta, par, 1))
    b = restrict(eta, par, 0) + kappa * hopping_eo(U, t_o, 0, par, t_bc)
    return site_apply(Ainv, b) * (par == 0)[..., None, None]


def schur_reconstruct(U, Ainv, eta, x_e, kappa, par, t_bc=-1.0):
    """psi = x_e on even sites, A_oo^{-1}(eta_o + kappa D_oe x_e) on odd."""
    b_o = restrict(eta, par, 1) + kappa * hopping_eo(U, x_e, 1, par, t_bc)
    return restrict(x_e, par, 0) + restrict(site_apply(Ainv, b_o), par, 1)


# ---------------------------------------------------------------------------
# BiCGStab (van der Vorst 1992), plain FP64
# ---------------------------------------------------------------------------

def inner(a: np.ndarray, b: np.ndarray) -> complex:
    """<a, b> = sum conj(a) b."""
    return complex(np.vdot(a, b))


def bicgstab(apply, b, tol=1e-12, maxiter=10000, x0=None):
    """Solve apply(x) = b to relative residual ||b - apply(x)|| / ||b|| <= tol.

    Returns (x, iterations, true relative residual). The loop stops on the
    recursively updated residual and confirms with the recomputed one.
    """
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, copy=True)
    r = b - apply(x)
    rhat = r.copy()
    rho = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    it = 0
    while it < maxiter:
        if np.linalg.norm(r) <= tol * bnorm:
            true_r = np.linalg.norm(b - apply(x)) / bnorm
            if true_r <= tol:
                return x, it, true_r
            r = b - apply(x)  # restart from the true residual
            rhat = r.copy()
            rho = alpha = omega = 1.0 + 0j
            v[...] = 0
            p[...] = 0
        rho_new = inner(rhat, r)
        beta = (rho_new / rho) * (alpha / omega)
        rho = rho_new
        p = r + beta * (p - omega * v)
        v = apply(p)
        alpha = rho / inner(rhat, v)
        s = r - alpha * v
        t = apply(s)
        omega = inner(t, s) / inner(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        it += 1
    true_r = np.linalg.norm(b - apply(x)) / bnorm
    return x, it, true_r


def solve(U, eta, kappa, csw, t_bc=-1.0, tol=1e-12, maxiter=10000, F=None):
    """psi = M^{-1} eta for one source, unpreconditioned BiCGStab."""
    if F is None:
        F = field_strength(U)
    return bicgstab(lambda v: apply_M(U, F, v, kappa, csw, t_bc), eta, tol, maxiter)


# ---------------------------------------------------------------------------
# Pion correlator epilogue
# ---------------------------------------------------------------------------

def pion_correlator(psi: np.ndarray, t_src: int = 0) -> np.ndarray:
    """C(dt) = sum over sites on timeslice (t_src + dt) mod T of
    sum_{s,c} |psi(x)|^2 for one solution vector psi = X_i.

    With psi = M^{-1} eta this is the stochastic estimate of
    sum_{x in t} sum_y tr[S(x, y) S(x, y)^dag] (the zero-momentum pion
    correlator via gamma5-hermiticity; Sec. "Stochastic propagators",
    the O_ij(t) rearrangement, and the sum_y tr S_p S_p^dag timing row of
    Table Lcomp). No 1/N_r or volume factor.
    """
    T = psi.shape[0]
    per_t = np.sum(np.abs(psi) ** 2, axis=(1, 2, 3, 4, 5))
    return np.array([per_t[(t_src + dt) % T] for dt in range(T)])


def stochastic_operator(eta: np.ndarray, X: np.ndarray) -> np.ndarray:
    """O[t, i, j] = sum over the sites y of timeslice t of
    eta_i(y)^dag gamma5 X_j(y), spin and colour contracted (Eq. stoop:
    the operators of the L^3 rearrangement of the pion correlator in
    Sec. "Stochastic propagators").

    eta, X: (n, T, Z, Y, X, 4, 3) sources and solution vectors; returns a
    complex (T, n, n) array.
    """
    g5X = _spin_all(GAMMA5, X)
    return np.einsum("itzyxsc,jtzyxsc->tij", np.conj(eta), g5X)


def _spin_all(G: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(G psi)[..., s, c] = sum_s' G[s, s'] psi[..., s', c]."""
    return np.einsum("ab,...bc->...ac", G, psi)


def stochastic_operator_correlator(O: np.ndarray) -> np.ndarray:
    """C(dt) = 1/(N_r^2 T) sum_t0 sum_ij O_ij((t0 + dt) mod T) O_ji(t0): the
    correlator contraction of the operators (Sec. "Stochastic propagators",
    the equation after Eq. stoop), averaged over the source timeslice t0
    (every timeslice carries noise for undiluted sources). Complex (T,)."""
    T, n, _ = O.shape
    C = np.zeros(T, dtype=np.complex128)
    for dt in range(T):
        for t0 in range(T):
            C[dt] += np.sum(O[(t0 + dt) % T] * O[t0].T)
    return C / (n * n * T)


def dilute(noise: np.ndarray, scheme: str) -> np.ndarray:
    """Time, spin-colour or full (time-spin-colour) dilution of noise vectors
    (Sec. "Stochastic propagators"): for each noise vector, one source per
    timeslice t ("time"), per spin-colour component a = 3*spin + colour
    ("spin_colour") or per pair (t, a) in the order 12*t + a ("full"), equal
    to the noise on that part and zero elsewhere. noise: (n, T, Z, Y, X, 4, 3);
    returns (n * D, T, Z, Y, X, 4, 3)."""
    n, T = noise.shape[0], noise.shape[1]
    parts = []
    if scheme == "time":
        parts = [(t, None) for t in range(T)]
    elif scheme == "spin_colour":
        parts = [(None, a) for a in range(12)]
    elif scheme == "full":
        parts = [(t, a) for t in range(T) for a in range(12)]
    else:
        raise ValueError(scheme)
    out = []
    for k in range(n):
        for t, a in parts:
            mask = np.zeros(noise.shape[1:], dtype=bool)
            tt = slice(None) if t is None else t
            if a is None:
                mask[tt] = True
            else:
                mask[tt, :, :, :, a // 3, a % 3] = True
            out.append(np.where(mask, noise[k], 0.0))
    return np.array(out)


def stochastic_propagator(eta: np.ndarray, X: np.ndarray, t0: int) -> np.ndarray:
    """The filled stochastic propagator of Eq. Sfill from the source
    timeslice t0 to every sink site:
        S(t, z; t0, x)_{ab} = (1/N_r) sum_i X_i(t, z)_a eta_i(t0, x)_b^*,
    a = (spin, colour) at the sink, b at the source (Sec. "Stochastic
    propagators"). Returns a complex array indexed
    [t, z, y, x (sink), z', y', x' (source on t0), s, c, s', c']."""
    n = eta.shape[0]
    return np.einsum("itzyxsc,iwvuSC->tzyxwvuscSC", X, np.conj(eta[:, t0])) / n


def propagator_trace(SA: np.ndarray, SB: np.ndarray) -> np.ndarray:
    """sum over every source site x and sink site z of the sink timeslice t
    of tr[SA(t, z; x) SB(t, z; x)^dag], the spin-colour trace of Table Lcomp's
    "sum_x sum_z tr S_s S_s^dag"; complex (T,)."""
    return np.einsum("tzyxwvuscSC,tzyxwvuscSC->t", SA, np.conj(SB))


def stochastic_propagator_trace(etaA, XA, etaB=None, XB=None) -> np.ndarray:
    """C[t0, t] = propagator_trace of the propagators filled from source
    timeslice t0 with set A (S) and set B (S^dag); one set (B = A) when
    etaB, XB are None, as in the paper's correlated option. Fills S for
    every t0 (the L^7 route the paper measured); complex (T, T)."""
    T = etaA.shape[1]
    C = np.zeros((T, T), dtype=np.complex128)
    for t0 in range(T):
        SA = stochastic_propagator(etaA, XA, t0)
        SB = SA if etaB is None else stochastic_propagator(etaB, XB, t0)
        C[t0] = propagator_trace(SA, SB)
    return C
