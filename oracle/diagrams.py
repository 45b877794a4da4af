"""Oracle: the four diagram contractions of the two-pion correlation function.

TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
CPU-baseline / reference leg may import this module. It shares no code with
the CUDA path and imports nothing from it.

What it computes (zero momentum, one gauge configuration). With S the quark
propagator (S(w; w') is the 12 x 12 spin-colour block of M^{-1} from source
site w' to sink site w), the origin 0 = (0, 0), x and y, z running over the
sites of timeslices 0 and t:

  P(t)   = sum_y tr[S(t,y;0,0) S(t,y;0,0)^+]               (point source)
  Q0(t)  = sum_x sum_z tr[S(t,z;0,x) S(t,z;0,x)^+]         (all-to-all)
  Qtt(t) = sum_y sum_z tr[S(t,z;t,y) S(t,z;t,y)^+]         (all-to-all)
  C0(t)  = P(t) Q0(t)            Diagram 0 (Sec. "Stochastic propagators")
  C1(t)  = Qtt(t) P(0)           Diagram 1 (Sec. "Correlation function")
  C2(t)  = sum_{x,y,z} tr[S^+(0,x;0,0) S(0,x;t,z) S^+(t,y;t,z) S(t,y;0,0)]
                                 Diagram 2 (same section)
  C3(t)  = conj C2(t)            Diagram 3 ("the complex conjugate of Diagram 2")

The dagger acts on spin-colour only (the paper has already used
gamma5-hermiticity to exchange the site indices). Sums over x, y, z with
unit phases are the zero-momentum projections of the paper's Fourier
transforms; each diagram's sum factorises into the factors above.

Reading of Diagram 0. Its printed second trace is tr[S(t,z;0,0) S^+(t,x;0,0)],
while the text says that its bottom contractions join a source at (0,x) to a
sink at (t,z) and that the diagram needs the all-to-all propagator
S(t,z;0,x). This module takes the text: the second factor is
tr[S(t,z;0,x) S^+(t,z;0,x)], whose sum over x and z is Table Lcomp's
"sum_x sum_z tr S_s S_s^+", and the first is its "sum_y tr S_p S_p^+".

Vacuum subtraction. C0 and C1 subtract products of ensemble averages
(<P><Q0> and <Qtt><P(0)>: Diagram 0's second line, Diagram 1's factors). Those
need many configurations, so the per-configuration functions return the raw
products and `ensemble` forms <C0> - <P><Q0>, <(Qtt - <Qtt>)(P(0) - <P(0)>)>,
<C2>, <C3> and the sum C = C0 + C1 - C2 - C3 of the paper's last equation.

Stochastic estimates. Replacing S by the filled stochastic propagators of
Eq. Sfill, S(w; w') ~ (1/N) sum_i X_i(w) eta_i(w')^+, with set A for every S
and set B for every S^+ (the paper's two independent sets; B = A is its
one-set option), gives unbiased estimates of every diagram when A and B are
independent. The point propagator S(.;0,0) is exact: twelve solutions of
unit sources at the origin.

Pins (tests/test_oracle_diagrams.py, mutations in tests/test_oracle_mutations.py):
explicit site loops of every formula on a 2^4 lattice; the gamma5-hermiticity
form of C2 from other blocks of the same inverse; a complete basis of scaled
unit sources for which the stochastic route is exact; unbiasedness within 5
sigma over independent Z4 sets; the sample-covariance form of the ensemble
subtraction.
"""

from __future__ import annotations

import numpy as np

from .dirac import GAMMA5

# quantities of one configuration, in output order
NAMES = ("P", "Q0", "Qtt", "C0", "C1", "C2", "C3")


def point_propagator(Xp: np.ndarray) -> np.ndarray:
    """S(t,y;0,0) from the twelve solutions Xp[a] = M^{-1} e_a (e_a: unit
    source on spin-colour a = 3*spin + colour at the origin):
    Sp[t, z, y, x, alpha, a] with alpha the sink's spin-colour index."""
    T, Z, Y, X = Xp.shape[1:5]
    return np.moveaxis(Xp.reshape(12, T, Z, Y, X, 12), 0, -1)


def blocks_from_inverse(Minv: np.ndarray, dims) -> np.ndarray:
    """The 12 x 12 blocks of a dense M^{-1} (rows and columns in the
    lexicographic spinor order, site i = x + X(y + Y(z + Z t)) times 12):
    S[t, z, y, x, t', z', y', x', alpha, beta] = S((t,z,y,x); (t',z',y',x'))."""
    X, Y, Z, T = dims
    S = Minv.reshape(T, Z, Y, X, 12, T, Z, Y, X, 12)
    return np.moveaxis(S, 4, 8)


def _per_config(Sp, SA, SB, T):
    """The seven quantities from the point propagator Sp[t,z,y,x,alpha,a]
    and two all-to-all propagators given as SA[t0] (and SB[t0]) =
    [t, z, y, x (sink), z', y', x' (source on timeslice t0), alpha, beta]."""
    out = np.zeros((7, T), dtype=np.complex128)
    V3 = Sp.shape[1] * Sp.shape[2] * Sp.shape[3]
    sp = Sp.reshape(T, V3, 12, 12)
    for t in range(T):
        out[0, t] = np.sum(np.abs(sp[t]) ** 2)
        A0, B0 = SA[0][t].reshape(V3, V3, 12, 12), SB[0][t].reshape(V3, V3, 12, 12)
        out[1, t] = np.einsum("zxab,zxab->", A0, np.conj(B0))
        At, Bt = SA[t][t].reshape(V3, V3, 12, 12), SB[t][t].reshape(V3, V3, 12, 12)
        out[2, t] = np.einsum("zyab,zyab->", At, np.conj(Bt))
        # S(0,x;t,z) from set A; S(t,y;t,z)^+ from set B
        Ax = SA[t][0].reshape(V3, V3, 12, 12)  # [x (sink on 0), z (source on t)]
        By = SB[t][t].reshape(V3, V3, 12, 12)  # [y (sink on t), z (source on t)]
        # tr[Sp(0,x)^+ A(x,z) B(y,z)^+ Sp(t,y)]
        out[5, t] = np.einsum("xba,xzbc,yzdc,yda->", np.conj(sp[0]), Ax, np.conj(By), sp[t], optimize=True)
    out[3] = out[0] * out[1]
    out[4] = out[2] * out[0, 0]
    out[6] = np.conj(out[5])
    return out


def diagrams_exact(Minv: np.ndarray, dims) -> np.ndarray:
    """The seven per-configuration quantities (NAMES) from a dense M^{-1};
    complex (7, T)."""
    T = dims[3]
    S = blocks_from_inverse(Minv, dims)
    Sp = S[:, :, :, :, 0, 0, 0, 0]  # [t, z, y, x, alpha, beta]: source at the origin
    Sall = [S[:, :, :, :, t0] for t0 in range(T)]
    return _per_config(Sp, Sall, Sall, T)


def filled_propagator(eta: np.ndarray, X: np.ndarray, t0: int) -> np.ndarray:
    """Eq. Sfill from source timeslice t0, spin-colour merged:
    S[t, z, y, x, z', y', x', alpha, beta] = (1/N) sum_i X_i(t,z,y,x)_alpha
    conj(eta_i(t0,z',y',x')_beta)."""
    n, T, Z, Y, Xd = eta.shape[:5]
    Xm = X.reshape(n, T, Z, Y, Xd, 12)
    em = eta[:, t0].reshape(n, Z, Y, Xd, 12)
    return np.einsum("itzyxa,iwvub->tzyxwvuab", Xm, np.conj(em)) / n


def diagrams_stochastic(Xp, etaA, XA, etaB=None, XB=None) -> np.ndarray:
    """The seven quantities with every all-to-all S filled from set A and
    every S^+ from set B (B = A when etaB, XB are None); the point
    propagator from the twelve solutions Xp. Complex (7, T)."""
    T = etaA.shape[1]
    SA = [filled_propagator(etaA, XA, t0) for t0 in range(T)]
    SB = SA if etaB is None else [filled_propagator(etaB, XB, t0) for t0 in range(T)]
    return _per_config(point_propagator(Xp), SA, SB, T)


def ensemble(per_cfg: np.ndarray) -> np.ndarray:
    """Vacuum-subtracted averages over configurations from per-configuration
    records (n_cfg, 7, T): rows C0 - <P><Q0>, <(Qtt - <Qtt>)(P(0) - <P(0)>)>,
    <C2>, <C3> and C = C0 + C1 - C2 - C3; complex (5, T)."""
    m = np.mean(per_cfg, axis=0)
    P, Q0, Qtt, C0, C1, C2, C3 = m
    c0 = C0 - P * Q0
    c1 = C1 - Qtt * P[0]
    return np.array([c0, c1, C2, C3, c0 + c1 - C2 - C3])


def c2_gamma5_form(Minv: np.ndarray, dims, t: int) -> complex:
    """Diagram 2 at sink time t written with gamma5-hermiticity,
    S(w;w')^+ = g5 S(w';w) g5, from the other blocks of the same inverse:
    sum tr[g5 S(0,0;0,x) g5 S(0,x;t,z) g5 S(t,z;t,y) g5 S(t,y;0,0)]."""
    X, Y, Z, T = dims
    V3 = X * Y * Z
    S = blocks_from_inverse(Minv, dims).reshape(T, V3, T, V3, 12, 12)
    g = np.kron(GAMMA5, np.eye(3))
    tot = 0j
    for x in range(V3):
        for y in range(V3):
            for z in range(V3):
                m = g @ S[0, 0, 0, x] @ g @ S[0, x, t, z] @ g @ S[t, z, t, y] @ g @ S[t, y, 0, 0]
                tot += np.trace(m)
    return tot
