"""Seeded synthetic inputs for the clover solve of noise sources.

This module is the only code shared by the CUDA path's tests/bench and the
FP64 oracle: it draws random numbers and shapes them into gauge links and
noise sources. It holds none of the solver's arithmetic (no hopping term,
no clover term, no Krylov step).

Array conventions (the host layout of the C ABI):

* gauge field ``U``: complex128, shape ``(T, Z, Y, X, 4, 3, 3)``; index
  ``[t, z, y, x, mu, a, b]`` is row ``a``, column ``b`` of the link
  ``U_mu(x)`` leaving site ``x`` in direction ``mu`` (0=x, 1=y, 2=z, 3=t).
* spinor field: complex128, shape ``(n, T, Z, Y, X, 4, 3)``; index
  ``[k, t, z, y, x, s, c]`` is source ``k``, spin ``s``, colour ``c``.

The paper's ensembles (quenched, beta = 5.96; Sec. "Correlation function")
are not available, so smooth random SU(3) fields stand in for them:
``U = exp(i eps H)`` with ``H`` a Gaussian traceless Hermitian matrix,
re-unitarised to SU(3). The paper's sources are Z2 noise (Sec. "Stochastic
propagators", Eq. Sfill); the workloads here use Z4 noise {1, i, -1, -i},
which has the same unit modulus and E[eta eta^*] = 1.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "WORKLOADS",
    "make_gaussian_spinors",
    "make_links",
    "make_z4",
    "reunitarize",
    "workload",
]


def _traceless_hermitian(g: np.ndarray) -> np.ndarray:
    """H = (A + A^dag)/2 - tr(A + A^dag)/6 * 1 with A_ab = g1 + i g2."""
    a = g[..., 0] + 1j * g[..., 1]
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1)
    h = h - (tr / 3.0)[..., None, None] * np.eye(3)
    return h


def reunitarize(u: np.ndarray) -> np.ndarray:
    """Project 3x3 matrices onto SU(3) by Gram-Schmidt on rows 0 and 1.

    Row 2 is rebuilt as conj(row0 x row1), which fixes det = 1.
    """
    u = np.array(u, dtype=np.complex128, copy=True)
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def make_links(dims, eps: float, seed: int) -> np.ndarray:
    """Random SU(3) gauge field U_mu(x) = exp(i eps H_mu(x)), reunitarised.

    ``dims`` = (X, Y, Z, T). Draw order: one PCG64 stream from ``seed``;
    Gaussian pairs in C order over (t, z, y, x, mu, a, b, re/im).
    """
    X, Y, Z, T = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((T, Z, Y, X, 4, 3, 3, 2))
    h = _traceless_hermitian(g)
    w, v = np.linalg.eigh(h)
    u = (v * np.exp(1j * eps * w)[..., None, :]) @ np.conj(np.swapaxes(v, -1, -2))
    return reunitarize(u)


def make_z4(dims, n: int, seed: int, tslices=None) -> np.ndarray:
    """``n`` Z4 noise sources; source k draws from ``default_rng(seed + k)``.

    Every entry is i^m with m uniform in {0, 1, 2, 3}. With ``tslices``
    (length n) source k is kept only on timeslice ``tslices[k]`` (time
    dilution) and is zero elsewhere.
    """
    X, Y, Z, T = (int(d) for d in dims)
    out = np.empty((n, T, Z, Y, X, 4, 3), dtype=np.complex128)
    phases = np.array([1.0, 1j, -1.0, -1j])
    for k in range(n):
        rng = np.random.default_rng(seed + k)
        out[k] = phases[rng.integers(0, 4, size=(T, Z, Y, X, 4, 3))]
        if tslices is not None:
            keep = np.zeros(T, dtype=bool)
            keep[int(tslices[k]) % T] = True
            out[k, ~keep] = 0.0
    return out


def make_gaussian_spinors(dims, n: int, seed: int) -> np.ndarray:
    """``n`` spinor fields with iid standard normal real and imaginary parts;
    field k draws from ``default_rng(seed + k)`` (real parts, then imaginary
    parts, C order)."""
    X, Y, Z, T = (int(d) for d in dims)
    out = np.empty((n, T, Z, Y, X, 4, 3), dtype=np.complex128)
    for k in range(n):
        rng = np.random.default_rng(seed + k)
        re = rng.standard_normal((T, Z, Y, X, 4, 3))
        out[k] = re + 1j * rng.standard_normal((T, Z, Y, X, 4, 3))
    return out


# Synthetic workloads: lattice, link smoothness, clover coefficient, kappa,
# number of Z4 sources, dilution, seeds (links 1000+i, sources 2000+i).
WORKLOADS = {
    "4x4x4x8": dict(dims=(4, 4, 4, 8), eps=0.25, csw=1.0, kappa=0.115,
                    n_rhs=4, diluted=False, link_seed=1001, src_seed=2001),
    "16x16x16x32": dict(dims=(16, 16, 16, 32), eps=0.25, csw=1.0, kappa=0.120,
                        n_rhs=16, diluted=False, link_seed=1002, src_seed=2002),
    "24x24x24x48": dict(dims=(24, 24, 24, 48), eps=0.25, csw=1.0, kappa=0.122,
                        n_rhs=64, diluted=True, link_seed=1003, src_seed=2003),
    "32x32x32x64": dict(dims=(32, 32, 32, 64), eps=0.25, csw=1.0, kappa=0.122,
                        n_rhs=24, diluted=False, link_seed=1004, src_seed=2004),
}


def workload(name: str, n_rhs: int | None = None):
    """Return (spec, U, eta) for a named workload; ``n_rhs`` may cut sources."""
    spec = dict(WORKLOADS[name])
    n = spec["n_rhs"] if n_rhs is None else int(n_rhs)
    U = make_links(spec["dims"], spec["eps"], spec["link_seed"])
    T = spec["dims"][3]
    ts = [k % T for k in range(n)] if spec["diluted"] else None
    eta = make_z4(spec["dims"], n, spec["src_seed"], ts)
    return spec, U, eta
