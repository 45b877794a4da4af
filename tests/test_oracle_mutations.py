"""Plant plausible mistakes in the oracle (CPU only) and check that the pins
in test_oracle_pins.py catch every one of them.

Each mutation replaces one oracle function by a subtly wrong copy for the
duration of one check; the check must then fail.
"""

import numpy as np
import pytest

from oracle import dirac
import test_oracle_pins as pins


def _hopping_variant(fwd_proj=-1, bwd_proj=+1, dag=True, fwd_site=0, bc=True):
    def hop(U, psi, t_bc=-1.0):
        tb = t_bc if bc else 1.0
        out = np.zeros_like(psi)
        for mu in range(4):
            U_mu = U[..., mu, :, :]
            if fwd_site:
                U_mu_f = dirac.shift(U_mu, mu, fwd_site, 2, 1.0)
            else:
                U_mu_f = U_mu
            fwd = dirac._colour(U_mu_f, dirac.shift(psi, mu, +1, 2, tb))
            out += dirac._spin(dirac.EYE4 + fwd_proj * dirac.GAMMA[mu], fwd)
            cd = dirac._colour_dag if dag else dirac._colour
            bwd = dirac.shift(cd(U_mu, psi), mu, -1, 2, tb)
            out += dirac._spin(dirac.EYE4 + bwd_proj * dirac.GAMMA[mu], bwd)
        return out
    return hop


def _leaves_variant(kind):
    orig = dirac.plaquette_leaves

    def leaves(U, mu, nu):
        Q = orig(U, mu, nu)
        if kind == "reverse_one_leaf":
            Um, Un = U[..., mu, :, :], U[..., nu, :, :]
            sm = lambda A, s: dirac._link_shift(A, mu, s)
            sn = lambda A, s: dirac._link_shift(A, nu, s)
            l1 = Um @ sm(Un, +1) @ dirac.dagger(sn(Um, +1)) @ dirac.dagger(Un)
            return Q - l1 + dirac.dagger(l1)
        if kind == "three_leaves":
            Um, Un = U[..., mu, :, :], U[..., nu, :, :]
            sm = lambda A, s: dirac._link_shift(A, mu, s)
            sn = lambda A, s: dirac._link_shift(A, nu, s)
            l1 = Um @ sm(Un, +1) @ dirac.dagger(sn(Um, +1)) @ dirac.dagger(Un)
            return Q - l1
        if kind == "double":
            return 2 * Q
        raise ValueError(kind)
    return leaves


def _no_trace_removal(U):
    out = []
    for mu, nu in dirac.PLANES:
        Q = dirac.plaquette_leaves(U, mu, nu)
        out.append((Q - dirac.dagger(Q)) / 8.0)
    return np.stack(out, axis=-3)


def _bad_bicgstab(apply, b, tol=1e-12, maxiter=400, x0=None):
    # beta without the alpha/omega factor
    x = np.zeros_like(b)
    r = b - apply(x)
    rhat = r.copy()
    rho = 1.0
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    omega = 1.0
    for it in range(maxiter):
        rho_new = dirac.inner(rhat, r)
        beta = rho_new / rho
        rho = rho_new
        p = r + beta * (p - omega * v)
        v = apply(p)
        alpha = rho / dirac.inner(rhat, v)
        s = r - alpha * v
        t = apply(s)
        omega = dirac.inner(t, s) / dirac.inner(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
    return x, maxiter, np.linalg.norm(b - apply(x)) / np.linalg.norm(b)


def _pion_off_by_one(psi, t_src=0):
    T = psi.shape[0]
    per_t = np.sum(np.abs(psi) ** 2, axis=(1, 2, 3, 4, 5))
    return np.array([per_t[(t_src + dt + 1) % T] for dt in range(T)])


def _run_pins(names):
    """Run the named pins; return True if every one passed."""
    U = pins.unit_links  # noqa: F841  (keeps the module imported)
    dims = (4, 4, 4, 6)
    from paper_1405_4524_gb300 import inputs
    Ur = inputs.make_links(dims, 0.8, 77)
    rough = (dims, Ur, dirac.field_strength(Ur))
    ok = True
    for name in names:
        fn = getattr(pins, name)
        try:
            if name in ("test_gamma5_hermiticity", "test_gauge_covariance",
                        "test_clover_structure"):
                fn(rough)
            elif name == "test_free_field_plane_waves":
                fn(-1.0)
            elif name == "test_constant_abelian_background":
                fn(0, 2, 1)
                fn(3, 1, 1)
            elif name == "test_dense_lu_vs_bicgstab":
                fn((4, 2, 2, 4))
            else:
                fn()
        except AssertionError:
            ok = False
        except (FloatingPointError, ZeroDivisionError, np.linalg.LinAlgError):
            ok = False
    return ok


ALL_OPERATOR_PINS = [
    "test_free_field_plane_waves",
    "test_free_field_propagator_closed_form",
    "test_gamma5_hermiticity",
    "test_gauge_covariance",
    "test_clover_structure",
    "test_constant_abelian_background",
    "test_dense_lu_vs_bicgstab",
    "test_schur_formulas_vs_dense",
]

MUTATIONS = {
    "backward projector sign": ("hopping", _hopping_variant(bwd_proj=-1)),
    "forward projector sign": ("hopping", _hopping_variant(fwd_proj=+1)),
    "both projector signs": ("hopping", _hopping_variant(fwd_proj=+1, bwd_proj=-1)),
    "backward link not daggered": ("hopping", _hopping_variant(dag=False)),
    "forward link at x+mu": ("hopping", _hopping_variant(fwd_site=+1)),
    "no time boundary sign": ("hopping", _hopping_variant(bc=False)),
    "one clover leaf reversed": ("plaquette_leaves", _leaves_variant("reverse_one_leaf")),
    "three clover leaves": ("plaquette_leaves", _leaves_variant("three_leaves")),
    "clover normalisation 1/4": ("plaquette_leaves", _leaves_variant("double")),
    "trace not removed": ("field_strength", _no_trace_removal),
}


def test_unmutated_oracle_passes_the_pins():
    assert _run_pins(ALL_OPERATOR_PINS)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_operator_mutation_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(dirac, attr, fn)
    with np.errstate(all="ignore"):
        assert not _run_pins(ALL_OPERATOR_PINS), f"mutation not caught: {name}"


def test_bicgstab_mutation_is_caught(monkeypatch):
    monkeypatch.setattr(dirac, "bicgstab", _bad_bicgstab)
    with np.errstate(all="ignore"):
        assert not _run_pins(["test_bicgstab_on_a_random_matrix",
                              "test_dense_lu_vs_bicgstab"])


def test_pion_mutation_is_caught(monkeypatch):
    monkeypatch.setattr(dirac, "pion_correlator", _pion_off_by_one)
    import oracle
    monkeypatch.setattr(oracle, "pion_correlator", _pion_off_by_one)
    assert not _run_pins(["test_pion_correlator_brute_force"])


def _stoch_op_no_gamma5(eta, X):
    return np.einsum("itzyxsc,jtzyxsc->tij", np.conj(eta), X)


def _stoch_op_no_conj(eta, X):
    return np.einsum("itzyxsc,jtzyxsc->tij", eta, dirac._spin_all(dirac.GAMMA5, X))


def _stoch_corr_same_t(O):
    T, n, _ = O.shape
    C = np.zeros(T, dtype=np.complex128)
    for dt in range(T):
        for t0 in range(T):
            C[dt] += np.sum(O[(t0 + dt) % T] * O[t0])  # O_ij O_ij instead of O_ij O_ji
    return C / (n * n * T)


STOCH_PINS = ["test_stochastic_operator_brute_force", "test_stochastic_operator_of_the_noise_itself",
              "test_stochastic_operator_estimate_matches_exact"]


@pytest.mark.parametrize("kind", ["no_gamma5", "transposed", "no_conj", "corr_same_t"])
def test_stochastic_operator_mutation_is_caught(kind, monkeypatch):
    import oracle

    orig = dirac.stochastic_operator
    attr, fn = {"no_gamma5": ("stochastic_operator", _stoch_op_no_gamma5),
                "transposed": ("stochastic_operator", lambda e, x: np.transpose(orig(e, x), (0, 2, 1))),
                "no_conj": ("stochastic_operator", _stoch_op_no_conj),
                "corr_same_t": ("stochastic_operator_correlator", _stoch_corr_same_t)}[kind]
    monkeypatch.setattr(dirac, attr, fn)
    monkeypatch.setattr(oracle, attr, fn)
    assert not _run_pins(STOCH_PINS), f"mutation not caught: {kind}"


def _fill_no_conj(eta, X, t0):
    n = eta.shape[0]
    return np.einsum("itzyxsc,iwvuSC->tzyxwvuscSC", X, eta[:, t0]) / n


def _fill_no_norm(eta, X, t0):
    return np.einsum("itzyxsc,iwvuSC->tzyxwvuscSC", X, np.conj(eta[:, t0]))


def _trace_no_dagger(SA, SB):
    return np.einsum("tzyxwvuscSC,tzyxwvuscSC->t", SA, SB)


def _trace_transposed(SA, SB):
    return np.einsum("tzyxwvuscSC,tzyxwvuSCsc->t", SA, np.conj(SB))


FILL_PINS = ["test_propagator_trace_brute_force", "test_propagator_trace_point_source_limit",
             "test_propagator_trace_estimate_matches_exact"]


@pytest.mark.parametrize("kind", ["no_conj", "no_norm", "no_dagger", "transposed"])
def test_propagator_trace_mutation_is_caught(kind, monkeypatch):
    import oracle

    attr, fn = {"no_conj": ("stochastic_propagator", _fill_no_conj),
                "no_norm": ("stochastic_propagator", _fill_no_norm),
                "no_dagger": ("propagator_trace", _trace_no_dagger),
                "transposed": ("propagator_trace", _trace_transposed)}[kind]
    monkeypatch.setattr(dirac, attr, fn)
    monkeypatch.setattr(oracle, attr, fn)
    assert not _run_pins(FILL_PINS), f"mutation not caught: {kind}"


def _dilute_component_major(noise, scheme):
    """full dilution enumerated component-major (d = T*a + t) instead of 12*t + a"""
    out = _orig_dilute(noise, scheme)
    if scheme != "full":
        return out
    n, T = noise.shape[0], noise.shape[1]
    idx = [12 * t + a for a in range(12) for t in range(T)]
    return np.concatenate([out[k * 12 * T:(k + 1) * 12 * T][idx] for k in range(n)])


def _dilute_shifted_time(noise, scheme):
    """time index off by one"""
    out = _orig_dilute(noise, scheme)
    if scheme != "time":
        return out
    n, T = noise.shape[0], noise.shape[1]
    return np.concatenate([np.roll(out[k * T:(k + 1) * T], 1, axis=0) for k in range(n)])


_orig_dilute = dirac.dilute
DILUTION_PINS = ["test_dilution_completeness_and_supports"]


@pytest.mark.parametrize("fn", [_dilute_component_major, _dilute_shifted_time])
def test_dilution_mutation_is_caught(fn, monkeypatch):
    import oracle

    monkeypatch.setattr(dirac, "dilute", fn)
    monkeypatch.setattr(oracle, "dilute", fn)
    caught = False
    for scheme, D in [("time", 4), ("spin_colour", 12), ("full", 48)]:
        try:
            pins.test_dilution_completeness_and_supports(scheme, D)
        except AssertionError:
            caught = True
    assert caught


# ---------------------------------------------------------------------------
# diagram contractions (oracle/diagrams.py)
# ---------------------------------------------------------------------------

def _per_config_variant(kind):
    from oracle import diagrams as dg

    def per_config(Sp, SA, SB, T):
        out = np.zeros((7, T), dtype=np.complex128)
        V3 = Sp.shape[1] * Sp.shape[2] * Sp.shape[3]
        sp = Sp.reshape(T, V3, 12, 12)
        for t in range(T):
            out[0, t] = np.sum(np.abs(sp[t]) ** 2)
            t0 = t if kind == "q0_source_on_t" else 0
            A0, B0 = SA[t0][t].reshape(V3, V3, 12, 12), SB[t0][t].reshape(V3, V3, 12, 12)
            out[1, t] = np.einsum("zxab,zxab->", A0, np.conj(B0))
            At, Bt = SA[t][t].reshape(V3, V3, 12, 12), SB[t][t].reshape(V3, V3, 12, 12)
            out[2, t] = np.einsum("zyab,zyab->", At, np.conj(Bt))
            Ax = SA[t][t if kind == "x_on_t" else 0].reshape(V3, V3, 12, 12)
            By = SB[t][t].reshape(V3, V3, 12, 12)
            if kind == "no_dagger_on_B":
                out[5, t] = np.einsum("xba,xzbc,ycd,yda->", np.conj(sp[0]), Ax, By.sum(axis=1), sp[t], optimize=True)
            elif kind == "point_transposed":
                out[5, t] = np.einsum("xab,xzbc,yzdc,yda->", sp[0], Ax, np.conj(By), sp[t], optimize=True)
            else:
                out[5, t] = np.einsum("xba,xzbc,yzdc,yda->", np.conj(sp[0]), Ax, np.conj(By), sp[t], optimize=True)
        out[3] = out[0] * out[1]
        out[4] = out[2] * (out[0] if kind == "c1_with_P_t" else out[0, 0])
        out[6] = np.conj(out[5])
        return out
    return per_config


def _filled_variant(kind):
    def fill(eta, X, t0):
        n, T, Z, Y, Xd = eta.shape[:5]
        Xm = X.reshape(n, T, Z, Y, Xd, 12)
        em = eta[:, t0].reshape(n, Z, Y, Xd, 12)
        e = em if kind == "no_conj" else np.conj(em)
        out = np.einsum("itzyxa,iwvub->tzyxwvuab", Xm, e)
        return out if kind == "no_norm" else out / n
    return fill


def _point_transposed(Xp):
    T, Z, Y, X = Xp.shape[1:5]
    return np.moveaxis(Xp.reshape(12, T, Z, Y, X, 12), 0, -2)


def _ensemble_P_t(per_cfg):
    m = np.mean(per_cfg, axis=0)
    P, Q0, Qtt, C0, C1, C2, C3 = m
    c0, c1 = C0 - P * Q0, C1 - Qtt * P
    return np.array([c0, c1, C2, C3, c0 + c1 - C2 - C3])


def _run_diagram_pins():
    import test_oracle_diagrams as pd

    tiny = pd.setup((2, 2, 2, 2), 61)
    small = pd.setup((4, 2, 2, 4), 62)
    tiny, small = ((2, 2, 2, 2), tiny[1]), ((4, 2, 2, 4), small[1])
    checks = [lambda: pd.test_exact_diagrams_site_loops(tiny),
              lambda: pd.test_diagram2_gamma5_hermiticity("tiny", tiny, small),
              lambda: pd.test_complete_basis_is_exact(tiny),
              lambda: pd.test_stochastic_estimates_are_unbiased(small),
              lambda: pd.test_point_factor_is_the_pion_contraction(small),
              lambda: pd.test_two_sets_trace_factors_match_the_filled_trace(small),
              lambda: pd.test_gram_rearrangement_of_diagram2(small),
              pd.test_ensemble_subtraction_is_a_covariance]
    for c in checks:  # the mutation is caught once one pin fails
        try:
            c()
        except AssertionError:
            return False
    return True


@pytest.mark.parametrize("kind", ["q0_source_on_t", "x_on_t", "no_dagger_on_B", "point_transposed_c2",
                                  "c1_with_P_t", "fill_no_conj", "fill_no_norm", "point_propagator_transposed",
                                  "ensemble_P_t"])
def test_diagram_mutation_is_caught(kind, monkeypatch):
    from oracle import diagrams as dg

    if kind in ("q0_source_on_t", "x_on_t", "no_dagger_on_B", "c1_with_P_t"):
        monkeypatch.setattr(dg, "_per_config", _per_config_variant(kind))
    elif kind == "point_transposed_c2":
        monkeypatch.setattr(dg, "_per_config", _per_config_variant("point_transposed"))
    elif kind in ("fill_no_conj", "fill_no_norm"):
        monkeypatch.setattr(dg, "filled_propagator", _filled_variant(kind[5:]))
    elif kind == "point_propagator_transposed":
        monkeypatch.setattr(dg, "point_propagator", _point_transposed)
    else:
        monkeypatch.setattr(dg, "ensemble", _ensemble_P_t)
    assert not _run_diagram_pins(), f"mutation not caught: {kind}"
