"""GPU parity of the batched even-odd BiCGStab solve (all inner
precisions), the pion epilogue and the error paths, through the C ABI.

Bars: every source reaches a true FP64 relative residual <= tol (checked
here by the oracle's own M on the host), and ||psi - psi_oracle|| /
||psi_oracle|| <= 1e-9 against the oracle's unpreconditioned FP64
BiCGStab solved to 1e-13, at tol = 1e-10.
"""

import numpy as np
import pytest

import oracle
from gpu_helpers import Setup, rel
from paper_1405_4524_gb300 import inputs

pytestmark = pytest.mark.gpu


def oracle_residual(s, psi, eta, kappa, csw):
    r = eta - oracle.apply_M(s.U, s.F, psi, kappa, csw, float(s.t_bc))
    return float(np.linalg.norm(r) / np.linalg.norm(eta))


@pytest.fixture(scope="module")
def small():
    spec = inputs.WORKLOADS["4x4x4x8"]
    s = Setup(spec["dims"], spec["eps"], spec["link_seed"])
    eta = inputs.make_z4(spec["dims"], spec["n_rhs"], spec["src_seed"])
    ref = []
    for k in range(eta.shape[0]):
        x, it, res = oracle.solve(s.U, eta[k], spec["kappa"], spec["csw"], -1.0, tol=1e-13, F=s.F)
        assert res <= 1e-13
        ref.append(x)
    yield s, spec, eta, np.array(ref)
    s.close()


@pytest.mark.parametrize("inner,outer", [(0, 0), (1, 0), (2, 0), (2, 1), (1, 1)])
def test_solve_matches_oracle(small, inner, outer):
    s, spec, eta, ref = small
    sq = s.sq
    n = eta.shape[0]
    sol = np.zeros_like(eta)
    prm = sq.sq_default_params(inner_prec=inner, outer=outer,
                               delta=0.1 if outer == 0 else 0.05)
    st, stats = sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], eta, sol, n, 1e-10, prm)
    assert st == 0
    for k in range(n):
        assert stats[k]["status"] == 0
        assert stats[k]["true_residual"] <= 1e-10
        assert oracle_residual(s, sol[k], eta[k], spec["kappa"], spec["csw"]) <= 1e-10
        assert rel(sol[k], ref[k]) <= 1e-9, (k, rel(sol[k], ref[k]))


def test_solve_without_graphs_and_fixed_shape(small):
    s, spec, eta, ref = small
    sq = s.sq
    n = eta.shape[0]
    sol = np.zeros_like(eta)
    prm = sq.sq_default_params(use_graph=0, sites_per_block=32, rhs_per_block=2, chunk=3)
    sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], eta, sol, n, 1e-10, prm)
    for k in range(n):
        assert rel(sol[k], ref[k]) <= 1e-9


@pytest.mark.parametrize("inner", [1, 2])
def test_graph_conditionals_match_plain_launches(small, inner):
    """The captured graph (update paths under conditional nodes, skipped
    when empty), the same graph with events around every kernel (no
    conditional nodes) and plain stream launches run the same kernels on
    the same data: bitwise identical solutions and stats. FP16 exercises
    the FP32-refresh path as well."""
    s, spec, eta, ref = small
    sq = s.sq
    n = eta.shape[0]
    out = []
    for use_graph, profile in ((1, 0), (1, 1), (0, 0), (1, 2)):
        sol = np.zeros_like(eta)
        prm = sq.sq_default_params(inner_prec=inner, use_graph=use_graph, profile=profile,
                                   sites_per_block=32, rhs_per_block=2, chunk=4)
        _, st = sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], eta, sol, n, 1e-10, prm)
        out.append((sol, [(x["iterations"], x["updates"], x["restarts"]) for x in st]))
        if profile:
            rows = {r["name"]: r for r in sq.sq_get_profile(s.ctx)}
            if profile == 2:  # only the two clover dslash launches are timed
                assert rows["dslash_clover"]["launches"] > 0 and rows["dslash_clover"]["ms"] > 0
                assert all(r["launches"] == 0 for k, r in rows.items() if k != "dslash_clover")
            else:
                assert all(r["launches"] > 0 for r in rows.values())
    for sol, st in out[1:]:
        assert np.array_equal(sol, out[0][0])
        assert st == out[0][1]
    for k in range(n):
        assert rel(out[0][0][k], ref[k]) <= 1e-9


@pytest.mark.parametrize("inner", [1, 2])
def test_default_chunks_match_fixed_chunks(small, inner):
    """The default chunks (24 iterations in the first graph launch, then 4 at
    a time) run the same iterations as fixed chunks of 16: bitwise identical
    solutions and stats, for a solve that ends in a tail launch and for a
    loose one that ends inside the first launch."""
    s, spec, eta, ref = small
    sq = s.sq
    n = eta.shape[0]
    kappa, csw = spec["kappa"], spec["csw"]

    def solve(chunk, tol):
        sol = np.zeros_like(eta)
        _, st = sq.sq_solve(s.ctx, kappa, csw, eta, sol, n, tol, sq.sq_default_params(inner_prec=inner, chunk=chunk))
        return sol, [(x["iterations"], x["updates"], x["restarts"]) for x in st]

    for tol in (1e-12, 1e-6):
        fixed, st_fixed = solve(16, tol)
        for _ in range(2):
            auto, st_auto = solve(0, tol)
            assert np.array_equal(auto, fixed) and st_auto == st_fixed
    assert max(x[0] for x in st_fixed) < 24  # the loose solve ends inside the first launch
    auto, _ = solve(0, 1e-10)
    for k in range(n):
        assert rel(auto[k], ref[k]) <= 1e-9


@pytest.mark.parametrize("inner", [1, 2])
def test_copies_of_a_source_give_identical_results(inner):
    """Four copies of one source in a batch: every reduction is per source
    in a fixed order, so the four solutions and their stats are bitwise
    equal. 8^4 has enough sites per parity that partial sums of one source
    would land in the next one's if the partial buffer were too small (the
    last copies would then differ)."""
    dims = (8, 8, 8, 8)
    s = Setup(dims, 0.25, 77)
    try:
        sq = s.sq
        n = 4
        eta = np.ascontiguousarray(np.repeat(inputs.make_z4(dims, 1, 78), n, axis=0))
        sol = np.zeros_like(eta)
        _, st = sq.sq_solve(s.ctx, 0.118, 1.0, eta, sol, n, 1e-10, sq.sq_default_params(inner_prec=inner))
        rows = [(x["iterations"], x["updates"], x["restarts"], x["true_residual"]) for x in st]
        for k in range(1, n):
            assert np.array_equal(sol[k], sol[0]), k
            assert rows[k] == rows[0], rows
        assert rows[0][1] >= 2  # an FP64-accurate update after the initial one ran
    finally:
        s.close()


def test_solve_is_deterministic(small):
    s, spec, eta, ref = small
    sq = s.sq
    n = eta.shape[0]
    a, b = np.zeros_like(eta), np.zeros_like(eta)
    prm = sq.sq_default_params(inner_prec=1)
    sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], eta, a, n, 1e-10, prm)
    sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], eta, b, n, 1e-10, prm)
    assert np.array_equal(a, b)


def test_solve_on_device_buffers(small):
    import torch

    s, spec, eta, ref = small
    sq = s.sq
    n = eta.shape[0]
    src = torch.from_numpy(eta).cuda()
    sol = torch.zeros_like(src)
    sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], src, sol, n, 1e-10)
    got = sol.cpu().numpy()
    for k in range(n):
        assert rel(got[k], ref[k]) <= 1e-9


def test_initial_guess_and_zero_source(small):
    s, spec, eta, ref = small
    sq = s.sq
    src = eta[:2].copy()
    src[1] = 0.0
    sol = np.zeros_like(src)
    sol[0] = ref[0]  # exact guess: converges at once
    prm = sq.sq_default_params(use_x0=1)
    st, stats = sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], src, sol, 2, 1e-10, prm)
    assert stats[0]["iterations"] == 0
    assert rel(sol[0], ref[0]) <= 1e-12
    assert np.all(sol[1] == 0) and stats[1]["status"] == 0


def test_pion_contraction(small):
    s, spec, eta, ref = small
    sq = s.sq
    n = eta.shape[0]
    C = sq.sq_contract_pion(s.ctx, ref, n)
    for k in range(n):
        want = oracle.pion_correlator(ref[k], 0)
        assert np.allclose(C[k], want, rtol=1e-14, atol=0)
    ts = [0, 3, 7, 5]
    C = sq.sq_contract_pion(s.ctx, ref, n, ts)
    for k in range(n):
        want = oracle.pion_correlator(ref[k], ts[k])
        assert np.allclose(C[k], want, rtol=1e-14, atol=0)


def test_fused_pion_epilogue(small):
    """sq_solve's pion output equals sq_contract_pion on the returned
    solutions (same kernel, same data) and the oracle's correlator, for
    host and device I/O, with and without time slices."""
    import torch

    s, spec, eta, ref = small
    sq = s.sq
    n, T = eta.shape[0], spec["dims"][3]
    ts = np.array([0, 3, 7, 5], dtype=np.int32)
    sol = np.zeros_like(eta)
    C = np.full((n, T), np.nan)
    sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], eta, sol, n, 1e-10, pion=C, pion_tslice=ts)
    assert np.array_equal(C, sq.sq_contract_pion(s.ctx, sol, n, list(ts)))
    for k in range(n):
        assert rel(sol[k], ref[k]) <= 1e-9
        assert np.allclose(C[k], oracle.pion_correlator(sol[k], int(ts[k])), rtol=1e-13, atol=0)
    src = torch.from_numpy(eta).cuda()
    sold = torch.zeros_like(src)
    Cd = torch.full((n, T), float("nan"), dtype=torch.float64, device="cuda")
    sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], src, sold, n, 1e-10, pion=Cd)
    assert np.array_equal(Cd.cpu().numpy(), sq.sq_contract_pion(s.ctx, sold.cpu().numpy(), n))
    Cd.fill_(float("nan"))
    sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], src, sold, n, 1e-10, pion=Cd,
                pion_tslice=torch.from_numpy(ts).cuda())
    assert np.array_equal(Cd.cpu().numpy(), C)
    with pytest.raises(ValueError):
        sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], eta, sol, n, 1e-10, pion=np.zeros((n, T + 1)))


def test_time_diluted_sources():
    dims = (4, 4, 4, 8)
    s = Setup(dims, 0.25, 1003)
    try:
        ts = [0, 3, 6]
        eta = inputs.make_z4(dims, 3, 2003, ts)
        sol = np.zeros_like(eta)
        s.sq.sq_solve(s.ctx, 0.122, 1.0, eta, sol, 3, 1e-10, s.sq.sq_default_params(inner_prec=2))
        for k in range(3):
            assert oracle_residual(s, sol[k], eta[k], 0.122, 1.0) <= 1e-10
        C = s.sq.sq_contract_pion(s.ctx, sol, 3, ts)
        for k in range(3):
            assert np.allclose(C[k], oracle.pion_correlator(sol[k], ts[k]), rtol=1e-14)
    finally:
        s.close()


# ---------------------------------------------------------------------------
# error paths (made on the host: bad inputs, tiny iteration caps)
# ---------------------------------------------------------------------------

def test_nonfinite_source_and_links(small):
    s, spec, eta, ref = small
    sq = s.sq
    bad = eta[:1].copy()
    bad[0, 1, 2, 3, 0, 2, 1] = np.nan
    sol = np.zeros_like(bad)
    with pytest.raises(sq.StochqError) as e:
        sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], bad, sol, 1, 1e-10)
    assert e.value.status == sq.SQ_ERR_NONFINITE
    U = s.U.copy()
    U[0, 0, 0, 1, 2, 0, 0] = np.inf
    ctx = sq.sq_create(s.dims)
    try:
        with pytest.raises(sq.StochqError) as e:
            sq.sq_load_gauge(ctx, U, 12)
        assert e.value.status == sq.SQ_ERR_NONFINITE
    finally:
        sq.sq_destroy(ctx)


def test_not_su3_needs_recon18(small):
    """Links that are not SU(3) are refused for reconstruct-12 and accepted
    with reconstruct-18; the FP32 and FP16 operators (both hop with the
    FP32 links) then solve the operator of those links, checked against the
    oracle's solve on the same links."""
    s, spec, eta, ref = small
    sq = s.sq
    U = 1.01 * s.U
    ctx = sq.sq_create(s.dims)
    try:
        with pytest.raises(sq.StochqError) as e:
            sq.sq_load_gauge(ctx, U, 12)
        assert e.value.status == sq.SQ_ERR_ARG
        sq.sq_load_gauge(ctx, U, 18)
        F = oracle.field_strength(U)
        want, _, res = oracle.solve(U, eta[0], spec["kappa"], spec["csw"], -1.0, tol=1e-13, F=F)
        assert res <= 1e-13
        for inner in (1, 2):
            sol = np.zeros_like(eta[:1])
            sq.sq_solve(ctx, spec["kappa"], spec["csw"], eta[:1], sol, 1, 1e-10,
                        sq.sq_default_params(inner_prec=inner))
            assert rel(sol[0], want) <= 1e-9
    finally:
        sq.sq_destroy(ctx)


def test_max_iter_gives_noconv_with_stats(small):
    s, spec, eta, ref = small
    sq = s.sq
    sol = np.zeros_like(eta)
    prm = sq.sq_default_params(max_iter=3)
    st, stats = sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], eta, sol, 4, 1e-10, prm,
                            raise_on_error=False)
    assert st == sq.SQ_ERR_NOCONV
    for k in range(4):
        assert stats[k]["status"] == sq.SQ_ERR_NOCONV
        assert 3 <= stats[k]["iterations"] <= 3 + 16
        assert 0 < stats[k]["true_residual"] < 1.0


def test_state_and_argument_errors():
    from paper_1405_4524_gb300 import stochq as sq

    ctx = sq.sq_create((4, 4, 4, 8))
    try:
        eta = np.zeros((1, 8, 4, 4, 4, 4, 3), dtype=np.complex128)
        sol = np.zeros_like(eta)
        with pytest.raises(sq.StochqError) as e:
            sq.sq_solve(ctx, 0.12, 1.0, eta, sol, 1, 1e-10)
        assert e.value.status == sq.SQ_ERR_STATE
        with pytest.raises(sq.StochqError) as e:
            sq.sq_build_clover(ctx, 0.12, 1.0)
        assert e.value.status == sq.SQ_ERR_STATE
        U = inputs.make_links((4, 4, 4, 8), 0.25, 1)
        sq.sq_load_gauge(ctx, U, 12)
        for tol in (0.0, -1.0, float("nan")):
            with pytest.raises(sq.StochqError) as e:
                sq.sq_solve(ctx, 0.12, 1.0, eta, sol, 1, tol)
            assert e.value.status == sq.SQ_ERR_ARG
        with pytest.raises(sq.StochqError) as e:
            sq.sq_load_gauge(ctx, U, 8)
        assert e.value.status == sq.SQ_ERR_ARG
    finally:
        sq.sq_destroy(ctx)


@pytest.mark.parametrize("dims", [(2, 2, 2, 4), (2, 4, 2, 6)])
def test_tiny_lattices(dims):
    """Fewer sites per parity than a warp (8 and 48): partial warps in
    every kernel and its reductions; FP32 and FP16 solves match the oracle."""
    s = Setup(dims, 0.25, 1005)
    try:
        eta = inputs.make_z4(dims, 3, 2005)
        refs = []
        for k in range(3):
            ref, _, res = oracle.solve(s.U, eta[k], 0.12, 1.0, -1.0, tol=1e-13, F=s.F)
            assert res <= 1e-13
            refs.append(ref)
        for inner in (1, 2):
            sol = np.zeros_like(eta)
            s.sq.sq_solve(s.ctx, 0.12, 1.0, eta, sol, 3, 1e-10, s.sq.sq_default_params(inner_prec=inner))
            for k in range(3):
                assert rel(sol[k], refs[k]) <= 1e-9, (inner, k)
    finally:
        s.close()


def test_empty_and_bad_batches(small):
    s, spec, eta, ref = small
    sq = s.sq
    sol = np.zeros_like(eta)
    with pytest.raises(sq.StochqError) as e:
        sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], eta, sol, 0, 1e-10)
    assert e.value.status == sq.SQ_ERR_ARG
    with pytest.raises(sq.StochqError) as e:
        sq.sq_contract_pion(s.ctx, sol, 0)
    assert e.value.status == sq.SQ_ERR_ARG


def test_solve_batch_mixed_lattices_and_kappas():
    """Three problems in one batch: two kappas sharing one lattice and a
    second lattice; every source against the oracle, and the same
    solutions as sq_solve gives problem by problem."""
    from paper_1405_4524_gb300 import stochq as sq

    dimsA, dimsB = (4, 4, 4, 8), (6, 4, 4, 6)
    sA, sB = Setup(dimsA, 0.25, 1003), Setup(dimsB, 0.25, 1004)
    try:
        csw = 1.0
        probs = [(sA, 0.118, 3, 91), (sA, 0.124, 2, 92), (sB, 0.121, 3, 93)]
        srcs = [inputs.make_z4(s.dims, n, seed) for (s, k, n, seed) in probs]
        sols = [np.zeros_like(e) for e in srcs]
        batch = [dict(ctx=s.ctx, kappa=k, c_sw=csw, sources=srcs[i], solutions=sols[i], n_rhs=n, tol=1e-10)
                 for i, (s, k, n, seed) in enumerate(probs)]
        st, stats = sq.sq_solve_batch(batch, sq.sq_default_params(inner_prec=1))
        assert st == 0 and len(stats) == 8
        assert all(x["status"] == 0 and x["true_residual"] <= 1e-10 for x in stats)
        for i, (s, k, n, seed) in enumerate(probs):
            for j in range(n):
                ref, _, res = oracle.solve(s.U, srcs[i][j], k, csw, -1.0, tol=1e-13, F=s.F)
                assert rel(sols[i][j], ref) <= 1e-9, (i, j)
            single = np.zeros_like(srcs[i])
            s.sq.sq_solve(s.ctx, k, csw, srcs[i], single, n, 1e-10, sq.sq_default_params(inner_prec=1))
            for j in range(n):
                assert rel(single[j], sols[i][j]) <= 1e-9
        # a second call reuses the cached graph and gives identical results
        again = [np.zeros_like(e) for e in srcs]
        for i, b in enumerate(batch):
            b["solutions"] = again[i]
        sq.sq_solve_batch(batch, sq.sq_default_params(inner_prec=1))
        for i in range(3):
            assert np.array_equal(again[i], sols[i])
    finally:
        sA.close()
        sB.close()


def test_near_breakdown_restarts_converge(small):
    """A loose near-breakdown threshold (|rho'| < 0.3 ||rhat|| ||r||) makes the
    recurrence restart repeatedly; the solve still reaches the oracle's
    solution, and the restarts are counted per source."""
    s, spec, eta, ref = small
    sq = s.sq
    n = eta.shape[0]
    sol = np.zeros_like(eta)
    st, stats = sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], eta, sol, n, 1e-10,
                            sq.sq_default_params(breakdown_tol=0.3))
    assert st == 0
    assert all(x["breakdowns"] >= 1 and x["restarts"] >= x["breakdowns"] for x in stats)
    for k in range(n):
        assert rel(sol[k], ref[k]) <= 1e-9


def test_repeated_breakdown_is_reported():
    """breakdown_tol > 1 declares a near breakdown at every iteration (|rho'| <=
    ||rhat|| ||r|| always); on a slowly converging system (kappa 0.128, near
    the critical kappa of these links) the 65th restart comes before
    convergence and ends every source with SQ_ERR_BREAKDOWN, with the
    per-source count in the statistics."""
    from paper_1405_4524_gb300 import stochq as sq

    spec = inputs.WORKLOADS["4x4x4x8"]
    s = Setup(spec["dims"], spec["eps"], spec["link_seed"])
    try:
        eta = inputs.make_z4(spec["dims"], 2, 2101)
        sol = np.zeros_like(eta)
        st, stats = sq.sq_solve(s.ctx, 0.128, spec["csw"], eta, sol, 2, 1e-12,
                                sq.sq_default_params(breakdown_tol=10.0), raise_on_error=False)
        assert st == sq.SQ_ERR_BREAKDOWN
        assert all(x["status"] == sq.SQ_ERR_BREAKDOWN and x["breakdowns"] > 64 for x in stats)
        assert "did not converge" in sq.sq_last_error(s.ctx)
    finally:
        s.close()


@pytest.mark.parametrize("io", ["host", "device"])
def test_fp16_fallback_to_fp32(small, io):
    """An FP16 solve cut off after 5 iterations leaves every source
    unconverged; the fallback solves them again with the FP32 inner solver
    from where the FP16 solve stopped: all converge to the oracle's
    solutions, carry fallback = 1 and their fused pion rows are those of the
    final solutions. Without the fallback the call reports SQ_ERR_NOCONV."""
    import torch

    s, spec, eta, ref = small
    sq = s.sq
    n, T = eta.shape[0], eta.shape[1]
    src = eta if io == "host" else torch.from_numpy(eta).cuda()
    sol = np.zeros_like(eta) if io == "host" else torch.zeros_like(src)
    pion = np.zeros((n, T)) if io == "host" else torch.zeros((n, T), dtype=torch.float64, device="cuda")
    prm = sq.sq_default_params(inner_prec=sq.SQ_F16, max_iter=5, fallback_max_iter=5000)
    st, stats = sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], src, sol, n, 1e-10, prm, pion=pion)
    assert st == 0
    got = sol if io == "host" else sol.cpu().numpy()
    C = pion if io == "host" else pion.cpu().numpy()
    for k in range(n):
        assert stats[k]["fallback"] == 1 and stats[k]["status"] == 0 and stats[k]["true_residual"] <= 1e-10
        assert rel(got[k], ref[k]) <= 1e-9
        assert np.allclose(C[k], oracle.pion_correlator(got[k], 0), rtol=1e-13)
    sol2 = np.zeros_like(eta)
    st, stats = sq.sq_solve(s.ctx, spec["kappa"], spec["csw"], eta, sol2, n, 1e-10,
                            sq.sq_default_params(inner_prec=sq.SQ_F16, max_iter=5, fallback=0),
                            raise_on_error=False)
    assert st == sq.SQ_ERR_NOCONV and all(x["fallback"] == 0 for x in stats)
