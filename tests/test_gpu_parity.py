"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, step by step and end to end."""
import numpy as np
import pytest

from oracle import coarse, fas, hierarchy, newton, tpfa
from synth.grids import cartesian_mesh, lognormal_field, problem_config, voronoi_problem, KAPPA_INV1P2

pytestmark = pytest.mark.gpu

# (name, scale, option overrides): small cases that span several thread blocks and leave ragged tails
CASES = {
    "cart2d_32": ("cart2d_32", None, {}),
    "cart2d_13": ("cart2d_32", 13, dict(agg_size=[9, 4], modes=[3, 2])),
    "chan3d_16": ("chan3d_64", 16, dict(n_levels=3, agg_size=[64, 8, 8], modes=[4, 4, 4])),
    "chan3d_11": ("chan3d_64", 11, dict(n_levels=3, agg_size=[27, 6, 4], modes=[4, 3, 3])),
    "vor3d_10": ("voronoi", 10, {}),     # unstructured: clipped Voronoi cells, 5-21 neighbours, kappa = 1/(1+p^2)
    # m_f = 3 flux unknowns per coarse interface (App. A.2): up to 51 local flux unknowns per coarse cell
    "chan3d_16_mf3": ("chan3d_64", 16, dict(n_levels=3, agg_size=[64, 8, 8], modes=[4, 4, 4], flux_modes=[3, 3, 3])),
}
TIGHT = dict(lin_tol=1e-13, lin_maxit=20000)


def _setup(nlmg_lib, key, **upd):
    name, scale, o = CASES[key]
    pr = voronoi_problem(scale) if name == "voronoi" else problem_config(name, scale=scale)
    opts = dict(pr.opts, **o)
    opts.update(upd)
    pr.opts = opts
    H = hierarchy.build(pr.mesh, opts)
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, opts)
    ctx.set_data(pr.f_cell, pr.g_face)
    return pr, H, ctx


@pytest.fixture(scope="module", params=list(CASES))
def case(request, nlmg_lib):
    return _setup(nlmg_lib, request.param, **TIGHT)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_fine_residual_and_flux(case):
    pr, H, ctx = case
    rng = np.random.default_rng(11)
    for p in (np.zeros(pr.mesh.n_cells), rng.uniform(-0.3, 1.2, pr.mesh.n_cells)):
        r = ctx.fine_residual(p)
        ro = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.f_cell, pr.g_face)
        sig = tpfa.face_fluxes(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.g_face)
        scale = np.abs(sig).max()
        assert np.abs(r - ro).max() <= 1e-13 * scale
        s = ctx.fine_flux(p)
        assert np.abs(s - sig[tpfa.flux_dofs(pr.mesh)]).max() <= 1e-14 * scale


def test_level_operator(case):
    pr, H, ctx = case
    rng = np.random.default_rng(12)
    for l in range(1, len(H.levels)):
        lev = H.levels[l]
        x = rng.uniform(-1, 1, lev.n_flux + lev.n_p)
        got = ctx.level_apply(l, x)
        ref = coarse.operator(lev, pr.kappa_kind, pr.kappa_a, x[:lev.n_flux], x[lev.n_flux:])
        # the two hierarchies agree to ~1e-12 (test_abi); bound the difference by 1e-10 of the largest row sum of
        # |terms| (|M(Pi~ p)| |sigma| + |D^T| |p|; |D| |sigma|)
        s = 1.0 / tpfa.kappa(coarse.pbar(lev, x[lev.n_flux:]), pr.kappa_kind, pr.kappa_a)
        M = abs(hierarchy.assemble_M(lev, s))
        D = abs(hierarchy.assemble_D(lev))
        ax = np.abs(x)
        bound = np.concatenate([M @ ax[:lev.n_flux] + D.T @ ax[lev.n_flux:], D @ ax[:lev.n_flux]])
        assert np.abs(got - ref).max() <= 1e-10 * bound.max()


def test_transfers(case, nlmg_lib):
    pr, H, ctx = case
    rng = np.random.default_rng(13)
    # the library's hierarchy is compared here through the oracle's: with m_f > 1 its interface traces come from an
    # SVD (App. A.2) taken by two different algorithms, which agree to 1e-9 relative (host hierarchy parity)
    tol = 1e-9 if max(pr.opts.get("flux_modes", [1])) > 1 else 1e-10
    for l, tr in enumerate(H.transfers):
        levc = H.levels[l + 1]
        if l == 0:
            p = rng.uniform(0, 1, pr.mesh.n_cells)
            sig = tpfa.face_fluxes(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.g_face)[tpfa.flux_dofs(pr.mesh)]
            ref = np.concatenate([tr.Qsigma @ sig, tr.Qp @ p])
            got = ctx.transfer(0, nlmg_lib.PROJECT, p)
            rp = rng.uniform(-1, 1, pr.mesh.n_cells)
            ref_r = np.concatenate([np.zeros(levc.n_flux), tr.Pp.T @ rp])
            got_r = ctx.transfer(0, nlmg_lib.RESTRICT, rp)
            e = rng.uniform(-1, 1, levc.n_flux + levc.n_p)
            ref_e = tr.Pp @ e[levc.n_flux:]
        else:
            lev = H.levels[l]
            x = rng.uniform(-1, 1, lev.n_flux + lev.n_p)
            ref = np.concatenate([tr.Qsigma @ x[:lev.n_flux], tr.Qp @ x[lev.n_flux:]])
            got = ctx.transfer(l, nlmg_lib.PROJECT, x)
            ref_r = np.concatenate([tr.Psigma.T @ x[:lev.n_flux], tr.Pp.T @ x[lev.n_flux:]])
            got_r = ctx.transfer(l, nlmg_lib.RESTRICT, x)
            e = rng.uniform(-1, 1, levc.n_flux + levc.n_p)
            ref_e = np.concatenate([tr.Psigma @ e[:levc.n_flux], tr.Pp @ e[levc.n_flux:]])
        got_e = ctx.transfer(l, nlmg_lib.PROLONG, e)
        for g_, r_ in ((got, ref), (got_r, ref_r), (got_e, ref_e)):
            assert np.abs(g_ - r_).max() <= tol * max(1.0, np.abs(r_).max())


def test_picard_updates(case):
    """Level 0: A(kappa(p)) dp = -R(p); coarse: the frozen saddle (hybridized PCG vs the oracle's sparse LU)."""
    pr, H, ctx = case
    rng = np.random.default_rng(14)
    p = rng.uniform(0, 1, pr.mesh.n_cells)
    dp, it = ctx.picard_update(0, p)
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, pr.opts)
    ref = -np.linalg.solve(S.picard_matrix0(p).toarray(), S.R(p)) if pr.mesh.n_cells <= 2000 else None
    if ref is None:
        import scipy.sparse.linalg as spla
        ref = -spla.spsolve(S.picard_matrix0(p).tocsc(), S.R(p))
    assert it > 0 and _rel(dp, ref) <= 1e-9
    for l in range(1, len(H.levels)):
        lev = H.levels[l]
        x = rng.uniform(-0.5, 0.5, lev.n_flux + lev.n_p)
        b = rng.uniform(-1, 1, lev.n_flux + lev.n_p)
        dx, _ = ctx.picard_update(l, x, b)
        sP, pP = coarse.picard_solve(lev, pr.kappa_kind, pr.kappa_a, x[:lev.n_flux], x[lev.n_flux:], b)
        assert _rel(dx, np.concatenate([sP, pP]) - x) <= 1e-9


def test_one_vcycle_matches_oracle(case):
    pr, H, ctx = case
    p0 = np.zeros(pr.mesh.n_cells)
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, pr.opts)
    r0 = S.Rnorm(p0)
    po, ro, eo = S.vcycle(p0, r0)
    pg, rg, eg = ctx.vcycle(p0, r0)
    assert eg == eo
    assert _rel(pg, po) <= 1e-8
    assert abs(rg - ro) <= 1e-6 * r0


def test_solve_matches_newton_solution(case):
    """The bar for the FP64 path: the GPU solution within 1e-10 of p* when run to relative residual 1e-12."""
    pr, H, ctx = case
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dp_clamp=pr.opts["dp_clamp"])
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face, tol_rel=1e-12, tol_abs=1e-300, max_cycles=60)
    assert st == 0, rep
    assert rep["res"] <= 1e-12 * rep["res0"]
    assert _rel(p, pstar) <= 1e-10
    # independent check of the returned iterate with the oracle's residual
    r = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.f_cell, pr.g_face)
    assert np.linalg.norm(r) <= 2e-12 * rep["res0"]


def test_fas_cycle_counts_follow_oracle(nlmg_lib):
    """At the default tolerances (rel 1e-8) both FAS implementations take the same number of cycles."""
    pr, H, ctx = _setup(nlmg_lib, "chan3d_16", **TIGHT)
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, pr.opts)
    S.solve()
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face)
    assert st == 0
    assert rep["cycles"] == S.stats.cycles and rep["early_exit"] == S.stats.early_exit
    h = np.array(rep["history"])
    ho = np.array(S.stats.history)
    assert np.allclose(h, ho, rtol=1e-6, atol=1e-9 * ho[0])


def test_flux_modes_cycle_counts_follow_oracle(nlmg_lib):
    """m_f = 3: both FAS implementations take the same cycles (fewer than with m_f = 1 on this case: 9 against 13)."""
    pr, H, ctx = _setup(nlmg_lib, "chan3d_16_mf3", **TIGHT)
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, pr.opts)
    S.solve()
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face)
    assert st == 0
    assert rep["cycles"] == S.stats.cycles and rep["early_exit"] == S.stats.early_exit
    h = np.array(rep["history"])
    ho = np.array(S.stats.history)
    assert np.allclose(h, ho, rtol=1e-6, atol=1e-9 * ho[0])


def test_more_than_64_local_flux_unknowns(nlmg_lib):
    """m_f = 4 on 64-cell aggregates gives coarse cells with up to 66 local flux unknowns: the GPU solve follows the
    oracle's cycles and residual history."""
    pr = problem_config("chan3d_64", scale=16)
    opts = dict(pr.opts, n_levels=3, agg_size=[64, 8, 8], modes=[4, 4, 4], flux_modes=[4, 4, 4], **TIGHT)
    H = hierarchy.build(pr.mesh, opts)
    assert max(len(x) for x in H.levels[1].loc) > 64
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, opts)
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, opts)
    po = S.solve()
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face)
    assert st == 0 and rep["cycles"] == S.stats.cycles
    ho = np.array(S.stats.history)
    assert np.allclose(np.array(rep["history"]), ho, rtol=1e-6, atol=1e-9 * ho[0])
    assert _rel(p, po) <= 1e-6


@pytest.mark.parametrize("key", ["cart2d_13", "chan3d_11"])
def test_cascadic_start_matches_oracle(nlmg_lib, key):
    """Nonlinear cascadic start (Sec. 4.2) then FAS cycles: the same iterate after the cascade (second history entry)
    and the same cycles as the oracle's FAS.cascade."""
    pr, H, ctx = _setup(nlmg_lib, key, cascadic=1, **TIGHT)
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, pr.opts)
    S.solve(cascadic=True)
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face)
    assert st == 0
    h = np.array(rep["history"])
    ho = np.array(S.stats.history)
    assert h.size == ho.size and rep["cycles"] == S.stats.cycles
    assert np.allclose(h, ho, rtol=1e-6, atol=1e-9 * ho[0])


def test_jacobi_smoother_cycle_matches_oracle(nlmg_lib):
    pr, H, ctx = _setup(nlmg_lib, "cart2d_32", smoother="jacobi", **TIGHT)
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, pr.opts)
    p = np.zeros(pr.mesh.n_cells)
    r0 = S.Rnorm(p)
    pg = p.copy()
    for _ in range(3):
        p, _, _ = S.vcycle(p, r0)
        pg, _, _ = ctx.vcycle(pg, r0)
        assert _rel(pg, p) <= 1e-9


def test_single_level_picard_baseline(nlmg_lib):
    pr, H, ctx = _setup(nlmg_lib, "chan3d_11", **TIGHT)
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dp_clamp=pr.opts["dp_clamp"])
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face, tol_rel=1e-12, tol_abs=1e-300, max_cycles=200, picard_only=True)
    assert st == 0
    assert _rel(p, pstar) <= 1e-10


def test_other_nonlinearity_and_single_level(nlmg_lib):
    """kappa = (1 + p^2)^-1, log-normal sigma = 2, one level only (FAS reduces to Picard smoothing)."""
    n = 9
    mesh = cartesian_mesh((n, n, n), lognormal_field((n, n, n), 2.0, 3.0, seed=5))
    g = np.zeros(mesh.n_faces)
    d = np.where(mesh.face_bc == 1)[0]
    g[d] = np.where(mesh.face_cells[d, 0] % n == 0, 1.5, -0.5)
    f = np.random.default_rng(3).uniform(-1, 1, mesh.n_cells)
    pstar, _ = newton.solve(mesh, KAPPA_INV1P2, 0.0, f, g)
    for levels in (1, 2):
        opts = dict(problem_config("cart2d_32").opts, n_levels=levels, agg_size=[27, 8], modes=[3, 3], **TIGHT)
        ctx = nlmg_lib.Context(mesh, KAPPA_INV1P2, 0.0, opts)
        p, rep, st = ctx.solve(f, g, tol_rel=1e-13, tol_abs=1e-300, max_cycles=80)
        assert st == 0, rep
        assert _rel(p, pstar) <= 1e-10


def test_degenerate_tiny_meshes(nlmg_lib):
    """One cell; a 2x1 strip whose single aggregate is the whole mesh (coarsest level of one cell)."""
    for shape in ((1, 1), (2, 1), (3, 2)):
        mesh = cartesian_mesh(shape, np.ones(int(np.prod(shape))))
        g = np.where(mesh.face_bc == 1, np.where(mesh.face_cells[:, 0] % shape[0] == 0, 1.0, 0.0), 0.0)
        f = np.zeros(mesh.n_cells)
        pstar, _ = newton.solve(mesh, 0, 1.0, f, g)
        opts = dict(problem_config("cart2d_32").opts, n_levels=2 if mesh.n_cells > 1 else 1, agg_size=[8, 8],
                    modes=[2, 2], **TIGHT)
        ctx = nlmg_lib.Context(mesh, 0, 1.0, opts)
        p, rep, st = ctx.solve(f, g, tol_rel=1e-12, tol_abs=1e-300, max_cycles=40)
        assert st == 0, (shape, rep)
        assert _rel(p, pstar) <= 1e-10


def test_mixed_precision_cg_reaches_fp64_solution(nlmg_lib):
    """FP32 CG inside the FP64 nonlinear iteration: the FAS still converges to the FP64 solution p* (the north
    star's bar for the mixed path: <= 1e-8 relative error after the FP64 outer residual check)."""
    pr, H, ctx = _setup(nlmg_lib, "chan3d_16", lin_precision=1, lin_tol=1e-6, coarse_lin_tol=1e-6)
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dp_clamp=pr.opts["dp_clamp"])
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face, tol_rel=1e-11, tol_abs=1e-300, max_cycles=80)
    assert st == 0, rep
    r = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.f_cell, pr.g_face)
    assert np.linalg.norm(r) <= 2e-11 * rep["res0"]
    assert _rel(p, pstar) <= 1e-8


def test_single_level_newton_baseline(nlmg_lib):
    """Exact Jacobian + GMRES (Sec. 2.2 / 3.3.2 on level 0). Linear case (kappa = 1): one Newton step solves the
    problem. Mild nonlinear 2D case: converges to p* and, once close, quadratically."""
    pr, H, ctx = _setup(nlmg_lib, "cart2d_32", **TIGHT)
    lin = nlmg_lib.Context(pr.mesh, pr.kappa_kind, 0.0, dict(pr.opts))
    pl, rep, st = lin.solve(pr.f_cell, pr.g_face, tol_rel=1e-11, tol_abs=1e-300, max_cycles=5, newton=True)
    assert st == 0 and rep["cycles"] <= 2, rep
    p_lin, _ = newton.solve(pr.mesh, pr.kappa_kind, 0.0, pr.f_cell, pr.g_face)
    assert _rel(pl, p_lin) <= 1e-10
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dp_clamp=pr.opts["dp_clamp"])
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face, tol_rel=1e-12, tol_abs=1e-300, max_cycles=200, newton=True)
    assert st == 0, rep
    assert _rel(p, pstar) <= 1e-10
    h = np.array(rep["history"]) / rep["history"][0]
    k = int(np.argmax(h < 1e-3))                     # first iterate in the local regime
    assert h[-1] <= 1e-12 and len(h) - k <= 4          # at most a few steps from 1e-3 to 1e-12


def test_full_size_bench_configuration(nlmg_lib):
    """The benchmarked 64^3 workload in its benchmarked configuration (Picard-then-Newton level-0 smoothing, the
    library's inner tolerances): the returned iterate meets the relative tolerance when its residual is recomputed by
    the oracle, and sampled residual rows agree."""
    pr = problem_config("chan3d_64")
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, dict(pr.opts, smoother="picard_newton"))
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face)
    assert st == 0, rep
    assert rep["newton_steps"] > 0
    r = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.f_cell, pr.g_face)
    r0 = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, np.zeros(pr.mesh.n_cells), pr.f_cell, pr.g_face)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(r0) * 1.0001
    ctx.set_data(pr.f_cell, pr.g_face)
    rg = ctx.fine_residual(p)
    rows = np.random.default_rng(5).choice(pr.mesh.n_cells, 4096, replace=False)
    sig = tpfa.face_fluxes(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.g_face)
    assert np.abs(rg[rows] - r[rows]).max() <= 1e-13 * np.abs(sig).max()


def test_bench_options_reach_the_newton_solution(nlmg_lib):
    """The benchmark's solver options (Picard-then-Newton smoothing, loose inner tolerances) on the 32^3 instance of
    the same generator and hierarchy shape, run to relative residual 1e-12: the solution is p* within 1e-10; at the
    benchmark's 1e-8 the error against p* is reported by the bench and bounded here by 1e-6."""
    pr = problem_config("chan3d_64", scale=32)
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, dict(pr.opts, smoother="picard_newton"))
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dp_clamp=pr.opts["dp_clamp"])
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face, tol_rel=1e-12, tol_abs=1e-300, max_cycles=60)
    assert st == 0, rep
    assert _rel(p, pstar) <= 1e-10
    p8, rep8, st8 = ctx.solve(pr.f_cell, pr.g_face)
    assert st8 == 0 and rep8["newton_steps"] > 0
    assert _rel(p8, pstar) <= 1e-6
