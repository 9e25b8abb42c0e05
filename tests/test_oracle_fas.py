"""Pins of Algorithm 1 and Algorithm 2 as implemented by the oracle."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fas, hierarchy, newton
from synth.grids import problem_config

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_backtracking_non_finite_trials():
    """A non-finite trial counts as +inf: the half step is taken if it is finite; if no trial is finite, x stays."""
    def r(y):
        return np.nan if y > 10.0 else abs(y - 1.0)
    # the full step (y = 16) is NaN, i.e. +inf; the halves y = 8, 4, 2 are finite and each is accepted (7, 3, 1),
    # halving stops once the trial is no worse than r(x) = 1: y = 2
    xn, rn, s, n = fas.backtracking(r, 0.0, 16.0, 1.0, 4, 0.9)
    assert xn == 2.0 and rn == 1.0 and s == 0.125 and n == 3
    # every trial non-finite: the iterate is returned unchanged
    xn, rn, s, n = fas.backtracking(lambda y: np.inf, 0.0, 1.0, 2.0, 4, 0.9)
    assert xn == 0.0 and rn == 2.0 and s == 0.0


def test_backtracking_hand_cases():
    rows = np.loadtxt(os.path.join(GOLD, "backtracking_quadratic.txt"))
    for x, dx, x_out, s_out, n_out in rows:
        xn, _, s, n = fas.backtracking(lambda y: abs(y * y - 2.0), x, dx, abs(x * x - 2.0), 4, 0.9)
        assert abs(xn - x_out) < 1e-15 and s == s_out and n == n_out


def _solve(pr, H, **kw):
    opts = dict(pr.opts, **kw)
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, opts)
    return S, S.solve()


@pytest.mark.parametrize("name,scale,levels", [("cart2d_32", 16, 2), ("chan3d_64", 8, 3)])
def test_fas_converges_to_newton_solution(name, scale, levels):
    """The FAS fixed point is the fine discrete solution p* (brute-force Newton), to 1e-10 at rel. residual 1e-12."""
    pr = problem_config(name, scale=scale)
    opts = dict(pr.opts, n_levels=levels)
    if name == "chan3d_64":
        opts.update(agg_size=[16, 4, 4], modes=[3, 3, 3])
    H = hierarchy.build(pr.mesh, opts)
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dp_clamp=opts["dp_clamp"])
    pr.opts = opts
    S, p = _solve(pr, H, tol_rel=1e-12, tol_abs=1e-300, max_cycles=40)
    h = S.stats.history
    assert h[-1] <= 1e-12 * h[0]
    assert np.linalg.norm(p - pstar) <= 1e-10 * np.linalg.norm(pstar)


def test_linear_two_grid_error_propagation():
    """kappa = 1, Jacobi smoothing, no backtracking: one cycle of Algorithm 2 equals the linear two-grid iteration
    p <- S^nu (p + P_p [A_c^-1 [0; P_p^T R(S^nu p)]]_p) with A_c the coarse saddle (eq. coarse_level_residual with a
    linear operator: y - Qx = -A_c^-1 R r, and the fine mixed residual is [0; -R(p)])."""
    pr = problem_config("cart2d_32", scale=8)
    pr.kappa_a = 0.0
    opts = dict(pr.opts, smoother="jacobi", bt_nmax=0, dp_clamp=0.0, nu_pre=2, nu_post=2, omega=0.8,
                agg_size=[8, 8], modes=[2, 2])
    H = hierarchy.build(pr.mesh, opts)
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, 0.0, pr.f_cell, pr.g_face, opts)
    A = newton.picard_matrix(pr.mesh, pr.kappa_kind, 0.0, np.zeros(pr.mesh.n_cells)).toarray()
    R = lambda q: S.R(q)
    d = np.diag(A)
    L1, tr = H.levels[1], H.transfers[0]
    Ac = sp.bmat([[hierarchy.assemble_M(L1), hierarchy.assemble_D(L1).T], [hierarchy.assemble_D(L1), None]]).toarray()
    Pp = tr.Pp.toarray()
    rng = np.random.default_rng(0)
    p = rng.uniform(0, 1, pr.mesh.n_cells)
    q = p.copy()
    for _ in range(2):
        q = q - 0.8 * R(q) / d
    rhs = np.concatenate([np.zeros(L1.n_flux), Pp.T @ R(q)])
    q = q + Pp @ np.linalg.solve(Ac, rhs)[L1.n_flux:]
    for _ in range(2):
        q = q - 0.8 * R(q) / d
    got, _, _ = S.vcycle(p, 0.0)
    assert np.allclose(got, q, rtol=0, atol=1e-12)


def test_jacobi_smoother_fas_reduces_residual_on_mild_problem():
    """The nonlinear Jacobi smoother is much weaker than a Picard step: on the mild 2D case every cycle still
    reduces the residual and 40 cycles gain at least three orders of magnitude."""
    pr = problem_config("cart2d_32", scale=16)
    H = hierarchy.build(pr.mesh, pr.opts)
    S, p = _solve(pr, H, smoother="jacobi", max_cycles=40)
    h = np.array(S.stats.history)
    assert np.all(h[1:] < h[:-1])
    assert h[-1] <= 1e-3 * h[0]


def test_early_exit_after_presmoothing():
    """Sec. 4: a cycle may stop after pre-smoothing once the tolerance is met (marked * in the paper's tables)."""
    pr = problem_config("cart2d_32", scale=16)
    H = hierarchy.build(pr.mesh, pr.opts)
    S, p = _solve(pr, H)
    assert S.stats.early_exit
    assert S.stats.history[-1] <= 1e-8 * S.stats.history[0]


def test_cascadic_start_reaches_the_newton_solution():
    """The nonlinear cascadic start (coarse problems solved bottom-up, corrections carried up with Algorithm 1)
    followed by FAS cycles converges to the same p* as Newton."""
    from oracle import hierarchy, newton
    from synth.grids import problem_config
    pr = problem_config("cart2d_32", scale=16)
    H = hierarchy.build(pr.mesh, pr.opts)
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face)
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dict(pr.opts, tol_rel=1e-11))
    p = S.solve(cascadic=True)
    assert S.stats.history[1] < S.stats.history[0]          # the cascadic iterate is better than p0 here
    assert np.linalg.norm(p - pstar) <= 1e-9 * np.linalg.norm(pstar)


def _fas(pr, H, **kw):
    return fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dict(pr.opts, **kw))


def test_newton_update_is_the_linearised_zero():
    """The level-0 Newton update (Sec. 3.3.2) zeroes the first-order model: R(p + e dp) = (1 - e) R(p) + O(e^2),
    checked by the second-order behaviour of the remainder as e halves (a wrong sign, a transposed or a missing
    Jacobian term leaves an O(e) remainder)."""
    pr = problem_config("chan3d_64", scale=6)
    H = hierarchy.build(pr.mesh, pr.opts)
    S = _fas(pr, H)
    rng = np.random.default_rng(3)
    p = rng.uniform(0.0, 1.0, pr.mesh.n_cells)
    Rp = S.R(p)
    dp = S.newton_update0(p)
    rem = []
    for e in (1e-2, 5e-3, 2.5e-3):
        rem.append(np.linalg.norm(S.R(p + e * dp) - (1.0 - e) * Rp))
    assert 3.5 <= rem[0] / rem[1] <= 4.5 and 3.5 <= rem[1] / rem[2] <= 4.5


def test_newton_smoothing_converges_quadratically_near_the_solution():
    """From p* + a small perturbation, successive level-0 Newton smoothing steps (switch = inf) square the error:
    log(r_{k+1}) / log(r_k) near 2 (Picard steps only contract linearly)."""
    pr = problem_config("cart2d_32", scale=12)
    H = hierarchy.build(pr.mesh, pr.opts)
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face)
    S = _fas(pr, H, smoother="picard_newton", newton_switch=np.inf)
    S.r0_ref = 1.0
    rng = np.random.default_rng(5)
    p = pstar + 0.05 * rng.standard_normal(pstar.size)
    r = [S.Rnorm(p)]
    for _ in range(3):
        p, rn = S.smooth0(p, 1)
        r.append(rn)
    rel = np.array(r) / r[0]
    assert S.stats.newton_steps == 3
    assert rel[2] <= 5.0 * rel[1] ** 2 and rel[3] <= 5.0 * rel[2] ** 2 and rel[3] < 1e-9
    P = _fas(pr, H)
    q = pstar + 0.05 * rng.standard_normal(pstar.size)
    rq = [P.Rnorm(q)]
    for _ in range(3):
        q, rn = P.smooth0(q, 1)
        rq.append(rn)
    # Picard contracts linearly (consecutive ratios alike); Newton's ratio collapses from step to step
    assert rq[3] / rq[2] > 0.2 * rq[2] / rq[1]
    assert r[3] / r[2] < 0.01 * r[2] / r[1]


def test_picard_newton_switch_extremes_and_fixed_point():
    """newton_switch = 0: bitwise the Picard FAS (no Newton step); the default switch reaches Newton's p* with fewer
    cycles on the channelized case, where the Newton steps remove the linear tail of the Picard iteration."""
    pr = problem_config("chan3d_64", scale=10)
    H = hierarchy.build(pr.mesh, pr.opts)
    S0 = _fas(pr, H)
    p0 = S0.solve()
    S1 = _fas(pr, H, smoother="picard_newton", newton_switch=0.0)
    p1 = S1.solve()
    assert np.array_equal(p0, p1) and S1.stats.newton_steps == 0
    S2 = _fas(pr, H, smoother="picard_newton", newton_switch=1e-2, tol_rel=1e-12, tol_abs=1e-300)
    p2 = S2.solve(max_cycles=40)
    assert S2.stats.newton_steps >= 1
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dp_clamp=pr.opts["dp_clamp"])
    assert np.linalg.norm(p2 - pstar) <= 1e-10 * np.linalg.norm(pstar)
    S3 = _fas(pr, H, smoother="picard_newton", newton_switch=1e-2)
    S3.solve()
    assert S3.stats.cycles < S0.stats.cycles


def test_failed_newton_step_returns_to_picard():
    """switch = inf on the channelized case: the first smoothing step is a Newton step from p = 0, outside Newton's
    region of fast convergence, so it does not halve the residual; every later step is a Picard step and the solve
    still reaches p*."""
    pr = problem_config("chan3d_64", scale=11)
    pr.opts = dict(pr.opts, n_levels=3, agg_size=[27, 6, 4], modes=[4, 3, 3])
    H = hierarchy.build(pr.mesh, pr.opts)
    S = _fas(pr, H, smoother="picard_newton", newton_switch=np.inf, tol_rel=1e-12, tol_abs=1e-300)
    p = S.solve(max_cycles=40)
    assert S.stats.newton_steps == 1 and S.newton_off
    assert S.stats.history[1] > 0.5 * S.stats.history[0]
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dp_clamp=pr.opts["dp_clamp"])
    assert np.linalg.norm(p - pstar) <= 1e-10 * np.linalg.norm(pstar)
    S.solve()                       # a new solve clears the latch
    assert S.stats.newton_steps == 2


def test_cascade_on_a_linear_problem_is_a_galerkin_coarse_correction():
    """kappa = 1 (linear): with two levels the cascade solves the coarse FAS problem exactly (its Picard steps are
    exact linear solves), so it moves p by s P_p e_p, e = (P^T A P)^-1 [0; P_p^T R(p)], with A the mixed matrix of
    eq. FV_matrix and s the step Algorithm 1 takes. Built here from tpfa's matrices and residual, not the oracle's
    coarse operators: a wrong sign or a transposed transfer in the cascade's right-hand side moves p elsewhere."""
    import scipy.sparse as sp
    from oracle import tpfa
    pr = problem_config("cart2d_32", scale=13)
    opts = dict(pr.opts, n_levels=2, agg_size=[9, 4], modes=[3, 2], dp_clamp=0.0)
    H = hierarchy.build(pr.mesh, opts)
    kind, a = tpfa.KAPPA_EXP, 0.0
    assert np.all(tpfa.kappa(np.linspace(-3, 3, 7), kind, a) == 1.0)
    S = fas.FAS(H, pr.mesh, kind, a, pr.f_cell, pr.g_face, opts)
    p0 = np.random.default_rng(5).uniform(0.0, 1.0, pr.mesh.n_cells)
    p1 = S.cascade(p0.copy())
    M, D, _, _, _ = tpfa.mixed_matrices(pr.mesh, kind, a, p0, pr.f_cell, pr.g_face)
    A0 = sp.bmat([[M, D.T], [D, None]]).tocsr()
    tr = H.transfers[0]
    P = sp.block_diag([tr.Psigma, tr.Pp]).tocsr()
    A1 = (P.T @ A0 @ P).toarray()
    R = tpfa.reduced_residual(pr.mesh, kind, a, p0, pr.f_cell, pr.g_face)
    nf1 = H.levels[1].n_flux
    e = np.linalg.solve(A1, np.concatenate([np.zeros(nf1), tr.Pp.T @ R]))
    dp = tr.Pp @ e[nf1:]
    assert np.linalg.norm(dp) > 0
    err = min(np.linalg.norm(p1 - (p0 + s * dp)) for s in (1.0, 0.5, 0.25, 0.125, 0.0625))
    assert err <= 1e-9 * np.linalg.norm(dp)
