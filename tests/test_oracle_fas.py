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
