"""Picard-then-Newton smoothing on level 0 (Sec. 3.3.2 in the reduced form): the Newton update by the persistent
FP64 BiCGStab, FAS cycles whose level-0 steps switch from Picard to Newton, and full solves, against the FP64
oracle (whose Newton update is a sparse direct solve with the exact Jacobian)."""
import numpy as np
import pytest

from oracle import fas, hierarchy, newton, tpfa
from synth.grids import problem_config, voronoi_problem

pytestmark = pytest.mark.gpu

# small cases spanning several 512-thread blocks with ragged tails (1,331, 1,024 and 1,000 cells)
CASES = {
    "chan3d_11": ("chan3d_64", 11, dict(n_levels=3, agg_size=[27, 6, 4], modes=[4, 3, 3])),
    "cart2d_32": ("cart2d_32", None, {}),
    "vor3d_10": ("voronoi", 10, {}),
}
TIGHT = dict(lin_tol=1e-13, newton_lin_tol=1e-13, lin_maxit=20000)


def _setup(nlmg_lib, key, **upd):
    name, scale, o = CASES[key]
    pr = voronoi_problem(scale) if name == "voronoi" else problem_config(name, scale=scale)
    pr.opts = dict(pr.opts, **o, **upd)
    H = hierarchy.build(pr.mesh, pr.opts)
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.opts)
    ctx.set_data(pr.f_cell, pr.g_face)
    return pr, H, ctx


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("key", list(CASES))
def test_newton_update_matches_oracle(nlmg_lib, key):
    """J(p) dx = -R(p): the BiCGStab update solves the oracle's exact Jacobian system (checked with the oracle's
    J, an independent assembly) and equals the oracle's direct solve. Tolerance: BiCGStab stops at 1e-13 on the
    Jacobi-scaled residual; the scaling and the conditioning of J (six decades of K) allow about 1e-9 in dx."""
    pr, H, ctx = _setup(nlmg_lib, key, **TIGHT)
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, pr.opts)
    rng = np.random.default_rng(21)
    for p in (np.zeros(pr.mesh.n_cells), rng.uniform(-0.2, 1.0, pr.mesh.n_cells)):
        dx, it = ctx.newton_update(p)
        R = S.R(p)
        J = tpfa.reduced_jacobian(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.g_face)
        assert it > 0
        assert np.linalg.norm(J @ dx + R) <= 1e-10 * np.linalg.norm(R)
        assert _rel(dx, S.newton_update0(p)) <= 1e-9


@pytest.mark.parametrize("key", ["chan3d_11", "cart2d_32"])
def test_picard_newton_cycles_match_oracle(nlmg_lib, key):
    """Cycle by cycle from p = 0 the GPU and the oracle switch to Newton at the same cycle and their iterates agree."""
    pr, H, ctx = _setup(nlmg_lib, key, smoother="picard_newton", newton_switch=1e-2, **TIGHT)
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, pr.opts)
    p = np.zeros(pr.mesh.n_cells)
    r0 = S.Rnorm(p)
    pg = p.copy()
    for _ in range(8):
        p, ro, eo = S.vcycle(p, r0)
        pg, rg, eg = ctx.vcycle(pg, r0)
        assert eg == eo
        assert _rel(pg, p) <= 1e-8
        assert abs(rg - ro) <= 1e-6 * r0
        if eo or ro <= 1e-8 * r0:
            break
    assert S.stats.newton_steps >= 1


def test_picard_newton_solve_reaches_newton_solution(nlmg_lib):
    """To relative residual 1e-12 the solution is Newton's p* within 1e-10 (the FP64 bar); at the default
    tolerances it takes Newton steps and no more cycles than Picard smoothing."""
    pr, H, ctx = _setup(nlmg_lib, "chan3d_11", smoother="picard_newton", **TIGHT)
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dp_clamp=pr.opts["dp_clamp"])
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face, tol_rel=1e-12, tol_abs=1e-300, max_cycles=60)
    assert st == 0, rep
    assert rep["newton_steps"] >= 1
    assert _rel(p, pstar) <= 1e-10
    r = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.f_cell, pr.g_face)
    assert np.linalg.norm(r) <= 2e-12 * rep["res0"]
    ctx.set_options(lin_tol=1e-2, coarse_lin_tol=1e-1, coarsest_lin_tol=2e-1, newton_lin_tol=1e-2, lin_maxit=5000)
    _, rep_n, st = ctx.solve(pr.f_cell, pr.g_face, max_cycles=60)
    assert st == 0 and rep_n["newton_steps"] >= 1
    ctx.set_options(smoother="picard")
    _, rep_p, st = ctx.solve(pr.f_cell, pr.g_face, max_cycles=60)
    assert st == 0 and rep_p["newton_steps"] == 0
    assert rep_n["cycles"] <= rep_p["cycles"]
    ctx.close()


def test_switch_zero_is_the_picard_smoother(nlmg_lib):
    """newton_switch = 0 never switches: bitwise the Picard-smoothed solve."""
    pr, H, ctx = _setup(nlmg_lib, "chan3d_11", smoother="picard_newton", newton_switch=0.0)
    p0, rep0, st0 = ctx.solve(pr.f_cell, pr.g_face, max_cycles=60)
    ctx.set_options(smoother="picard")
    p1, rep1, st1 = ctx.solve(pr.f_cell, pr.g_face, max_cycles=60)
    assert st0 == 0 and st1 == 0 and rep0["newton_steps"] == 0
    assert np.array_equal(p0, p1)
    ctx.close()


def test_mixed_precision_with_newton_steps(nlmg_lib):
    """FP32 inner CG for the Picard steps, FP64 BiCGStab for the Newton steps: the solution at relative residual
    1e-8 meets the tolerance in the oracle's FP64 residual."""
    pr, H, ctx = _setup(nlmg_lib, "chan3d_11", smoother="picard_newton", lin_precision=1)
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face, max_cycles=60)
    assert st == 0, rep
    r = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.f_cell, pr.g_face)
    assert np.linalg.norm(r) <= 1e-8 * rep["res0"] * 1.0001
    ctx.close()


def test_failed_newton_step_latches_like_the_oracle(nlmg_lib):
    """switch = inf: the first level-0 step is a Newton step from p = 0 that does not halve the residual; GPU and
    oracle then both return to Picard steps, cycle by cycle."""
    pr, H, ctx = _setup(nlmg_lib, "chan3d_11", smoother="picard_newton", newton_switch=float("inf"), **TIGHT)
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, pr.opts)
    p = np.zeros(pr.mesh.n_cells)
    r0 = S.Rnorm(p)
    pg = p.copy()
    for _ in range(4):
        p, ro, eo = S.vcycle(p, r0)
        pg, rg, eg = ctx.vcycle(pg, r0)
        assert eg == eo
        assert _rel(pg, p) <= 1e-8
    assert S.newton_off and S.stats.newton_steps == 1
    _, rep, st = ctx.solve(pr.f_cell, pr.g_face, max_cycles=60)
    assert st == 0 and rep["newton_steps"] == 1
    ctx.close()
