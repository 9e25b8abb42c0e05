"""Unstructured workload at a size that spans many thread blocks and four levels: clipped Voronoi cells of a jittered
40^3 lattice (64,000 cells, 5-21 neighbours), ln K ~ N(0, 2^2), kappa = (1 + p^2)^-1, aggregates of 64 then 8."""
import numpy as np
import pytest

from oracle import tpfa
from synth.grids import voronoi_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vor40(nlmg_lib):
    pr = voronoi_problem(40)
    opts = dict(pr.opts, n_levels=4, agg_size=[64, 8, 8], modes=[4, 4, 4])
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, opts)
    yield pr, ctx
    ctx.close()


def test_fp64_solution_has_oracle_residual(vor40):
    pr, ctx = vor40
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face, max_cycles=80)
    assert st == 0, rep
    r0 = np.linalg.norm(tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, np.zeros(pr.mesh.n_cells),
                                              pr.f_cell, pr.g_face))
    r = np.linalg.norm(tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.f_cell, pr.g_face))
    assert abs(rep["res0"] - r0) <= 1e-12 * r0
    assert r <= 1e-8 * r0 * 1.0001


def test_mixed_precision_reaches_the_fp64_solution(vor40):
    """FP32 inner CG, FP64 outer residual: the solution at relative residual 1e-11 agrees with the FP64 one within
    1e-8 (the bar for the mixed path)."""
    pr, ctx = vor40
    p64, rep64, st = ctx.solve(pr.f_cell, pr.g_face, tol_rel=1e-11, tol_abs=1e-300, max_cycles=120)
    assert st == 0, rep64
    ctx.set_options(lin_precision=1)
    try:
        p32, rep32, st = ctx.solve(pr.f_cell, pr.g_face, tol_rel=1e-11, tol_abs=1e-300, max_cycles=120)
    finally:
        ctx.set_options(lin_precision=0)
    assert st == 0, rep32
    assert np.linalg.norm(p32 - p64) <= 1e-8 * np.linalg.norm(p64)
    r = np.linalg.norm(tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p32, pr.f_cell, pr.g_face))
    assert r <= 1e-11 * rep32["res0"] * 1.0001


def test_full_size_unstructured_workload(nlmg_lib):
    """The 1M-cell Voronoi workload as the bench runs it (4 levels, aggregates 64 then 8, 4 modes, clamp 0.5): the
    oracle's FP64 residual of the GPU solution meets the tolerance, in FP64 and with the FP32 inner CG."""
    pr = voronoi_problem(100)
    opts = dict(pr.opts, n_levels=4, agg_size=[64, 8, 8], modes=[4, 4, 4])
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, opts)
    r0 = np.linalg.norm(tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, np.zeros(pr.mesh.n_cells),
                                              pr.f_cell, pr.g_face))
    p64, rep, st = ctx.solve(pr.f_cell, pr.g_face, max_cycles=80)
    assert st == 0, rep
    r = np.linalg.norm(tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p64, pr.f_cell, pr.g_face))
    assert r <= 1e-8 * r0 * 1.0001
    ctx.set_options(lin_precision=1)
    p32, rep, st = ctx.solve(pr.f_cell, pr.g_face, max_cycles=80)
    assert st == 0, rep
    r = np.linalg.norm(tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p32, pr.f_cell, pr.g_face))
    assert r <= 1e-8 * r0 * 1.0001
    assert np.linalg.norm(p32 - p64) <= 1e-5 * np.linalg.norm(p64)     # two solutions at relative residual 1e-8
    ctx.close()
