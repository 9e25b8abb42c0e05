"""Several right-hand sides on one hierarchy: shared-hierarchy instances and the multi-right-hand-side solve.

The hierarchy is built from the reference operator at kappa = 1 (App. A), so one setup serves every right-hand side,
boundary datum and nonlinearity parameter; each row must come out as the single solve would give it, and match the
FP64 oracle's p* for that row.
"""
import numpy as np
import pytest

from oracle import newton, tpfa
from synth.grids import multi_rhs_rows, problem_config

pytestmark = pytest.mark.gpu

TIGHT = dict(lin_tol=1e-13, lin_maxit=20000)


def _rows(pr, n_rhs, seed):
    return multi_rhs_rows(pr.mesh, n_rhs, seed)


def _problem(scale=11):
    pr = problem_config("chan3d_64", scale=scale)
    pr.opts = dict(pr.opts, n_levels=3, agg_size=[27, 6, 4], modes=[4, 3, 3])
    return pr


def _sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("max_sms", [0, 40])
def test_many_rows_equal_single_solves(nlmg_lib, max_sms):
    """Each row equals the single solve on a context with the SM share the batch used (given, or SMs / min(3, 4)
    for n_streams = 3): bitwise, whatever ran beside it."""
    pr = _problem()
    F, G = _rows(pr, 6, seed=50)
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, dict(pr.opts, max_sms=max_sms))
    P, reps, sts = ctx.solve_many(F, G, max_cycles=60, n_streams=3)
    assert np.all(sts == 0)
    ctx.set_options(max_sms=max_sms or _sms() // 3)
    for r in range(F.shape[0]):
        p1, rep1, st1 = ctx.solve(F[r], G[r], max_cycles=60)
        assert st1 == 0
        assert np.array_equal(P[r], p1)          # bitwise: private buffers, fixed-order reductions
        assert reps[r]["cycles"] == rep1["cycles"]
        res = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, P[r], F[r], G[r])
        assert np.linalg.norm(res) <= 1e-8 * reps[r]["res0"] * 1.0001
    ctx.close()


def test_many_rows_match_oracle(nlmg_lib):
    pr = _problem()
    F, G = _rows(pr, 3, seed=51)
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, dict(pr.opts, **TIGHT))
    P, reps, sts = ctx.solve_many(F, G, tol_rel=1e-12, tol_abs=1e-300, max_cycles=80, n_streams=3)
    assert np.all(sts == 0)
    for r in range(F.shape[0]):
        pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, F[r], G[r], dp_clamp=pr.opts["dp_clamp"])
        assert np.linalg.norm(P[r] - pstar) <= 1e-10 * np.linalg.norm(pstar)
    ctx.close()


def test_instance_with_other_parameter_equals_fresh_setup(nlmg_lib):
    """An instance with kappa = exp(a p), a != base's, solves exactly as a context set up for that a."""
    pr = _problem(scale=9)
    F, G = _rows(pr, 1, seed=52)
    base = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.opts)
    a2 = 1.25
    inst = base.instance(pr.kappa_kind, a2)
    fresh = nlmg_lib.Context(pr.mesh, pr.kappa_kind, a2, pr.opts)
    p_i, rep_i, st_i = inst.solve(F[0], G[0], max_cycles=60)
    p_f, rep_f, st_f = fresh.solve(F[0], G[0], max_cycles=60)
    assert st_i == 0 and st_f == 0
    assert np.array_equal(p_i, p_f)
    # the instance outlives its base: the shared hierarchy is freed with the last context
    base.close()
    p_j, _, st_j = inst.solve(F[0], G[0], max_cycles=60)
    assert st_j == 0 and np.array_equal(p_j, p_i)
    inst.close()
    fresh.close()


def test_empty_and_bad_batches(nlmg_lib):
    pr = _problem(scale=6)
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.opts)
    P, reps, sts = ctx.solve_many(np.zeros((0, pr.mesh.n_cells)), np.zeros((0, pr.mesh.n_faces)))
    assert P.shape == (0, pr.mesh.n_cells) and reps == []
    with pytest.raises(ValueError):
        ctx.solve_many(np.zeros((2, pr.mesh.n_cells)), np.zeros((3, pr.mesh.n_faces)))
    ctx.close()


def test_set_options_between_solves(nlmg_lib):
    pr = _problem(scale=8)
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.opts)
    p64, rep64, st = ctx.solve(pr.f_cell, pr.g_face, max_cycles=60)
    assert st == 0
    ctx.set_options(lin_precision=1)
    p32, rep32, st = ctx.solve(pr.f_cell, pr.g_face, max_cycles=60)
    assert st == 0
    assert np.linalg.norm(p32 - p64) <= 1e-6 * np.linalg.norm(p64)     # both at relative residual 1e-8
    ctx.set_options(lin_precision=0)
    p64b, _, st = ctx.solve(pr.f_cell, pr.g_face, max_cycles=60)
    assert st == 0 and np.array_equal(p64b, p64)
    ctx.close()


def test_loose_inner_tolerances_do_not_stall(nlmg_lib):
    """Row 0 of this batch stalls near relative residual 3e-5 with fixed inner tolerances 1e-2 / 1e-1 (measured);
    the solver divides them by 100 after a stalled cycle and then converges like the exact-inner-solve oracle."""
    pr = _problem()
    F, G = _rows(pr, 1, seed=50)
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, dict(pr.opts, lin_tol=1e-2, coarse_lin_tol=1e-1))
    p, rep, st = ctx.solve(F[0], G[0], max_cycles=60)
    assert st == 0, rep
    assert rep["tol_tightened"] >= 1
    r = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p, F[0], G[0])
    assert np.linalg.norm(r) <= 1e-8 * rep["res0"] * 1.0001
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, F[0], G[0], dp_clamp=pr.opts["dp_clamp"])
    assert np.linalg.norm(p - pstar) <= 1e-6 * np.linalg.norm(pstar)
    ctx.close()


def test_sm_share_tuner_returns_a_candidate(nlmg_lib):
    """The autotuner times the four SM shares and returns one of them; the context's options are left alone."""
    pr = _problem(scale=8)
    F, G = _rows(pr, 2, seed=53)
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.opts)
    p0, _, st = ctx.solve(F[0], G[0], max_cycles=60)
    assert st == 0
    best, rates = ctx.tune_sm_share(F, G)
    sms = _sms()
    assert best in (sms, sms // 2, sms // 4, sms // 8)
    assert np.all(rates > 0)
    p1, _, st = ctx.solve(F[0], G[0], max_cycles=60)
    assert st == 0 and np.array_equal(p0, p1)      # same options as before the tuning
    ctx.close()
