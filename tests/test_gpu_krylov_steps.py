"""Step parity of the Krylov kernels the benchmarked solves run, at the loose tolerances they run with.

A Krylov iterate after k steps from a zero start is fixed by the method, whatever recurrences compute it, and so is
the step at which a residual test stops it. The oracle's plain fixed-length iterations (oracle.krylov) on the
oracle's independently assembled systems (the frozen TPFA matrix, the exact Jacobian, the hybridized coarse saddle of
Sec. 3.4) must therefore match every variant the library selects, step count and iterate:
  * level-0 Picard CG (nlmg_picard_update, level 0): the register-resident pipelined FP64 CG (tolerance >= 1e-6, at most
    4 cells per thread), the memory-resident pipelined FP64 CG (max_sms = 1: more than 4 cells per thread), the
    two-barrier FP64 CG (tolerance < 1e-6), the FP32 pipelined CG with residual replacement and the FP32 two-barrier
    CG (lin_precision = 1; max_sms = 1 gives more than 8 cells per thread);
  * level-0 Newton BiCGStab (nlmg_newton_update);
  * the hybridized CG inside the fused coarse step (nlmg_picard_update, level >= 1): pipelined with the lambdas in
    registers (every lambda gets lanes in one pass of the grid), pipelined in memory (max_sms = 1 on level 1, whose
    lambdas then outnumber the grid's lanes), and the two-synchronisation form (tolerance < 1e-6).
The 32^3 channelized case has 32,768 cells: with all SMs every thread of the level-0 kernels holds one cell; with
max_sms = 1 the grid has at most 2 x 512 threads, i.e. 32 cells per thread.
"""
import numpy as np
import pytest

from oracle import coarse, fas, hierarchy, krylov, newton, tpfa
from synth.grids import problem_config

pytestmark = pytest.mark.gpu

N_SIDE = 32


@pytest.fixture(scope="module")
def setup(nlmg_lib):
    pr = problem_config("chan3d_64", scale=N_SIDE)
    opts = dict(pr.opts, n_levels=3, agg_size=[64, 8, 8], modes=[4, 4, 4])
    H = hierarchy.build(pr.mesh, opts)
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, opts)
    ctx.set_data(pr.f_cell, pr.g_face)
    # an iterate of the kind a solve meets: the solution of the same problem with half the nonlinearity, perturbed
    # (at random pressures the exact Jacobian is far from an M-matrix and BiCGStab's rounding grows chaotically)
    p = newton.solve(pr.mesh, pr.kappa_kind, 0.5 * pr.kappa_a, pr.f_cell, pr.g_face)[0]
    p = p + 0.05 * np.random.default_rng(31).uniform(-1, 1, pr.mesh.n_cells)
    A = newton.picard_matrix(pr.mesh, pr.kappa_kind, pr.kappa_a, p)
    R = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.f_cell, pr.g_face)
    return pr, H, ctx, p, A, R


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _scaled_res(A, dx, R):
    S = 1.0 / np.sqrt(A.diagonal())
    return np.linalg.norm(S * (A @ dx + R)) / np.linalg.norm(S * R)


# (label, options, relative tolerance of the iterate against the FP64 oracle)
FINE_VARIANTS = [
    ("fp64_pipelined_registers", dict(lin_precision=0, max_sms=0, lin_tol=1e-6), 1e-10),
    ("fp64_pipelined_memory", dict(lin_precision=0, max_sms=1, lin_tol=1e-6), 1e-10),
    ("fp64_two_barrier", dict(lin_precision=0, max_sms=0, lin_tol=1e-8), 1e-10),
    ("fp32_pipelined_replacement", dict(lin_precision=1, max_sms=0, lin_tol=1e-6), 2e-4),
    ("fp32_two_barrier", dict(lin_precision=1, max_sms=1, lin_tol=1e-6), 2e-4),
]


@pytest.mark.parametrize("label,o,tol", FINE_VARIANTS, ids=[v[0] for v in FINE_VARIANTS])
@pytest.mark.parametrize("k", [7, 60])
def test_fine_cg_variants_follow_the_oracle_step_for_step(setup, label, o, tol, k):
    """k steps of each level-0 CG variant equal k steps of Jacobi-preconditioned CG on the oracle's frozen TPFA
    matrix (k = 60 passes the FP32 variant's residual replacement at step 50)."""
    pr, H, ctx, p, A, R = setup
    ctx.set_options(lin_maxit=k, **o)
    dx, it = ctx.picard_update(0, p)
    ref, it_ref = krylov.jacobi_pcg(A, -R, k)
    assert it == it_ref == k
    # FP32 recurrences drift from the FP64 iterate with the step count (and the replacement at step 50 restarts them
    # from the FP32-rounded true residual): 150x the 7-step bound at 60 steps (FP32 unit roundoff 6e-8 times the
    # scaled matrix's condition number, about 1e5 here)
    assert _rel(dx, ref) <= tol * (150 if (k == 60 and tol > 1e-8) else 1), label


@pytest.mark.parametrize("label,o,tol", FINE_VARIANTS[:2] + FINE_VARIANTS[3:4], ids=["fp64_reg", "fp64_mem", "fp32"])
def test_fine_cg_at_the_solver_tolerance(setup, label, o, tol):
    """At the library's level-0 tolerance (1e-2 of the scaled residual) the FP64 variants stop at the oracle's step
    with the oracle's iterate; every variant's update meets ||S (A dx + R)|| <= 1e-2 ||S R|| on the oracle's matrix
    (S = diag(A)^-1/2), up to the FP32 rounding of the FP32 one."""
    pr, H, ctx, p, A, R = setup
    ctx.set_options(**dict(o, lin_tol=1e-2, lin_maxit=5000))
    dx, it = ctx.picard_update(0, p)
    ref, it_ref = krylov.jacobi_pcg(A, -R, 5000, tol=1e-2)
    if o["lin_precision"] == 0:
        assert it == it_ref
        assert _rel(dx, ref) <= 1e-9
        assert _scaled_res(A, dx, R) <= 1e-2 * (1 + 1e-6)
    else:
        assert abs(it - it_ref) <= max(2, it_ref // 10)
        assert _scaled_res(A, dx, R) <= 1.05e-2


@pytest.mark.parametrize("k", [6, 25])
def test_newton_bicgstab_follows_the_oracle_step_for_step(setup, k):
    """k steps of the level-0 Newton BiCGStab equal k steps of BiCGStab on the oracle's exact Jacobian, scaled with
    the nonlinear Jacobi weights 1 / max(J_KK, d_K / 2)."""
    pr, H, ctx, p, A, R = setup
    ctx.set_options(lin_precision=0, max_sms=0, newton_lin_tol=1e-12, lin_maxit=k)
    dx, it = ctx.newton_update(p)
    J = tpfa.reduced_jacobian(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.g_face)
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, pr.opts)
    w = 1.0 / S.jacobi_diag(p)
    ref, it_ref = krylov.bicgstab_scaled(J, -R, w, k)
    assert it == it_ref == k
    assert _rel(dx, ref) <= (1e-9 if k <= 6 else 1e-6)


def test_newton_bicgstab_at_the_solver_tolerance(setup):
    pr, H, ctx, p, A, R = setup
    ctx.set_options(lin_precision=0, max_sms=0, newton_lin_tol=1e-2, lin_maxit=5000)
    dx, it = ctx.newton_update(p)
    J = tpfa.reduced_jacobian(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.g_face)
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, pr.opts)
    w = 1.0 / S.jacobi_diag(p)
    ref, it_ref = krylov.bicgstab_scaled(J, -R, w, 5000, tol=1e-2)
    # BiCGStab amplifies rounding differences over many steps: the step count within a few of the oracle's, and the
    # update meets the tolerance on the oracle's Jacobian (the recursive residual tracks the true one to ~1e-3 of it)
    assert abs(it - it_ref) <= max(3, it_ref // 10), (it, it_ref)
    sw = np.sqrt(w)
    assert np.linalg.norm(sw * (J @ dx + R)) <= 1.05e-2 * np.linalg.norm(sw * R)


def _coarse_problem(H, l, seed):
    lev = H.levels[l]
    rng = np.random.default_rng(seed)
    x = rng.uniform(-0.5, 0.5, lev.n_flux + lev.n_p)
    b = rng.uniform(-1, 1, lev.n_flux + lev.n_p)
    return lev, x, b


COARSE_VARIANTS = [
    ("pipelined_registers", dict(max_sms=0), 1e-6),
    ("pipelined_memory", dict(max_sms=1), 1e-6),
    ("two_synchronisation", dict(max_sms=0), 1e-9),
]


@pytest.mark.parametrize("label,o,ctol", COARSE_VARIANTS, ids=[v[0] for v in COARSE_VARIANTS])
@pytest.mark.parametrize("k", [5, 14])
def test_coarse_hybridized_cg_follows_the_oracle_step_for_step(setup, label, o, ctol, k):
    """k steps of the fused coarse step's hybridized CG equal k steps of Jacobi-preconditioned CG on the oracle's
    hybridized system H lambda = xi, recovered cell by cell (eq. hybridized-system), on both coarse levels."""
    pr, H, ctx, p, A, R = setup
    ctx.set_options(coarse_lin_tol=ctol, coarsest_lin_tol=ctol, lin_maxit=k, **o)
    for l in (1, 2):
        lev, x, b = _coarse_problem(H, l, 40 + l)
        nf = lev.n_flux
        dx, it = ctx.picard_update(l, x, b)
        r = coarse.operator(lev, pr.kappa_kind, pr.kappa_a, x[:nf], x[nf:]) - b
        ref, it_ref = krylov.hybridized(lev, pr.kappa_kind, pr.kappa_a, x[:nf], x[nf:], -r, k=k)
        assert it == it_ref == k, (label, l)
        assert _rel(dx, ref) <= 1e-9, (label, l)


@pytest.mark.parametrize("label,o", [("registers", dict(max_sms=0)), ("memory", dict(max_sms=1))])
def test_coarse_hybridized_cg_at_the_solver_tolerances(setup, label, o):
    """At the library's coarse tolerances (1e-1 on level 1, 2e-1 on the coarsest level) the pipelined hybridized CG
    stops at the oracle's step with the oracle's iterate."""
    pr, H, ctx, p, A, R = setup
    ctx.set_options(coarse_lin_tol=1e-1, coarsest_lin_tol=2e-1, lin_maxit=5000, **o)
    for l, t in ((1, 1e-1), (2, 2e-1)):
        lev, x, b = _coarse_problem(H, l, 50 + l)
        nf = lev.n_flux
        dx, it = ctx.picard_update(l, x, b)
        r = coarse.operator(lev, pr.kappa_kind, pr.kappa_a, x[:nf], x[nf:]) - b
        ref, it_ref = krylov.hybridized(lev, pr.kappa_kind, pr.kappa_a, x[:nf], x[nf:], -r, k=5000, tol=t)
        assert it == it_ref, (label, l)
        assert _rel(dx, ref) <= 1e-9, (label, l)


def test_memory_resident_coarse_variant_is_reachable(setup):
    """The memory-resident pipelined form needs more lambdas on level 1 than one SM's lanes (2 x 512)."""
    pr, H, ctx, p, A, R = setup
    lev = H.levels[1]
    shared = int(np.sum(lev.flux_owner[:, 1] >= 0))
    assert shared > 1024
