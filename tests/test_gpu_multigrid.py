"""The multigrid-preconditioned level-0 Krylov solves (lin_precond = 1) against the oracle's preconditioner
(oracle/precond.py) and against the definitional solution p*.

The library builds the preconditioner on the FAS hierarchy extended for it (oracle.precond.extended_options) and cut
at the first level with at most 128 pressure unknowns (oracle.precond.levels_for); it runs in FP32 inside the FP64
Krylov iteration, so one application agrees with the oracle's FP64 V-cycle to FP32 accuracy, and the Krylov results
are checked by their residuals on the oracle's own matrices."""
import numpy as np
import pytest

from oracle import fas, hierarchy, newton, precond, tpfa
from synth.grids import problem_config, voronoi_problem

pytestmark = pytest.mark.gpu


def _case(nlmg_lib, name, scale, **upd):
    pr = voronoi_problem(scale) if name == "voronoi" else problem_config(name, scale=scale)
    opts = dict(pr.opts, lin_precond=1, **upd)
    pr.opts = opts
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, opts)
    ctx.set_data(pr.f_cell, pr.g_face)
    return pr, ctx


def _oracle_levels(pr, A):
    H = hierarchy.build(pr.mesh, precond.extended_options(pr.opts))
    L = precond.levels_for(H)
    return H, precond.build(A, H, L)


CASES = [("chan3d_64", 16, dict(n_levels=3, agg_size=[64, 8, 8], modes=[4, 4, 4])),
         ("cart2d_32", 32, {}),
         ("voronoi", 10, {})]


@pytest.mark.parametrize("name,scale,upd", CASES, ids=[c[0] for c in CASES])
def test_one_application_matches_the_oracle_vcycle(nlmg_lib, name, scale, upd):
    pr, ctx = _case(nlmg_lib, name, scale, **upd)
    rng = np.random.default_rng(61)
    p = rng.uniform(0, 1, pr.mesh.n_cells)
    A = newton.picard_matrix(pr.mesh, pr.kappa_kind, pr.kappa_a, p).tocsr()
    H, lv = _oracle_levels(pr, A)
    for _ in range(2):
        r = rng.uniform(-1, 1, pr.mesh.n_cells)
        z = ctx.precond_apply(p, r)
        ref = precond.vcycle(lv, H, r)
        assert np.linalg.norm(z - ref) <= 2e-4 * np.linalg.norm(ref), name


@pytest.mark.parametrize("name,scale,upd", CASES, ids=[c[0] for c in CASES])
def test_preconditioned_cg_update(nlmg_lib, name, scale, upd):
    """The Picard update by the multigrid-preconditioned CG meets ||S (A dx + R)|| <= tol ||S R|| on the oracle's
    matrix, in about as many steps as the oracle's preconditioned CG, and far fewer than Jacobi-preconditioned CG."""
    pr, ctx = _case(nlmg_lib, name, scale, **upd)
    p = np.random.default_rng(62).uniform(0, 1, pr.mesh.n_cells)
    A = newton.picard_matrix(pr.mesh, pr.kappa_kind, pr.kappa_a, p).tocsr()
    R = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.f_cell, pr.g_face)
    H, lv = _oracle_levels(pr, A)
    S = 1.0 / np.sqrt(A.diagonal())
    for tol in (1e-2, 1e-8):
        ctx.set_options(lin_tol=tol, lin_maxit=500)
        dx, it = ctx.picard_update(0, p)
        _, it_ref = precond.pcg(A, -R, lambda r: precond.vcycle(lv, H, r), 500, tol=tol, w=S)
        res = np.linalg.norm(S * (A @ dx + R)) / np.linalg.norm(S * R)
        assert res <= tol * (1 + 1e-6), (name, tol, res)
        assert abs(it - it_ref) <= 1 + it_ref // 10, (name, tol, it, it_ref)


@pytest.mark.parametrize("name,scale,upd", CASES, ids=[c[0] for c in CASES])
def test_row_parallel_block_levels(nlmg_lib, name, scale, upd):
    """mg_row_cells = 0: every block level outside the shared-memory tail runs the row-parallel smoothing and
    residual kernels (one thread per cell component). One application still equals the oracle's cycle, and the
    warp-per-cell form to FP32 rounding (only the order of the sums differs); the preconditioned CG update still
    meets its tolerance on the oracle's matrix, and a FAS solve reaches p*."""
    pr, ctx = _case(nlmg_lib, name, scale, **upd)
    rng = np.random.default_rng(65)
    p = rng.uniform(0, 1, pr.mesh.n_cells)
    A = newton.picard_matrix(pr.mesh, pr.kappa_kind, pr.kappa_a, p).tocsr()
    H, lv = _oracle_levels(pr, A)
    r = rng.uniform(-1, 1, pr.mesh.n_cells)
    z_warp = ctx.precond_apply(p, r)
    ctx.set_options(mg_row_cells=0)
    z_row = ctx.precond_apply(p, r)
    ref = precond.vcycle(lv, H, r)
    assert np.linalg.norm(z_row - ref) <= 2e-4 * np.linalg.norm(ref), name
    assert np.linalg.norm(z_row - z_warp) <= 1e-5 * np.linalg.norm(z_warp), name
    if name == "chan3d_64":   # level 1 (64 cells) runs its own kernels here: the other form really ran
        assert not np.array_equal(z_row, z_warp)
    R = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.f_cell, pr.g_face)
    S = 1.0 / np.sqrt(A.diagonal())
    ctx.set_options(mg_row_cells=0, lin_tol=1e-8, lin_maxit=500)
    dx, it = ctx.picard_update(0, p)
    assert np.linalg.norm(S * (A @ dx + R)) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(S * R), name
    ctx.set_options(mg_row_cells=0, smoother="picard_newton")
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dp_clamp=pr.opts["dp_clamp"])
    ps, rep, st = ctx.solve(pr.f_cell, pr.g_face, tol_rel=1e-12, tol_abs=1e-300, max_cycles=80)
    assert st == 0, (name, rep)
    assert np.linalg.norm(ps - pstar) <= 1e-10 * np.linalg.norm(pstar), name


def test_preconditioned_bicgstab_newton_update(nlmg_lib):
    pr, ctx = _case(nlmg_lib, "chan3d_64", 16, n_levels=3, agg_size=[64, 8, 8], modes=[4, 4, 4])
    # an iterate of the kind a solve meets (at random pressures the Jacobian is far from an M-matrix)
    p = newton.solve(pr.mesh, pr.kappa_kind, 0.5 * pr.kappa_a, pr.f_cell, pr.g_face)[0]
    p = p + 0.05 * np.random.default_rng(63).uniform(-1, 1, pr.mesh.n_cells)
    J = tpfa.reduced_jacobian(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.g_face)
    R = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.f_cell, pr.g_face)
    S = fas.FAS(hierarchy.Hierarchy([hierarchy.level0(pr.mesh)], []), pr.mesh, pr.kappa_kind, pr.kappa_a,
                pr.f_cell, pr.g_face, pr.opts)
    w = 1.0 / S.jacobi_diag(p)
    for tol in (1e-2, 1e-8):
        ctx.set_options(newton_lin_tol=tol, lin_maxit=500)
        dx, it = ctx.newton_update(p)
        res = np.linalg.norm(np.sqrt(w) * (J @ dx + R)) / np.linalg.norm(np.sqrt(w) * R)
        assert res <= tol * (1 + 1e-6), (tol, res)
        assert it <= 60


@pytest.mark.parametrize("name,scale,upd", CASES, ids=[c[0] for c in CASES])
def test_solves_reach_the_newton_solution(nlmg_lib, name, scale, upd):
    """FAS with the multigrid-preconditioned level-0 solves, Picard and Picard-then-Newton smoothing, to relative
    residual 1e-12: p* within 1e-10; two solves are bitwise equal."""
    pr, ctx = _case(nlmg_lib, name, scale, **upd)
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dp_clamp=pr.opts["dp_clamp"])
    for sm in ("picard", "picard_newton"):
        ctx.set_options(smoother=sm)
        p, rep, st = ctx.solve(pr.f_cell, pr.g_face, tol_rel=1e-12, tol_abs=1e-300, max_cycles=80)
        assert st == 0, (name, sm, rep)
        assert np.linalg.norm(p - pstar) <= 1e-10 * np.linalg.norm(pstar), (name, sm)
        r = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.f_cell, pr.g_face)
        assert np.linalg.norm(r) <= 2e-12 * rep["res0"]
        p2, rep2, _ = ctx.solve(pr.f_cell, pr.g_face, tol_rel=1e-12, tol_abs=1e-300, max_cycles=80)
        assert np.array_equal(p, p2)


def test_bench_workload_shape_with_the_preconditioner(nlmg_lib):
    """The benchmark's options with lin_precond = 1 on the 32^3 instance of its generator: p* within 1e-10 at
    relative residual 1e-12, and at 1e-8 far fewer level-0 Krylov steps than with Jacobi preconditioning."""
    pr = problem_config("chan3d_64", scale=32)
    opts = dict(pr.opts, smoother="picard_newton", lin_precond=1)
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, opts)
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dp_clamp=pr.opts["dp_clamp"])
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face, tol_rel=1e-12, tol_abs=1e-300, max_cycles=60)
    assert st == 0, rep
    assert np.linalg.norm(p - pstar) <= 1e-10 * np.linalg.norm(pstar)
    _, rep_mg, _ = ctx.solve(pr.f_cell, pr.g_face)
    jac = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, dict(pr.opts, smoother="picard_newton"))
    _, rep_j, _ = jac.solve(pr.f_cell, pr.g_face)
    assert rep_mg["lin_iters_level"][0] * 4 <= rep_j["lin_iters_level"][0], (rep_mg, rep_j)


def _bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_transfers(nlmg_lib):
    """lin_precision = 2: the V-cycle's transfers in BF16. One application equals the oracle's cycle built on the
    BF16-rounded P (same Galerkin operators), and FAS solves still reach p* to 1e-10 at relative residual 1e-12 (the
    Krylov iterations and every residual stay FP64)."""
    from types import SimpleNamespace
    import scipy.sparse as sp
    pr, ctx = _case(nlmg_lib, "chan3d_64", 16, n_levels=3, agg_size=[64, 8, 8], modes=[4, 4, 4])
    ctx.set_options(lin_precision=2)
    rng = np.random.default_rng(64)
    p = rng.uniform(0, 1, pr.mesh.n_cells)
    A = newton.picard_matrix(pr.mesh, pr.kappa_kind, pr.kappa_a, p).tocsr()
    H = hierarchy.build(pr.mesh, precond.extended_options(pr.opts))
    L = precond.levels_for(H)
    tr = [SimpleNamespace(Pp=sp.csr_matrix((_bf16(t.Pp.data), t.Pp.indices, t.Pp.indptr), shape=t.Pp.shape))
          for t in H.transfers]
    Hb = SimpleNamespace(levels=H.levels, transfers=tr)
    lv = precond.build(A, Hb, L)
    r = rng.uniform(-1, 1, pr.mesh.n_cells)
    z = ctx.precond_apply(p, r)
    ref = precond.vcycle(lv, Hb, r)
    assert np.linalg.norm(z - ref) <= 2e-4 * np.linalg.norm(ref)
    ref32 = precond.vcycle(precond.build(A, H, L), H, r)
    assert np.linalg.norm(z - ref32) > 1e-6 * np.linalg.norm(ref32)      # the rounding is really applied
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dp_clamp=pr.opts["dp_clamp"])
    pb, rep, st = ctx.solve(pr.f_cell, pr.g_face, tol_rel=1e-12, tol_abs=1e-300, max_cycles=80)
    assert st == 0, rep
    assert np.linalg.norm(pb - pstar) <= 1e-10 * np.linalg.norm(pstar)
