"""Pins of the oracle's fixed-length Krylov iterations and of its hybridized coarse solve (Sec. 3.4)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import coarse, fas, hierarchy, krylov, newton, tpfa
from synth.grids import problem_config


def _orth(K):
    Q, R = np.linalg.qr(K)
    keep = np.abs(np.diag(R)) > 1e-12 * np.abs(R).max()
    return Q[:, keep]


def _krylov(A, v, k):
    cols = [v / np.linalg.norm(v)]
    for _ in range(k - 1):
        w = A @ cols[-1]
        cols.append(w / np.linalg.norm(w))
    return _orth(np.stack(cols, 1))


@pytest.fixture(scope="module")
def tpfa_system():
    pr = problem_config("chan3d_64", scale=5)
    rng = np.random.default_rng(4)
    p = rng.uniform(0, 1, pr.mesh.n_cells)
    A = newton.picard_matrix(pr.mesh, pr.kappa_kind, pr.kappa_a, p)
    R = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.f_cell, pr.g_face)
    J = tpfa.reduced_jacobian(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.g_face)
    S = fas.FAS(hierarchy.Hierarchy([hierarchy.level0(pr.mesh)], []), pr.mesh, pr.kappa_kind, pr.kappa_a,
                pr.f_cell, pr.g_face, pr.opts)
    return pr, p, A, R, J, 1.0 / S.jacobi_diag(p)


@pytest.mark.parametrize("k", [1, 4, 9])
def test_pcg_iterate_is_the_krylov_galerkin_projection(tpfa_system, k):
    """CG's k-th iterate from zero minimises the energy error over the k-dimensional Krylov space: with S A S and S b
    (S = diag(A)^-1/2), y_k = V (V^T S A S V)^-1 V^T S b for any basis V of K_k(S A S, S b)."""
    pr, p, A, R, J, w = tpfa_system
    dx, it = krylov.jacobi_pcg(A, -R, k)
    assert it == k
    S = 1.0 / np.sqrt(A.diagonal())
    As = (sp.diags(S) @ A @ sp.diags(S)).toarray()
    bs = -S * R
    V = _krylov(As, bs, k)
    y = V @ np.linalg.solve(V.T @ As @ V, V.T @ bs)
    assert np.allclose(dx, S * y, rtol=0, atol=1e-10 * np.abs(S * y).max())


def test_pcg_converges_to_the_direct_solution(tpfa_system):
    pr, p, A, R, J, w = tpfa_system
    dx, _ = krylov.jacobi_pcg(A, -R, 400)
    ref = -spla.spsolve(A.tocsc(), R)
    assert np.allclose(dx, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_bicgstab_iterates_lie_in_the_krylov_space_and_converge(tpfa_system):
    """BiCGStab's k-th iterate lies in K_2k(S J S, S b) (each step applies the operator twice); run long enough it
    reaches the direct solution of the non-symmetric Newton system."""
    pr, p, A, R, J, w = tpfa_system
    S = np.sqrt(w)
    Js = (sp.diags(S) @ J @ sp.diags(S)).toarray()
    bs = -S * R
    for k in (1, 2, 3):
        dx, it = krylov.bicgstab_scaled(J, -R, w, k)
        assert it == k
        y = dx / S
        V = _krylov(Js, bs, 2 * k)
        assert np.linalg.norm(y - V @ (V.T @ y)) <= 1e-9 * np.linalg.norm(y)
        V1 = _krylov(Js, bs, 2 * k - 1)
        assert np.linalg.norm(y - V1 @ (V1.T @ y)) > 1e-6 * np.linalg.norm(y)   # and uses all of it
    dx, _ = krylov.bicgstab_scaled(J, -R, w, 300)
    ref = -spla.spsolve(J.tocsc(), R)
    assert np.allclose(dx, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


@pytest.fixture(scope="module", params=["cart2d", "chan3d", "chan3d_mf3"])
def coarse_case(request):
    if request.param == "cart2d":
        pr = problem_config("cart2d_32", scale=16)
        opts = dict(pr.opts, n_levels=3, agg_size=[16, 4], modes=[3, 2])
    else:
        pr = problem_config("chan3d_64", scale=8)
        opts = dict(pr.opts, agg_size=[16, 4, 4], modes=[3, 3, 3])
        if request.param.endswith("mf3"):
            opts["flux_modes"] = [3, 3, 3]
    return pr, hierarchy.build(pr.mesh, opts)


def test_hybridized_solve_equals_the_direct_saddle_solve(coarse_case):
    """eqs. hybridized-block-system / hybridized-system: eliminating the broken fluxes and solving H lambda = xi
    exactly, then recovering cell by cell, gives the solution of the frozen saddle (sparse LU of the full system)."""
    pr, Hh = coarse_case
    rng = np.random.default_rng(8)
    for l in range(1, len(Hh.levels)):
        lev = Hh.levels[l]
        x = rng.uniform(-0.5, 0.5, lev.n_flux + lev.n_p)
        b = rng.uniform(-1, 1, lev.n_flux + lev.n_p)
        r = coarse.operator(lev, pr.kappa_kind, pr.kappa_a, x[:lev.n_flux], x[lev.n_flux:]) - b
        dx, _ = krylov.hybridized(lev, pr.kappa_kind, pr.kappa_a, x[:lev.n_flux], x[lev.n_flux:], -r)
        sP, pP = coarse.picard_solve(lev, pr.kappa_kind, pr.kappa_a, x[:lev.n_flux], x[lev.n_flux:], b)
        ref = np.concatenate([sP, pP]) - x
        assert np.allclose(dx, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
        # CG on H run for many steps reaches the same solution
        dk, it = krylov.hybridized(lev, pr.kappa_kind, pr.kappa_a, x[:lev.n_flux], x[lev.n_flux:], -r, k=2000)
        assert np.allclose(dk, ref, rtol=0, atol=1e-8 * np.abs(ref).max())


def test_hybridized_iterate_moves_with_its_step_count(coarse_case):
    """A truncated solve is not the exact one, and each CG step on H changes it: the step count is honoured."""
    pr, Hh = coarse_case
    lev = Hh.levels[1]
    rng = np.random.default_rng(9)
    x = rng.uniform(-0.5, 0.5, lev.n_flux + lev.n_p)
    r = rng.uniform(-1, 1, lev.n_flux + lev.n_p)
    ex, _ = krylov.hybridized(lev, pr.kappa_kind, pr.kappa_a, x[:lev.n_flux], x[lev.n_flux:], r)
    prev = None
    for k in (1, 2, 3):
        dk, it = krylov.hybridized(lev, pr.kappa_kind, pr.kappa_a, x[:lev.n_flux], x[lev.n_flux:], r, k=k)
        assert it == k
        assert np.linalg.norm(dk - ex) > 1e-8 * np.linalg.norm(ex)
        if prev is not None:
            assert np.linalg.norm(dk - prev) > 1e-8 * np.linalg.norm(ex)
        prev = dk
