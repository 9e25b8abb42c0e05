"""Pins of the oracle's multigrid preconditioner for the level-0 Krylov solves (oracle/precond.py) to facts fixed
outside it: the Chebyshev polynomial's closed form, the two-level identity when the coarse space is everything,
symmetry and positive definiteness of the cycle, and CG convergence to the direct solution."""
from types import SimpleNamespace

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from numpy.polynomial import chebyshev as npcheb

from oracle import hierarchy, krylov, newton, precond, tpfa
from synth.grids import problem_config


def test_chebyshev_steps_are_the_scaled_chebyshev_polynomial():
    """For A = diag(lam_i) with D = I, k steps from x = 0 leave the error p_k(A) e_0 with
    p_k(t) = T_k((theta - t) / delta) / T_k(theta / delta) on [lmin, lmax] (textbook Chebyshev iteration), so
    x_i = (1 - p_k(lam_i)) b_i / lam_i."""
    lam = np.linspace(0.05, 2.0, 40)
    A = sp.diags(lam).tocsr()
    lv = precond.MGLevel(A, sp.identity(lam.size, format="csr"), 2.0)
    b = np.random.default_rng(1).uniform(-1, 1, lam.size)
    lmax, lmin = 2.0, 2.0 / precond.ALPHA
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    for k in (1, 2, 3, 5):
        x = precond.chebyshev(lv, b, np.zeros(lam.size), k)
        Tk = npcheb.Chebyshev.basis(k)
        p = Tk((theta - lam) / delta) / Tk(theta / delta)
        assert np.allclose(x, (1.0 - p) * b / lam, rtol=1e-12, atol=1e-14)


def test_full_coarse_space_makes_the_cycle_an_exact_solve():
    """With P = I the coarse correction solves the residual equation exactly and the post-smoothing sees a zero
    residual: one V-cycle is A^-1."""
    pr = problem_config("chan3d_64", scale=6)
    p = np.random.default_rng(2).uniform(0, 1, pr.mesh.n_cells)
    A = newton.picard_matrix(pr.mesh, pr.kappa_kind, pr.kappa_a, p).tocsr()
    n = A.shape[0]
    lev1 = SimpleNamespace(n_cells=n, p_off=np.arange(n + 1))
    H = SimpleNamespace(levels=[None, lev1], transfers=[SimpleNamespace(Pp=sp.identity(n, format="csr"))])
    lv = precond.build(A, H)
    b = np.random.default_rng(3).uniform(-1, 1, n)
    assert np.allclose(precond.vcycle(lv, H, b), spla.spsolve(A.tocsc(), b), rtol=1e-10, atol=1e-12)


@pytest.fixture(scope="module")
def case():
    pr = problem_config("chan3d_64", scale=12)
    opts = precond.extended_options(dict(pr.opts, n_levels=2, agg_size=[27, 8], modes=[4, 4]))
    H = hierarchy.build(pr.mesh, opts)
    L = precond.levels_for(H)
    assert 2 <= L <= len(H.levels)
    p = newton.solve(pr.mesh, pr.kappa_kind, 1.0, pr.f_cell, pr.g_face)[0]
    A = newton.picard_matrix(pr.mesh, pr.kappa_kind, pr.kappa_a, p).tocsr()
    R = tpfa.reduced_residual(pr.mesh, pr.kappa_kind, pr.kappa_a, p, pr.f_cell, pr.g_face)
    return pr, H, L, A, R


def test_cycle_is_symmetric_positive_definite(case):
    pr, H, L, A, R = case
    lv = precond.build(A, H, L)
    n = A.shape[0]
    B = np.stack([precond.vcycle(lv, H, e) for e in np.eye(n)], 1)
    assert np.abs(B - B.T).max() <= 1e-10 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0.0


def test_levels_stop_at_the_first_small_coarse_level(case):
    pr, H, L, A, R = case
    for l in range(1, L - 1):
        lev = H.levels[l]
        assert lev.n_cells * int(np.max(lev.m)) > precond.MAX_COARSE
    lev = H.levels[L - 1]
    assert lev.n_cells * int(np.max(lev.m)) <= precond.MAX_COARSE


def test_preconditioned_cg_reaches_the_direct_solution_in_few_steps(case):
    pr, H, L, A, R = case
    lv = precond.build(A, H, L)
    w = 1.0 / np.sqrt(A.diagonal())
    x, it = precond.pcg(A, -R, lambda r: precond.vcycle(lv, H, r), 500, tol=1e-12, w=w)
    ref = -spla.spsolve(A.tocsc(), R)
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
    _, it_mg = precond.pcg(A, -R, lambda r: precond.vcycle(lv, H, r), 500, tol=1e-2, w=w)
    _, it_j = krylov.jacobi_pcg(A, -R, 5000, tol=1e-2)
    assert it_mg * 3 <= it_j, (it_mg, it_j)
