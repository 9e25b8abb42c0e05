"""Pins of the oracle's coarse-level Newton linearization (Sec. 3.3.2, Props. 2-3) against what the mathematics fixes:

  * Prop. 2: M(Pi~ p) sigma equals N(sigma) kappa_inv(Pi~ p) for any sigma, p (the product decomposition);
  * the Jacobian J(x) applied to a direction v equals the central difference of the coarse operator
    (A(x + h v) - A(x - h v)) / 2h to the difference's truncation error, for every nonlinearity kind, on 2D, 3D and
    unstructured hierarchies and on the first and second coarse levels;
  * a pressure-independent coefficient (kappa = exp(0 p) = 1) leaves the Picard saddle [M D^T; D 0] (the N(sigma)
    term vanishes);
  * Newton's method on a coarse problem with a known solution converges quadratically;
  * FAS with Newton smoothing on the coarse levels reaches the fine discrete solution p* (brute-force Newton).
A dropped term of Prop. 3 (the N(sigma) product, or D^T), a wrong sign of d kappa_inv, a transposed Pi~ or a wrong
cell in N fails the finite-difference pin; the FAS test needs the whole step to be a descent direction.
"""
import numpy as np
import pytest

from oracle import coarse, fas, hierarchy, newton, tpfa
from synth.grids import problem_config, voronoi_problem


def _hierarchy(name, scale):
    pr = voronoi_problem(scale) if name == "voronoi" else problem_config(name, scale=scale)
    opts = dict(pr.opts)
    if name == "chan3d_64":
        opts.update(n_levels=3, agg_size=[16, 4, 4], modes=[3, 3, 3])
    if name == "cart2d_32":
        opts.update(n_levels=3, agg_size=[16, 4, 4], modes=[2, 2, 2])
    if name == "voronoi":
        opts.update(n_levels=3)
    pr.opts = opts
    return pr, hierarchy.build(pr.mesh, opts)


CASES = [("cart2d_32", 16), ("chan3d_64", 8), ("voronoi", 6)]
KINDS = [(tpfa.KAPPA_EXP, 1.5), (tpfa.KAPPA_INV1P2, 0.0)]


def _state(lev, rng):
    return rng.uniform(-1, 1, lev.n_flux), rng.uniform(0, 1, lev.n_p)


@pytest.mark.parametrize("name,scale", CASES, ids=[c[0] for c in CASES])
def test_product_decomposition(name, scale):
    """Prop. 2: M(Pi~ p) sigma = N(sigma) kappa_inv(Pi~ p), with M assembled cell by cell (Prop. 1)."""
    pr, H = _hierarchy(name, scale)
    rng = np.random.default_rng(3)
    for l in range(1, len(H.levels)):
        lev = H.levels[l]
        s, p = _state(lev, rng)
        for kind, a in KINDS:
            kinv = 1.0 / tpfa.kappa(coarse.pbar(lev, p), kind, a)
            lhs = hierarchy.assemble_M(lev, kinv) @ s
            rhs = coarse.n_matrix(lev, s) @ kinv
            assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(lhs), (name, l, kind)
        assert np.allclose(coarse.pi_matrix(lev) @ p, coarse.pbar(lev, p), rtol=1e-14, atol=0.0)


@pytest.mark.parametrize("name,scale", CASES, ids=[c[0] for c in CASES])
def test_jacobian_matches_central_differences(name, scale):
    """J(x) v = (A(x + h v) - A(x - h v)) / 2h + O(h^2), every kind, levels 1 and 2."""
    pr, H = _hierarchy(name, scale)
    rng = np.random.default_rng(5)
    for l in range(1, len(H.levels)):
        lev = H.levels[l]
        nf = lev.n_flux
        for kind, a in KINDS:
            s, p = _state(lev, rng)
            x = np.concatenate([s, p])
            v = rng.uniform(-1, 1, x.size)
            J = coarse.jacobian(lev, kind, a, s, p)
            jv = J @ v
            h = 1e-5
            xp, xm = x + h * v, x - h * v
            fd = (coarse.operator(lev, kind, a, xp[:nf], xp[nf:]) - coarse.operator(lev, kind, a, xm[:nf], xm[nf:]))
            fd /= 2.0 * h
            assert np.linalg.norm(jv - fd) <= 1e-7 * np.linalg.norm(jv), (name, l, kind)
            # the pressure columns alone (the N(sigma) term of Prop. 3 lives there)
            vp = np.concatenate([np.zeros(nf), v[nf:]])
            xp, xm = x + h * vp, x - h * vp
            fdp = (coarse.operator(lev, kind, a, xp[:nf], xp[nf:]) - coarse.operator(lev, kind, a, xm[:nf], xm[nf:]))
            fdp /= 2.0 * h
            jp = J @ vp
            assert np.linalg.norm(jp - fdp) <= 1e-7 * np.linalg.norm(jp), (name, l, kind)
            D = hierarchy.assemble_D(lev)
            assert np.linalg.norm(jp[:nf] - D.T @ v[nf:]) > 1e-6 * np.linalg.norm(jp[:nf])   # N term present


def test_constant_coefficient_gives_the_picard_saddle():
    """kappa = exp(0 p) = 1: d kappa_inv / d pbar = 0, so J = [M D^T; D 0] with the static M."""
    pr, H = _hierarchy("chan3d_64", 8)
    lev = H.levels[1]
    rng = np.random.default_rng(7)
    s, p = _state(lev, rng)
    J = coarse.jacobian(lev, tpfa.KAPPA_EXP, 0.0, s, p).toarray()
    M = hierarchy.assemble_M(lev).toarray()
    D = hierarchy.assemble_D(lev).toarray()
    ref = np.block([[M, D.T], [D, np.zeros((lev.n_p, lev.n_p))]])
    assert np.array_equal(J, ref)


def test_newton_converges_quadratically_on_a_coarse_problem():
    """A(x) = b with b = A(x*), x* = (sigma*, p*) a flux-consistent state (M(Pi~ p*) sigma* = -D^T p*, p* random):
    from a start near x*, the residual and the error fall quadratically to rounding."""
    import scipy.sparse.linalg as spla
    pr, H = _hierarchy("chan3d_64", 8)
    lev = H.levels[1]
    nf = lev.n_flux
    kind, a = tpfa.KAPPA_EXP, 2.0
    rng = np.random.default_rng(11)
    ps = rng.uniform(0, 1, lev.n_p)
    kinv = 1.0 / tpfa.kappa(coarse.pbar(lev, ps), kind, a)
    ss = spla.spsolve(hierarchy.assemble_M(lev, kinv).tocsc(), -(hierarchy.assemble_D(lev).T @ ps))
    xs = np.concatenate([ss, ps])
    b = coarse.operator(lev, kind, a, ss, ps)
    x = xs + 0.01 * np.abs(xs).mean() * rng.uniform(-1, 1, xs.size)
    err = []
    for _ in range(4):
        err.append(float(np.linalg.norm(x - xs)))
        x = x + coarse.newton_update(lev, kind, a, x[:nf], x[nf:], b)
    err.append(float(np.linalg.norm(x - xs)))
    nx = np.linalg.norm(xs)
    assert err[-1] <= 1e-12 * nx, err
    # quadratic: e_{k+1} <= C e_k^2 with a modest C while the error is above rounding (a linear rate rho would need
    # C ~ rho / e_k, growing without bound as e_k falls)
    ks = [k for k in range(len(err) - 1) if err[k + 1] > 1e-12 * nx]
    assert len(ks) >= 2, err
    assert max(err[k + 1] / err[k] ** 2 for k in ks) <= 10.0, err
    assert err[2] <= 1e-3 * err[1], err


@pytest.mark.parametrize("name,scale,cs", [("cart2d_32", 16, "newton"), ("voronoi", 6, "newton"),
                                           ("chan3d_64", 8, "picard_newton"), ("cart2d_32", 16, "picard_newton")])
def test_fas_with_coarse_newton_reaches_the_newton_solution(name, scale, cs):
    """FAS with Newton smoothing on the coarse levels (level 0 Picard-then-Newton): p* to 1e-10 at relative residual
    1e-12. "newton": Newton on every coarse level from the first cycle; "picard_newton": once the level-0 smoother has
    switched to Newton. (From p = 0 on the strongly nonlinear channelized case, Newton on the coarse levels from the
    first cycle stalls, like single-level Newton there.)"""
    pr, H = _hierarchy(name, scale)
    opts = dict(pr.opts, smoother="picard_newton", coarse_smoother=cs, tol_rel=1e-12, tol_abs=1e-300,
                max_cycles=40)
    pstar, _ = newton.solve(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, dp_clamp=opts["dp_clamp"])
    S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, opts)
    p = S.solve()
    h = S.stats.history
    assert h[-1] <= 1e-12 * h[0], h
    assert np.linalg.norm(p - pstar) <= 1e-10 * np.linalg.norm(pstar)
    assert S.stats.coarse_newton_steps > 0
