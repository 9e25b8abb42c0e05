"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every declared symbol, and its host-side
hierarchy setup (aggregation, spectral bases, flux space) agrees with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import hierarchy
from synth.grids import problem_config, voronoi_problem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nlmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nlmg_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(nlmg_lib):
    import ctypes
    L = ctypes.CDLL(nlmg_lib.LIB_PATH)
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(nlmg_lib.SIGNATURES), set(names) ^ set(nlmg_lib.SIGNATURES)


def test_default_options_are_the_papers(nlmg_lib):
    o = nlmg_lib.default_options()
    assert o.bt_nmax == 4 and abs(o.bt_theta - 0.9) < 1e-15 and o.coarsest_steps == 10
    assert o.smoother == nlmg_lib.SMOOTH_PICARD and o.newton_switch == 1e-3 and o.newton_lin_tol == 1e-2
    assert o.coarse_lin_tol == 1e-1 and o.coarsest_lin_tol == 2e-1


def test_setup_rejects_bad_mesh(nlmg_lib):
    pr = problem_config("cart2d_32", scale=4)
    m = pr.mesh
    bad = m.face_cells.copy()
    bad[0] = bad[0][::-1]                  # K > L on an interior face
    m2 = type(m)(m.n_cells, m.cell_volume, bad, m.half_trans, m.face_bc, m.face_area, m.shape)
    with pytest.raises(nlmg_lib.NlmgError):
        nlmg_lib.Context(m2, pr.kappa_kind, pr.kappa_a, pr.opts, device=False)


CASES = [("cart2d_32", None, {}), ("cart2d_32", 13, dict(agg_size=[9, 4], modes=[3, 2])),
         ("chan3d_64", 8, dict(agg_size=[16, 4, 4], modes=[3, 3, 3])),
         ("chan3d_64", 12, dict(n_levels=3, agg_size=[27, 6, 4], modes=[4, 3, 3])),
         ("voronoi", 9, {}),
         ("cart2d_32", 13, dict(agg_size=[9, 4], modes=[3, 2], flux_modes=[3, 3])),
         ("chan3d_64", 12, dict(n_levels=3, agg_size=[27, 6, 4], modes=[4, 3, 3], flux_modes=[3, 2, 2])),
         ("voronoi", 9, dict(flux_modes=[2, 2]))]


@pytest.mark.parametrize("name,scale,upd", CASES)
def test_host_hierarchy_matches_oracle(nlmg_lib, name, scale, upd):
    pr = voronoi_problem(scale) if name == "voronoi" else problem_config(name, scale=scale)
    opts = dict(pr.opts, **upd)
    H = hierarchy.build(pr.mesh, opts)
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, opts, device=False)
    for l, tr in enumerate(H.transfers):
        agg, m = ctx.aggregates(l)
        assert np.array_equal(agg, tr.agg_of)                   # bit-exact aggregation
        assert np.array_equal(m, H.levels[l + 1].m)
        info = ctx.level_info(l + 1)
        assert info["n_flux"] == H.levels[l + 1].n_flux and info["n_p"] == H.levels[l + 1].n_p
        Pp, Ppo = ctx.transfer_dense(l, 0), tr.Pp.toarray()
        assert np.abs(Pp @ Pp.T - Ppo @ Ppo.T).max() < 1e-10
        gap = tr.extra["eig_gap"]
        assert np.all(gap[np.isfinite(gap)] > 1e-8)            # bases unique up to sign (C7 reading)
        Ps, Qs = ctx.transfer_dense(l, 1), ctx.transfer_dense(l, 2)
        scale_ = max(1.0, np.abs(tr.Psigma).max())
        assert np.abs(Ps - tr.Psigma.toarray()).max() < 1e-9 * scale_
        assert np.abs(Qs @ Ps - np.eye(Ps.shape[1])).max() < 1e-10
        assert np.abs(Qs - tr.Qsigma.toarray()).max() < 1e-9 * max(1.0, np.abs(tr.Qsigma).max())


def test_set_options_keeps_the_hierarchy_fixed(nlmg_lib):
    pr = problem_config("cart2d_32", scale=8)
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.opts, device=False)
    ctx.set_options(nu_pre=3, lin_tol=1e-4, lin_precision=1)
    assert ctx.opts.nu_pre == 3 and ctx.opts.lin_precision == 1
    ctx.set_options(smoother="picard_newton", newton_switch=1e-3)
    assert ctx.opts.smoother == nlmg_lib.SMOOTH_PICARD_NEWTON and ctx.opts.newton_switch == 1e-3
    ctx.set_options(cascadic=1)
    assert ctx.opts.cascadic == 1
    for bad in (dict(n_levels=3), dict(modes=(ctypes.c_int32 * 8)(3, 3, 3, 3, 3, 3, 3, 3)), dict(lin_precision=3),
                dict(omega=0.0), dict(smoother=3), dict(newton_switch=-1.0), dict(newton_switch=float("nan")),
                dict(newton_lin_tol=0.0), dict(flux_modes=(ctypes.c_int32 * 8)(2, 1, 1, 1, 1, 1, 1, 1)), dict(cascadic=2)):
        with pytest.raises(nlmg_lib.NlmgError):
            ctx.set_options(**bad)
    ctx.close()


def test_flux_modes_option_range(nlmg_lib):
    """m_f is a hierarchy option: 1..8 per coarsening step, checked at setup."""
    pr = problem_config("cart2d_32", scale=8)
    for bad in (0, 9):
        with pytest.raises(nlmg_lib.NlmgError):
            nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, dict(pr.opts, flux_modes=[bad] * 8), device=False)
    c1 = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.opts, device=False)
    c2 = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, dict(pr.opts, flux_modes=[2] * 8), device=False)
    assert c2.opts.flux_modes[0] == 2 and c1.opts.flux_modes[0] == 1
    assert c2.level_info(1)["n_flux"] > c1.level_info(1)["n_flux"]
    c1.close()
    c2.close()


def test_multigrid_preconditioner_option_builds_its_extra_levels(nlmg_lib):
    """lin_precond = 1 is a hierarchy option: the host setup coarsens beyond n_levels for the preconditioner alone
    (the exported FAS levels are unchanged) and rejects an unknown value."""
    pr = problem_config("chan3d_64", scale=12)
    opts = dict(pr.opts, n_levels=2, agg_size=[27, 8], modes=[4, 4])
    base = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, opts, device=False)
    mg = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, dict(opts, lin_precond=1), device=False)
    for l in range(2):
        assert base.level_info(l) == mg.level_info(l)
    with pytest.raises(nlmg_lib.NlmgError):
        mg.level_info(2)
    with pytest.raises(nlmg_lib.NlmgError):
        nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, dict(opts, lin_precond=2), device=False)
