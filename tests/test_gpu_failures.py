"""Failure detection and reporting, made on the host or by a bounded wait, never by a GPU fault.

  * data that are not finite end a solve with NLMG_EDIVERGED;
  * a solve that runs out of cycles ends with NLMG_ENOCONV and still returns its last iterate;
  * polling a request that is still running returns NLMG_ETIMEOUT at once;
  * every grid-wide wait of the persistent kernels is bounded: the barrier, run alone with one block that never
    arrives and a short spin limit, returns NLMG_ETIMEOUT, and the same context then solves normally;
  * the request loop's admission estimate covers the device memory a context really holds.
"""
import numpy as np
import pytest

from synth.grids import cartesian_mesh, lognormal_field, problem_config

pytestmark = pytest.mark.gpu


def _ctx(nlmg_lib, scale=16, **upd):
    pr = problem_config("cart2d_32", scale=scale)
    return pr, nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, dict(pr.opts, **upd))


@pytest.mark.parametrize("where", ["source", "boundary"])
def test_non_finite_data_report_diverged(nlmg_lib, where):
    pr, ctx = _ctx(nlmg_lib)
    f, g = pr.f_cell.copy(), pr.g_face.copy()
    if where == "source":
        f[17] = np.nan
    else:
        g[np.where(pr.mesh.face_bc == 1)[0][3]] = np.inf
    with pytest.raises(nlmg_lib.NlmgError) as e:
        ctx.solve(f, g)
    assert e.value.status == nlmg_lib.EDIVERGED
    # the context is still usable
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face)
    assert st == nlmg_lib.OK


def test_cycle_limit_reports_noconv_with_the_last_iterate(nlmg_lib):
    """max_cycles = 1: NLMG_ENOCONV, and the returned iterate is the one cycle from the start (Algorithm 2 once)."""
    pr = problem_config("chan3d_64", scale=16)
    opts = dict(pr.opts, n_levels=3, agg_size=[64, 8, 8], modes=[4, 4, 4])
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, opts)
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face, max_cycles=1, allow_noconv=True)
    assert st == nlmg_lib.ENOCONV and rep["cycles"] == 1
    assert rep["res"] > 1e-8 * rep["res0"]
    ctx.set_data(pr.f_cell, pr.g_face)
    p1, r1, _ = ctx.vcycle(np.zeros(pr.mesh.n_cells), rep["res0"])
    assert np.array_equal(p, p1)
    assert abs(r1 - rep["res"]) <= 1e-12 * rep["res0"]


def test_poll_of_a_running_request_times_out(nlmg_lib):
    srv = nlmg_lib.Server(max_inflight=1, mem_budget_bytes=4 << 30, setup_threads_per_request=1, hierarchy_cache=0)
    n = 40
    mesh = cartesian_mesh((n, n, n), lognormal_field((n, n, n), 1.0, 4.0, seed=4))
    g = np.where(mesh.face_bc == 1, np.where(mesh.face_cells[:, 0] % n == 0, 1.0, 0.0), 0.0)
    opts = dict(problem_config("chan3d_64").opts)
    t = srv.submit(mesh, 0, 1.0, opts, np.zeros(mesh.n_cells), g)
    assert srv.poll(t, wait_ms=0) is None          # host setup of 64,000 cells alone takes far longer
    res = srv.poll(t, wait_ms=120000)
    assert res is not None and res[3] == nlmg_lib.OK
    srv.close()


def test_bounded_grid_barrier_gives_up_and_the_context_recovers(nlmg_lib):
    pr, ctx = _ctx(nlmg_lib)
    st, passed = ctx.check_grid_barrier(4, -1, 1 << 16)
    assert st == nlmg_lib.OK and passed == 4
    st, passed = ctx.check_grid_barrier(4, 2, 1 << 16)   # block 2 never arrives: ~2 ms of polling, then give up
    assert st == nlmg_lib.ETIMEOUT and passed == 0
    assert "gave up" in ctx.last_error()
    p, rep, st = ctx.solve(pr.f_cell, pr.g_face)
    assert st == nlmg_lib.OK and rep["res"] <= 1e-8 * rep["res0"]


@pytest.mark.parametrize("shape", [(64, 64), (128, 128), (16, 16, 16), (40, 40, 40), (64, 64, 64)])
def test_admission_estimate_covers_a_contexts_device_memory(nlmg_lib, shape):
    """The serving requests' meshes (2D and 3D, 4k to 262k cells): after a solve with Picard-then-Newton smoothing
    (which allocates the Newton buffers) the shared and own device bytes of the context stay within the estimate."""
    n = int(np.prod(shape))
    mesh = cartesian_mesh(shape, lognormal_field(shape, 1.0, 4.0, seed=7))
    g = np.where(mesh.face_bc == 1, np.where(mesh.face_cells[:, 0] % shape[0] == 0, 1.0, 0.0), 0.0)
    opts = dict(problem_config("chan3d_64").opts, smoother="picard_newton")
    if len(shape) == 2:
        opts.update(agg_size=[16, 8, 8], modes=[4, 4, 4])
    ctx = nlmg_lib.Context(mesh, 0, 1.5, opts)
    p, rep, st = ctx.solve(np.zeros(n), g)
    assert st == nlmg_lib.OK
    shared, own = ctx.device_bytes()
    est = nlmg_lib.request_bytes(mesh)
    assert shared > 0 and own > 0
    assert shared + own <= est, (shared, own, est)
    assert est <= 4 * (shared + own), (shared, own, est)      # and not so loose that it starves the loop
