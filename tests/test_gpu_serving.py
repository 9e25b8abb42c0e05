"""The request loop: every result is the same alone and in a concurrent mix, admission respects the memory budget."""
import numpy as np
import pytest

from oracle import tpfa
from synth.grids import cartesian_mesh, lognormal_field, multi_rhs_rows, problem_config

pytestmark = pytest.mark.gpu


def _requests(n_req=6, seed=40):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_req):
        if i % 2 == 0:
            side = int(rng.integers(10, 24))
            shape = (side, side)
            opts = dict(problem_config("cart2d_32").opts, n_levels=2, agg_size=[16, 8], modes=[2, 2])
        else:
            side = int(rng.integers(6, 11))
            shape = (side, side, side)
            opts = dict(problem_config("chan3d_64").opts, n_levels=2, agg_size=[27, 8], modes=[3, 3])
        K = lognormal_field(shape, 1.0, 3.0, seed=100 + i)
        mesh = cartesian_mesh(shape, K)
        a = float(rng.uniform(0.5, 2.0))
        opts["dp_clamp"] = float(np.log(1.5) / a)
        g = np.zeros(mesh.n_faces)
        d = np.where(mesh.face_bc == 1)[0]
        g[d] = np.where(mesh.face_cells[d, 0] % shape[0] == 0, rng.uniform(0.5, 1.5), rng.uniform(-0.5, 0.5))
        out.append((mesh, a, opts, np.zeros(mesh.n_cells), g))
    return out


def test_results_identical_alone_and_in_the_mix(nlmg_lib):
    """Alone = a context of its own with the SM share the server gives each request (explicit here)."""
    reqs = [(m, a, dict(o, max_sms=50), f, g) for m, a, o, f, g in _requests()]
    alone = []
    for mesh, a, opts, f, g in reqs:
        ctx = nlmg_lib.Context(mesh, 0, a, opts)
        p, rep, st = ctx.solve(f, g, max_cycles=60)
        assert st == 0, rep
        alone.append(p)
        ctx.close()
    srv = nlmg_lib.Server(max_inflight=3, mem_budget_bytes=1 << 30)
    tickets = [srv.submit(mesh, 0, a, opts, f, g, max_cycles=60) for mesh, a, opts, f, g in reqs]
    for t, p_ref, (mesh, a, opts, f, g) in zip(tickets, alone, reqs):
        res = srv.poll(t, wait_ms=120000)
        assert res is not None
        p, rep, times, st = res
        assert st == 0
        assert np.array_equal(p, p_ref)                 # bitwise: fixed-order reductions, private buffers
        assert times["latency_ms"] >= times["solve_ms"] >= 0.0
        r = tpfa.reduced_residual(mesh, 0, a, p, f, g)
        assert np.linalg.norm(r) <= 1e-8 * rep["res0"] * 1.0001
    srv.close()


def test_admission_by_memory_and_oversized_request(nlmg_lib):
    reqs = _requests(3, seed=41)
    # a budget of the largest request's estimate: the requests fit one at a time
    budget = max(nlmg_lib.request_bytes(r[0]) for r in reqs)
    srv = nlmg_lib.Server(max_inflight=3, mem_budget_bytes=budget)
    tickets = [srv.submit(mesh, 0, a, opts, f, g) for mesh, a, opts, f, g in reqs]
    res = [srv.poll(t, wait_ms=120000) for t in tickets]
    assert all(r is not None and r[3] == 0 for r in res)
    mesh, a, opts, f, g = reqs[0]
    tiny = nlmg_lib.Server(max_inflight=1, mem_budget_bytes=1 << 10)
    with pytest.raises(nlmg_lib.NlmgError):
        tiny.submit(mesh, 0, a, opts, f, g)
    srv.close()
    tiny.close()


def test_kept_hierarchy_is_reused_with_identical_results(nlmg_lib):
    """Requests on one mesh with other nonlinearity parameters, data and clamps run on the kept hierarchy (no new
    setup) and return exactly what a fresh context returns."""
    pr = problem_config("chan3d_64", scale=9)
    base_opts = dict(pr.opts, n_levels=3, agg_size=[27, 6, 4], modes=[4, 3, 3])
    F, G = multi_rhs_rows(pr.mesh, 4, seed=60)
    alphas = [2.0, 1.0, 1.5, 0.75]
    reqs = [(a, dict(base_opts, dp_clamp=float(np.log(1.5) / a), max_sms=76), F[r], G[r])
            for r, a in enumerate(alphas)]
    alone = []
    for a, o, f, g in reqs:
        ctx = nlmg_lib.Context(pr.mesh, 0, a, o)
        p, rep, st = ctx.solve(f, g, max_cycles=60)
        assert st == 0
        alone.append(p)
        ctx.close()
    srv = nlmg_lib.Server(max_inflight=2, mem_budget_bytes=1 << 30, hierarchy_cache=2)
    a, o, f, g = reqs[0]
    p, rep, times, st = srv.poll(srv.submit(pr.mesh, 0, a, o, f, g), wait_ms=120000)
    assert st == 0 and not times["hierarchy_reused"] and np.array_equal(p, alone[0])
    tickets = [srv.submit(pr.mesh, 0, a, o, f, g) for a, o, f, g in reqs[1:]]
    for t, p_ref in zip(tickets, alone[1:]):
        p, rep, times, st = srv.poll(t, wait_ms=120000)
        assert st == 0 and times["hierarchy_reused"]
        assert np.array_equal(p, p_ref)
    srv.close()
    off = nlmg_lib.Server(max_inflight=1, mem_budget_bytes=1 << 30, hierarchy_cache=0)
    for a, o, f, g in reqs[:2]:
        p, rep, times, st = off.poll(off.submit(pr.mesh, 0, a, o, f, g), wait_ms=120000)
        assert st == 0 and not times["hierarchy_reused"]
    off.close()
