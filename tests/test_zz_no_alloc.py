"""The allocation-free residual entry point, for callers that cannot allocate device memory when they call (their
caching allocator already holds the memory they may use, a fixed device-memory budget, or loops that must not stall
other streams with cudaMalloc/cudaFree). It must return what nlmg_fine_residual returns.

This file is collected last on purpose: a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from synth.grids import cartesian_mesh, problem_config

pytestmark = pytest.mark.gpu


def _setup(nlmg_lib):
    pr = problem_config("chan3d_64", scale=12)
    opts = dict(pr.opts, n_levels=2, agg_size=[27, 8], modes=[4, 4])
    ctx = nlmg_lib.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, opts)
    ctx.set_data(pr.f_cell, pr.g_face)
    return pr, ctx


def test_noalloc_residual_matches_allocating_entry_point(nlmg_lib):
    torch = pytest.importorskip("torch")
    pr, ctx = _setup(nlmg_lib)
    n = pr.mesh.n_cells
    dev = torch.device("cuda", 0)
    r_d = torch.empty(n, dtype=torch.float64, device=dev)
    nrm_d = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    rng = np.random.default_rng(21)
    for call in range(2):                       # two calls in a row share (and reuse) the fixed scratch
        p = rng.uniform(-0.2, 1.1, n)
        p_d = torch.from_numpy(p).to(dev)
        torch.cuda.synchronize()
        st = ctx.fine_residual_noalloc(p_d.data_ptr(), r_d.data_ptr(), nrm_d.data_ptr(), stream.cuda_stream)
        assert st == nlmg_lib.OK, ctx.last_error()
        stream.synchronize()
        ref = ctx.fine_residual(p)
        got = r_d.cpu().numpy()
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-13 * scale, call
        assert abs(float(nrm_d.item()) - float(ref @ ref)) <= 1e-12 * float(ref @ ref), call


def test_noalloc_rejects_meshes_beyond_its_scratch(nlmg_lib):
    torch = pytest.importorskip("torch")
    n = (1 << 20) + 1                           # one cell more than the fixed scratch holds
    mesh = cartesian_mesh((n, 1), np.ones(n))
    ctx = nlmg_lib.Context(mesh, 0, 1.0, dict(problem_config("cart2d_32").opts, n_levels=1))
    ctx.set_data(np.zeros(n), np.zeros(mesh.n_faces))
    dev = torch.device("cuda", 0)
    buf = torch.zeros(n + 1, dtype=torch.float64, device=dev)
    st = ctx.fine_residual_noalloc(buf.data_ptr(), buf.data_ptr(), buf.data_ptr() + 8 * n, 0)
    assert st == nlmg_lib.EINVAL
    assert "1048576" in ctx.last_error()
