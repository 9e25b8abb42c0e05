"""Pins of the oracle's local problems of App. A.2 (sigma^PV, trace extensions, bubbles, coarse boundary traces) and
of the Neumann data term of [f] (definitions under eq. FV_matrix).

Every check restates a definition of the paper here and solves it again, with operators assembled without the
oracle's cell-by-cell data and with a sparse direct solver instead of the oracle's dense bordered solves:
  * level 0: M and D of eq. FV_matrix at kappa = 1 (oracle.tpfa.mixed_matrices, which assembles face by face);
  * level l+1: the explicit Galerkin products M^{l+1} = P_sigma^T M^l P_sigma and D^{l+1} = P_p^T D^l P_sigma
    (Sec. 3.1, App. C), built level by level from the level-0 matrices, and 1^{l+1} = Q_p 1^l;
  * restrictions to a set of cells keep the flux unknowns whose owners all lie in the set (the edges joining two
    of its vertices, and the bubbles of its cells), written out below from the unknowns' owners.
A wrong mass matrix, a wrong sign or scaling of a right-hand side, or a dropped term in any local solve changes the
columns of P_sigma and fails these tests, although the identities Q_sigma P_sigma = I and D Q_sigma = Q_p D hold for
any columns with the right net flux.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import hierarchy, newton, tpfa
from synth.grids import BC_DIRICHLET, BC_NEUMANN, KAPPA_EXP, cartesian_mesh, problem_config, voronoi_problem

IFACE, BDRY, BUBBLE = hierarchy.KIND_IFACE, hierarchy.KIND_BDRY, hierarchy.KIND_BUBBLE


def _independent_operators(mesh, Hh):
    """M^l, D^l and 1^l of every level without the oracle's per-cell matrices (module docstring)."""
    N, F = mesh.n_cells, mesh.n_faces
    M0, D0, _, _, dofs = tpfa.mixed_matrices(mesh, KAPPA_EXP, 0.0, np.zeros(N), np.zeros(N), np.zeros(F))
    assert np.array_equal(dofs, Hh.levels[0].face_ids)
    Ms, Ds, ones = [M0.tocsr()], [D0.tocsr()], [np.ones(N)]
    for tr in Hh.transfers:
        Ms.append((tr.Psigma.T @ Ms[-1] @ tr.Psigma).tocsr())
        Ds.append((tr.Pp.T @ Ds[-1] @ tr.Psigma).tocsr())
        ones.append(tr.Pp.T @ ones[-1])
    return Ms, Ds, ones


def _owners_and_kinds(mesh, Hh, l):
    """Owner cells (c, d or -1) and kind of every flux unknown of level l. Level 0 reads them off the mesh: interior
    faces join their two cells, Dirichlet faces belong to their one cell."""
    if l == 0:
        dofs = tpfa.flux_dofs(mesh)
        K = mesh.face_cells[dofs, 0].astype(np.int64)
        L = mesh.face_cells[dofs, 1].astype(np.int64)
        kind = np.where(mesh.face_bc[dofs] == BC_DIRICHLET, BDRY, IFACE)
        return np.stack([K, np.where(kind == IFACE, L, -1)], 1), kind
    lev = Hh.levels[l]
    return lev.flux_owner, lev.flux_kind


class _Level:
    """Index sets of level l for the restrictions of App. A.2."""

    def __init__(self, mesh, Hh, l, M, D, one):
        self.M, self.D, self.one = M, D, one
        self.own, self.kind = _owners_and_kinds(mesh, Hh, l)
        lev = Hh.levels[l]
        self.p_off = lev.p_off
        self.n_cells = lev.n_cells

    def pdofs(self, cells):
        return np.concatenate([np.arange(self.p_off[c], self.p_off[c + 1]) for c in cells])

    def inner(self, cells):
        """Flux unknowns with every owner in `cells`: interfaces joining two of its cells and bubbles of its cells."""
        ins = np.zeros(self.n_cells, bool)
        ins[cells] = True
        c0, c1 = self.own[:, 0], self.own[:, 1]
        iface = (self.kind == IFACE) & ins[c0] & (c1 >= 0) & ins[np.maximum(c1, 0)]
        bub = (self.kind == BUBBLE) & ins[c0]
        return np.where(iface | bub)[0]


def _sparse_saddle(M, D, rs, rp, null=None):
    """Solve [M D^T; D 0][s; p] = [rs; rp] with a sparse LU; `null` (a pressure null vector) borders the system with
    null^T p = 0. Returns s."""
    ns = M.shape[0]
    if null is None:
        K = sp.bmat([[M, D.T], [D, None]], format="csc")
        rhs = np.concatenate([rs, rp])
    else:
        n = sp.csr_matrix(null.reshape(-1, 1))
        K = sp.bmat([[M, D.T, None], [D, None, n], [None, n.T, None]], format="csc")
        rhs = np.concatenate([rs, rp, [0.0]])
    x = spla.spsolve(K, rhs)
    return np.asarray(x[:ns])


def _sub(A, r, c):
    return A[r][:, c].tocsc()


def _check_transfer(mesh, Hh, l, Ms, Ds, ones):
    """Every column of P_sigma of step l -> l+1 against the local problems of App. A.2. Returns counts per kind."""
    tr = Hh.transfers[l]
    lv = _Level(mesh, Hh, l, Ms[l], Ds[l], ones[l])
    coarse = Hh.levels[l + 1]
    agg = tr.agg_of
    cells_of = [np.where(agg == a)[0] for a in range(coarse.n_cells)]
    Ps = tr.Psigma.tocsc()
    Pp = tr.Pp.tocsc()
    c_off = coarse.p_off
    n_pairs = len(tr.extra["pairs"])
    own = lv.own

    def interface_unknowns(a, b):
        c0, c1 = agg[own[:, 0]], np.where(own[:, 1] >= 0, agg[np.maximum(own[:, 1], 0)], -1)
        sel = (lv.kind == IFACE) & (own[:, 1] >= 0) & (((c0 == a) & (c1 == b)) | ((c0 == b) & (c1 == a)))
        return np.where(sel)[0]

    def boundary_unknowns(a):
        return np.where((lv.kind == BDRY) & (agg[own[:, 0]] == a))[0]

    def extension(a, Fd, t):
        """eq. local_neumann_boundary_value_problem: s on the inner unknowns of aggregate a from the trace t on Fd,
        c = q_PV^T D_{A,F} t."""
        ia, pa = lv.inner(cells_of[a]), lv.pdofs(cells_of[a])
        q = lv.one[pa] / np.linalg.norm(lv.one[pa])
        DaF_t = _sub(lv.D, pa, Fd) @ t
        c = q @ DaF_t
        if ia.size == 0:
            return np.zeros(0)
        return _sparse_saddle(_sub(lv.M, ia, ia), _sub(lv.D, pa, ia), -(_sub(lv.M, ia, Fd) @ t), c * q - DaF_t,
                              null=lv.one[pa])

    counts = {"sigma_pv": 0, "boundary": 0, "bubble": 0, "extension": 0}
    bubble_index = {}
    for J in range(coarse.n_flux):
        col = Ps[:, J].toarray().ravel()
        scale = np.abs(col).max()
        assert scale > 0
        tol = 1e-9 * scale
        kind = coarse.flux_kind[J]
        a, b = (int(v) for v in coarse.flux_owner[J])
        if kind == IFACE and J < n_pairs:
            # eq. local_problem_to_define_sigma_pv on A_a U A_b, f = [-1_a / ||1_a||^2; 1_b / ||1_b||^2]
            assert (a, b) == tr.extra["pairs"][J] and a < b
            U = np.concatenate([cells_of[a], cells_of[b]])
            iU = lv.inner(U)
            pa, pb = lv.pdofs(cells_of[a]), lv.pdofs(cells_of[b])
            f = np.concatenate([-lv.one[pa] / (lv.one[pa] @ lv.one[pa]), lv.one[pb] / (lv.one[pb] @ lv.one[pb])])
            pU = np.concatenate([pa, pb])
            s = _sparse_saddle(_sub(lv.M, iU, iU), _sub(lv.D, pU, iU), np.zeros(iU.size), f, null=lv.one[pU])
            Fd = interface_unknowns(a, b)
            # sigma^PV is the restriction to F; with one trace per interface its extension into A_a and A_b is the
            # rest of the same local solution (both solve the same Neumann problem), so the whole column is s
            assert np.all(np.isin(Fd, iU))
            assert np.allclose(col[iU], s, rtol=0, atol=tol)
            out = np.ones(col.size, bool)
            out[iU] = False
            assert np.all(col[out] == 0.0)
            counts["sigma_pv"] += 1
        elif kind == BDRY:
            # coarse Dirichlet unknown of aggregate a: the local saddle on A_a with its Dirichlet unknowns kept and
            # pressure data -1_a / ||1_a||^2 (nonsingular: the Dirichlet unknowns fix the pressure)
            Bd = boundary_unknowns(a)
            ia, pa = lv.inner(cells_of[a]), lv.pdofs(cells_of[a])
            ids = np.concatenate([ia, Bd])
            s = _sparse_saddle(_sub(lv.M, ids, ids), _sub(lv.D, pa, ids), np.zeros(ids.size),
                               -lv.one[pa] / (lv.one[pa] @ lv.one[pa]))
            assert np.allclose(col[ids], s, rtol=0, atol=tol)
            out = np.ones(col.size, bool)
            out[ids] = False
            assert np.all(col[out] == 0.0)
            counts["boundary"] += 1
        elif kind == BUBBLE:
            # eq. local_neumann_boundary_value_problem with right-hand side [0; q], q the next column of P_NPV of a
            k = bubble_index.get(a, 1)
            bubble_index[a] = k + 1
            pa = lv.pdofs(cells_of[a])
            q = Pp[pa, c_off[a] + k].toarray().ravel()
            ia = lv.inner(cells_of[a])
            s = _sparse_saddle(_sub(lv.M, ia, ia), _sub(lv.D, pa, ia), np.zeros(ia.size), q, null=lv.one[pa])
            assert np.allclose(col[ia], s, rtol=0, atol=tol)
            out = np.ones(col.size, bool)
            out[ia] = False
            assert np.all(col[out] == 0.0)
            counts["bubble"] += 1
        if kind in (IFACE, BDRY):
            # every trace (sigma^PV, the added traces of m_f > 1, boundary traces) is extended into each owner by
            # eq. local_neumann_boundary_value_problem
            Fd = interface_unknowns(a, b) if kind == IFACE else boundary_unknowns(a)
            t = col[Fd]
            for c in ((a, b) if kind == IFACE else (a,)):
                ic = lv.inner(cells_of[c])
                assert np.allclose(col[ic], extension(c, Fd, t), rtol=0, atol=tol)
                counts["extension"] += 1
    # every aggregate got all its bubbles (m_a - 1 each)
    for a in range(coarse.n_cells):
        assert bubble_index.get(a, 1) == coarse.m[a]
    return counts


@pytest.fixture(scope="module", params=["cart2d", "chan3d", "chan3d_mf3", "voronoi"])
def case(request):
    if request.param == "cart2d":
        pr = problem_config("cart2d_32", scale=16)
        opts = dict(pr.opts, n_levels=3, agg_size=[16, 4], modes=[3, 2])
    elif request.param.startswith("chan3d"):
        pr = problem_config("chan3d_64", scale=8)
        opts = dict(pr.opts, agg_size=[16, 4, 4], modes=[3, 3, 3])
        if request.param.endswith("mf3"):
            opts["flux_modes"] = [3, 3, 3]
    else:
        pr = voronoi_problem(7)
        opts = dict(pr.opts, n_levels=3, agg_size=[16, 4], modes=[3, 2])
    Hh = hierarchy.build(pr.mesh, opts)
    return pr, Hh


def test_local_problems_of_every_coarse_flux_unknown(case):
    """App. A.2: sigma^PV (eq. local_problem_to_define_sigma_pv), the trace extensions (eq.
    local_neumann_boundary_value_problem), the bubbles (the same problem with data [0; q]) and the coarse boundary
    traces, on every level, recomputed from independently assembled operators."""
    pr, Hh = case
    Ms, Ds, ones = _independent_operators(pr.mesh, Hh)
    for l in range(len(Hh.transfers)):
        counts = _check_transfer(pr.mesh, Hh, l, Ms, Ds, ones)
        assert counts["sigma_pv"] > 0 and counts["extension"] >= 2 * counts["sigma_pv"]
        assert counts["boundary"] > 0 and counts["bubble"] > 0


def test_sigma_pv_carries_unit_net_flux(case):
    """With the data f_F of eq. local_problem_to_define_sigma_pv, the flux sigma^PV takes out of A_a through F is
    1^T f|_{A_a} times -1, i.e. exactly 1 (in the level's 1^l weighting), and the paper's non-degeneracy
    q_PV^T D_{A,F} sigma^PV != 0 holds."""
    pr, Hh = case
    Ms, Ds, ones = _independent_operators(pr.mesh, Hh)
    for l, tr in enumerate(Hh.transfers):
        lv = _Level(pr.mesh, Hh, l, Ms[l], Ds[l], ones[l])
        Ps = tr.Psigma.tocsc()
        for J, (a, b) in enumerate(tr.extra["pairs"]):
            pa = lv.pdofs(np.where(tr.agg_of == a)[0])
            out_a = -(lv.one[pa] @ (lv.D[pa] @ Ps[:, J].toarray().ravel()))
            assert abs(out_a - 1.0) <= 1e-10


def _neumann_1d_brute_force(nx, ups_half, area, vol, a, gl, gn, f):
    """Dense Newton written with plain loops for the 1D TPFA problem kappa = exp(a p): Dirichlet g_D = gl at the left
    end, the Neumann flux density gn through the right end (the flux leaving the last cell there is -area * gn, so
    it enters [f] as +area * gn), source density f in every cell."""
    p = [gl] * nx
    for _ in range(100):
        R = [0.0] * nx
        J = [[0.0] * nx for _ in range(nx)]
        for i in range(nx):
            k = np.exp(a * p[i])
            dk = a * k
            for j in (i - 1, i + 1):
                if j < 0 or j >= nx:
                    continue
                kj = np.exp(a * p[j])
                hi, hj = k * ups_half, kj * ups_half
                u = 1.0 / (1.0 / hi + 1.0 / hj)
                R[i] += u * (p[i] - p[j])
                J[i][i] += u + u * u / (hi * hi) * dk * ups_half * (p[i] - p[j])
                J[i][j] += -u + u * u / (hj * hj) * a * kj * ups_half * (p[i] - p[j])
            if i == 0:
                R[i] += k * ups_half * (p[i] - gl)
                J[i][i] += dk * ups_half * (p[i] - gl) + k * ups_half
            R[i] -= vol * f
            if i == nx - 1:
                R[i] -= area * gn
        if max(abs(v) for v in R) < 1e-14:
            break
        dp = np.linalg.solve(np.array(J), -np.array(R))
        p = [p[i] + dp[i] for i in range(nx)]
    return np.array(p)


@pytest.mark.parametrize("gn,f", [(0.7, 0.0), (-0.4, 0.0), (0.3, 1.5)])
def test_neumann_data_enter_the_residual(gn, f):
    """Definitions under eq. FV_matrix: a Neumann face carries the prescribed flux -|eps| g_N out of its cell, so
    [f]_K = |tau_K| f_K + sum_Neumann |eps| g_N. A 2D strip with uniform K_0, Dirichlet data on x = 0, a uniform
    flux density g_N through x = 1 and no flow through the other sides reduces to one 1D problem per row; the
    oracle's p* must equal the loop-written 1D Newton solution in every row, and its residual must vanish there."""
    nx, ny = 9, 3
    mesh = cartesian_mesh((nx, ny), np.ones(nx * ny))
    right = np.where((mesh.face_bc == BC_DIRICHLET) & (mesh.face_cells[:, 0] % nx == nx - 1))[0]
    mesh.face_bc[right] = BC_NEUMANN
    g = np.zeros(mesh.n_faces)
    left = np.where(mesh.face_bc == BC_DIRICHLET)[0]
    g[left] = 1.0
    g[right] = gn
    a = 1.2
    fc = np.full(mesh.n_cells, f)
    p, _ = newton.solve(mesh, KAPPA_EXP, a, fc, g)
    area = 1.0 / ny
    ups_half = area * 1.0 / (0.5 / nx)
    p1 = _neumann_1d_brute_force(nx, ups_half, area, 1.0 / (nx * ny), a, 1.0, gn, f)
    for j in range(ny):
        assert np.allclose(p[j * nx:(j + 1) * nx], p1, rtol=0, atol=1e-12)
    # the solution is not the Dirichlet-only one: the data moved it
    assert np.abs(p1 - 1.0).max() > 1e-2
    r = tpfa.reduced_residual(mesh, KAPPA_EXP, a, np.tile(p1, ny), fc, g)
    assert np.abs(r).max() <= 1e-12
