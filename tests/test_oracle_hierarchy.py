"""Pins of the oracle's aggregation and spectral hierarchy (App. A-C of the paper) to independent facts."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import aggregation, coarse, hierarchy, tpfa
from synth.grids import cartesian_mesh, lognormal_field, problem_config

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _grid_edges(nx, ny):
    e = []
    for j in range(ny):
        for i in range(nx):
            v = i + nx * j
            if i + 1 < nx:
                e.append((v, v + 1))
            if j + 1 < ny:
                e.append((v, v + nx))
    return np.array(e)


def test_aggregation_hand_example():
    expect = np.loadtxt(os.path.join(GOLD, "aggregation_grid4x4.txt"), dtype=np.int64)
    nb = aggregation.adjacency(16, _grid_edges(4, 4))
    assert np.array_equal(aggregation.aggregate(16, nb, 4), expect)


def test_aggregation_path_merge_rule():
    """Path 0-1-...-8, target 4: {0..3}, {4..7}, {8}; {8} has 2*1 < 4 and merges into its only neighbour."""
    nb = aggregation.adjacency(9, np.array([(i, i + 1) for i in range(8)]))
    assert aggregation.aggregate(9, nb, 4).tolist() == [0, 0, 0, 0, 1, 1, 1, 1, 1]
    nb = aggregation.adjacency(10, np.array([(i, i + 1) for i in range(9)]))
    assert aggregation.aggregate(10, nb, 4).tolist() == [0, 0, 0, 0, 1, 1, 1, 1, 2, 2]


def test_aggregates_connected_and_cover():
    nx, ny = 23, 17
    nb = aggregation.adjacency(nx * ny, _grid_edges(nx, ny))
    agg = aggregation.aggregate(nx * ny, nb, 16)
    assert agg.min() == 0 and len(np.unique(agg)) == agg.max() + 1
    for a in range(agg.max() + 1):
        members = set(np.where(agg == a)[0].tolist())
        seen, stack = set(), [next(iter(members))]
        while stack:
            v = stack.pop()
            if v in seen:
                continue
            seen.add(v)
            stack += [u for u in nb[v] if u in members]
        assert seen == members


@pytest.fixture(scope="module")
def hier2d():
    pr = problem_config("cart2d_32", scale=16)
    return pr, hierarchy.build(pr.mesh, pr.opts)


@pytest.fixture(scope="module")
def hier3d():
    pr = problem_config("chan3d_64", scale=8)
    opts = dict(pr.opts, agg_size=[16, 4, 4], modes=[3, 3, 3])
    return pr, hierarchy.build(pr.mesh, opts)


@pytest.fixture(scope="module")
def hier3d_mf():
    """m_f = 3 flux unknowns per coarse interface at most (App. A.2), three levels."""
    pr = problem_config("chan3d_64", scale=8)
    opts = dict(pr.opts, agg_size=[16, 4, 4], modes=[3, 3, 3], flux_modes=[3, 3, 3])
    return pr, hierarchy.build(pr.mesh, opts)


def _levels(request):
    return request.getfixturevalue(request.param)


@pytest.fixture(params=["hier2d", "hier3d", "hier3d_mf"])
def H(request):
    return _levels(request)


def test_bases_orthonormal_with_constant_first(H):
    pr, Hh = H
    for l, tr in enumerate(Hh.transfers):
        lev = Hh.levels[l]
        for a, PA in enumerate(tr.extra["PA"]):
            assert np.allclose(PA.T @ PA, np.eye(PA.shape[1]), atol=1e-13)
            cells = np.where(tr.agg_of == a)[0]
            ones = lev.ones[lev.pdofs(cells)]
            assert np.allclose(PA[:, 0], ones / np.linalg.norm(ones), atol=1e-14)


def test_level0_basis_spans_low_eigenvectors(hier2d):
    """eq. local-eigenvalue-problem at level 0 is the kappa = 1 TPFA graph Laplacian of N(A) (interior faces inside
    N(A) only); the span of P_A equals the span of q_PV and the restricted low eigenvectors."""
    pr, Hh = hier2d
    m = pr.mesh
    tr = Hh.transfers[0]
    K, L = m.face_cells[:, 0], m.face_cells[:, 1]
    it = np.where(m.face_bc == 0)[0]
    T = 1.0 / (1.0 / m.half_trans[it, 0] + 1.0 / m.half_trans[it, 1])
    for a in range(0, tr.agg_of.max() + 1, 3):
        cells = np.where(tr.agg_of == a)[0]
        nbr = set()
        for j, f in enumerate(it):
            if K[f] in set(cells.tolist()):
                nbr.add(L[f])
            if L[f] in set(cells.tolist()):
                nbr.add(K[f])
        N = np.array(sorted(set(cells.tolist()) | nbr))
        idx = {c: i for i, c in enumerate(N)}
        Lap = np.zeros((N.size, N.size))
        for j, f in enumerate(it):
            if K[f] in idx and L[f] in idx:
                u, v = idx[K[f]], idx[L[f]]
                Lap[u, u] += T[j]
                Lap[v, v] += T[j]
                Lap[u, v] -= T[j]
                Lap[v, u] -= T[j]
        lam, vec = sla.eigh(Lap)
        PA = tr.extra["PA"][a]
        k = PA.shape[1]
        assert np.allclose(vec[:, 0], vec[0, 0])          # connected Neumann graph: constant null vector
        V = vec[[idx[c] for c in cells], 1:k]
        Q, _ = np.linalg.qr(np.column_stack([np.ones(cells.size), V]))
        assert np.allclose(PA @ PA.T, Q @ Q.T, atol=1e-9)


def test_projection_identities(H):
    """QP = I for flux and pressure (Sec. 3.1), Pi = PQ idempotent (eq. projection_property), and the commuting
    property D^{l+1} Q_sigma = Q_p D^l."""
    pr, Hh = H
    for l, tr in enumerate(Hh.transfers):
        QsPs = (tr.Qsigma @ tr.Psigma).toarray()
        assert np.allclose(QsPs, np.eye(QsPs.shape[0]), atol=1e-11)
        QpPp = (tr.Qp @ tr.Pp).toarray()
        assert np.allclose(QpPp, np.eye(QpPp.shape[0]), atol=1e-13)
        Pi = (tr.Psigma @ tr.Qsigma).toarray()
        assert np.allclose(Pi @ Pi, Pi, atol=1e-10)
        D0 = hierarchy.assemble_D(Hh.levels[l])
        D1 = hierarchy.assemble_D(Hh.levels[l + 1])
        lhs = (D1 @ tr.Qsigma).toarray()
        rhs = (tr.Qp @ D0).toarray()
        assert np.allclose(lhs, rhs, atol=1e-11 * max(1.0, np.abs(rhs).max()))


def test_prop1_local_assembly_equals_galerkin(hier2d):
    """Prop. 1 / App. C at level 0 -> 1: with kappa constant on each aggregate, the assembled coarse
    M^1 = sum_A W^T M_A / kappa_A W equals P_sigma^T M^0(p) P_sigma, where M^0(p) comes from eq. FV_matrix."""
    pr, Hh = hier2d
    m = pr.mesh
    tr = Hh.transfers[0]
    rng = np.random.default_rng(7)
    n_agg = tr.agg_of.max() + 1
    pa = rng.uniform(-1, 1, n_agg)
    p_fine = pa[tr.agg_of]
    M0, _, _, _, _ = tpfa.mixed_matrices(m, pr.kappa_kind, pr.kappa_a, p_fine, pr.f_cell, pr.g_face)
    gal = (tr.Psigma.T @ M0 @ tr.Psigma).toarray()
    s = 1.0 / tpfa.kappa(pa, pr.kappa_kind, pr.kappa_a)
    loc = hierarchy.assemble_M(Hh.levels[1], s).toarray()
    assert np.allclose(loc, gal, rtol=1e-12, atol=1e-12 * np.abs(gal).max())


def test_linear_coarse_saddle_is_galerkin_product(H):
    """kappa = 1: the coarse saddle [M D^T; D 0] equals P^T A P (eq. coarse-saddle)."""
    pr, Hh = H
    for l, tr in enumerate(Hh.transfers):
        L0, L1 = Hh.levels[l], Hh.levels[l + 1]
        A0 = sp.bmat([[hierarchy.assemble_M(L0), hierarchy.assemble_D(L0).T], [hierarchy.assemble_D(L0), None]])
        P = sp.block_diag([tr.Psigma, tr.Pp])
        gal = (P.T @ A0 @ P).toarray()
        A1 = sp.bmat([[hierarchy.assemble_M(L1), hierarchy.assemble_D(L1).T],
                      [hierarchy.assemble_D(L1), None]]).toarray()
        assert np.allclose(A1, gal, atol=1e-11 * np.abs(gal).max())


def test_pwc_projector_closed_form(hier2d):
    """eq. pwc_projector with uniform volumes at level 1: pbar_A = (P_A^T p)_1 / sqrt(|A|)."""
    pr, Hh = hier2d
    L1 = Hh.levels[1]
    tr = Hh.transfers[0]
    for a in range(L1.n_cells):
        n = np.sum(tr.agg_of == a)
        expect = np.zeros(L1.m[a])
        expect[0] = 1.0 / np.sqrt(n)
        assert np.allclose(L1.w[a], expect, atol=1e-14)


def test_pwc_projector_commutes_with_kappa(hier3d):
    """App. B: kappa evaluated on Pi~ p equals the volume average of kappa of the interpolated piecewise constant."""
    pr, Hh = hier3d
    m = pr.mesh
    rng = np.random.default_rng(9)
    l = len(Hh.levels) - 1
    lev = Hh.levels[l]
    p = rng.uniform(-1, 1, lev.n_p)
    pb = coarse.pbar(lev, p)
    fine_of = np.arange(m.n_cells)
    for tr in Hh.transfers[:l]:
        fine_of = tr.agg_of[fine_of]
    kf = tpfa.kappa(pb[fine_of], pr.kappa_kind, pr.kappa_a)
    avg = np.bincount(fine_of, weights=m.cell_volume * kf) / np.bincount(fine_of, weights=m.cell_volume)
    assert np.allclose(avg, tpfa.kappa(pb, pr.kappa_kind, pr.kappa_a), rtol=1e-14)
    # Pi~ p is the volume mean of the prolongated p over each aggregate (eq. pwc_projector)
    P0 = sp.identity(m.n_cells)
    for tr in Hh.transfers[:l]:
        P0 = P0 @ tr.Pp
    pf = P0 @ p
    mean = np.bincount(fine_of, weights=m.cell_volume * pf) / np.bincount(fine_of, weights=m.cell_volume)
    assert np.allclose(mean, pb, atol=1e-13)


def test_level0_mixed_operator_matches_fv_matrix():
    """The cell-by-cell level-0 data reassemble exactly the M(p) and D of eq. FV_matrix."""
    pr = problem_config("chan3d_64", scale=5)
    m = pr.mesh
    lev = hierarchy.level0(m)
    rng = np.random.default_rng(3)
    p = rng.uniform(0, 1, m.n_cells)
    M0, D0, _, _, _ = tpfa.mixed_matrices(m, pr.kappa_kind, pr.kappa_a, p, pr.f_cell, pr.g_face)
    M1 = hierarchy.assemble_M(lev, 1.0 / tpfa.kappa(p, pr.kappa_kind, pr.kappa_a))
    assert np.allclose(M1.toarray(), M0.toarray(), rtol=1e-14)
    assert np.array_equal(hierarchy.assemble_D(lev).toarray(), D0.toarray())


def test_flux_modes_add_divergence_free_traces(hier3d, hier3d_mf):
    """m_f > 1 keeps the m_f = 1 space as its leading columns (sigma^PV, boundary traces, bubbles are unchanged) and
    adds interface unknowns whose coarse divergence vanishes: they carry no net flux through their interface, so
    D^{l+1} of the m_f = 1 space is unchanged too."""
    _, H1 = hier3d
    _, H3 = hier3d_mf
    for l, (t1, t3) in enumerate(zip(H1.transfers, H3.transfers)):
        L3 = H3.levels[l + 1]
        n0 = int(np.sum(L3.flux_kind != hierarchy.KIND_IFACE)) + len(t3.extra["pairs"])   # m_f = 1 unknowns
        assert t3.Psigma.shape[1] > n0
        if l == 0:   # same fine level: the m_f = 1 space is the leading block
            P1, P3 = t1.Psigma.toarray(), t3.Psigma.toarray()
            assert t1.Psigma.shape[1] == n0
            assert np.allclose(P3[:, :n0], P1, rtol=0, atol=1e-12 * np.abs(P1).max())
            assert np.allclose(t3.Qsigma.toarray()[:n0], t1.Qsigma.toarray(), rtol=0, atol=1e-12)
        assert np.all(L3.flux_kind[n0:] == hierarchy.KIND_IFACE)
        own = L3.flux_owner[n0:]
        assert np.all(own[:, 0] >= 0) and np.all(own[:, 1] >= 0)
        Dc = hierarchy.assemble_D(L3).toarray()
        assert np.abs(Dc[:, n0:]).max() <= 1e-10 * np.abs(Dc[:, :n0]).max()
        # at most m_f unknowns per coarse interface
        pairs, counts = np.unique(np.sort(L3.flux_owner[L3.flux_kind == hierarchy.KIND_IFACE], 1), axis=0,
                                  return_counts=True)
        assert counts.max() <= 3 and counts.max() >= 2


def test_flux_modes_reproduce_the_local_traces():
    """eq. definition-traces: with m_f = 1 + (number of traces), so that no trace is cut by m_f, every trace
    (M_N^-1 D_N^T q_i)|_F of both aggregates' pressure modes, computed here by a sparse direct solve on N(A), lies in
    the span of the coarse flux unknowns of F restricted to F (checked where that span is not all of F)."""
    import scipy.sparse.linalg as spla
    pr = problem_config("chan3d_64", scale=8)
    modes = 3
    opts = dict(pr.opts, agg_size=[16, 4], modes=[modes, 2], flux_modes=[1 + 2 * modes, 1], n_levels=2)
    Hh = hierarchy.build(pr.mesh, opts)
    lev, tr = Hh.levels[0], Hh.transfers[0]
    M = hierarchy.assemble_M(lev).tocsc()
    D = hierarchy.assemble_D(lev).tocsr()
    own = lev.flux_owner
    ifc = np.where(lev.flux_kind == hierarchy.KIND_IFACE)[0]
    nbrs = [set() for _ in range(lev.n_cells)]
    for j in ifc:
        nbrs[own[j, 0]].add(int(own[j, 1]))
        nbrs[own[j, 1]].add(int(own[j, 0]))
    agg = tr.agg_of
    Ps = tr.Psigma.tocsc()
    L1 = Hh.levels[1]
    checked = 0
    for (a, b) in tr.extra["pairs"]:
        F = np.array(sorted(j for j in ifc if {agg[own[j, 0]], agg[own[j, 1]]} == {a, b}))
        cols = [J for J in range(L1.n_flux) if L1.flux_kind[J] == hierarchy.KIND_IFACE
                and sorted(L1.flux_owner[J]) == [a, b]]
        assert len(cols) <= min(F.size, 1 + 2 * modes)
        if len(cols) == F.size:
            continue                                  # the span is all of F: nothing to check
        B = Ps[:, cols].toarray()[F]
        for c in (a, b):
            cells = np.where(agg == c)[0]
            N = set(cells.tolist())
            for x in cells:
                N |= nbrs[x]
            inN = np.zeros(lev.n_cells, bool)
            inN[list(N)] = True
            sN = np.array([j for j in ifc if inN[own[j, 0]] and inN[own[j, 1]]])
            PA = tr.extra["PA"][c]
            for i in range(PA.shape[1]):
                q = np.zeros(lev.n_cells)
                q[cells] = PA[:, i]
                v = spla.spsolve(M[sN][:, sN].tocsc(), D[:, sN].T @ q)
                v = v[np.searchsorted(sN, F)]
                if np.linalg.norm(v) == 0:
                    continue
                coef, *_ = np.linalg.lstsq(B, v, rcond=None)
                assert np.linalg.norm(B @ coef - v) <= 1e-7 * np.linalg.norm(v)
                checked += 1
    assert checked > 50
