"""Multilevel spectral coarsening in FP64 (oracle; test only).

Builds, level by level, the objects of App. A of the paper with m_f >= 1 flux unknowns per coarse interface:
  * Level: the mixed operator data of one level, stored cell by cell as in Prop. 1 / eq. assemble: for every cell
    c its static local flux matrix Mloc[c] (so that M(Pi~ p) = sum_c W_c^T Mloc[c] W_c / kappa(pbar_c)), its local
    divergence block Dloc[c] (so that D = sum_c rows_c Dloc[c] W_c) and its Pi~ weights w[c] (pbar_c = w[c].p_c).
  * coarsen(): App. A.1 (aggregates, local eigenproblem eq. local-eigenvalue-problem on the extended aggregate,
    SVD, q_PV first column eqs. structure_pressure_interpolation / definition_q_pv, Q_p = P_p^T), App. A.2
    (sigma^PV from eq. local_problem_to_define_sigma_pv, trace extension by eq.
    local_neumann_boundary_value_problem, bubbles), D^{l+1} = P_p^T D^l P_sigma (Sec. 3.1), the static local
    matrices of Prop. 1 (App. C: M_A^{l+1} = P_sigma,A^T M_A^l P_sigma,A) and the Pi~ weights of eq. pwc_projector.

Readings where the paper is silent:
  * the reference operator for the local eigenproblems is the one at kappa = 1 ("for a given discrete pressure");
  * M restricted to N(A) keeps the flux unknowns whose cells all lie in N(A): interfaces with both owners in N(A)
    and the bubbles of cells in N(A); boundary (Dirichlet) unknowns are not graph edges and are left out;
  * eigenvectors are restricted to A, q_PV is projected out of them, and the left singular vectors with singular
    value > 1e-10 * the largest are kept (at most m - 1); each kept column is signed so that its entry of largest
    magnitude (lowest index on ties) is positive;
  * coarse Dirichlet boundary: the boundary unknowns owned by an aggregate's cells form one coarse boundary unknown,
    whose trace comes from the local problem on the aggregate with those unknowns kept and pressure data
    -1/||1_A||^2 1_A, then extended like an interface trace;
  * Q_sigma (whose construction the paper defers): an interface (or boundary) coefficient is the total flux
    leaving the aggregate through that interface divided by the same total for its basis function; the bubble
    coefficients of A are P_NPV,A^T (D sigma)|_A. This gives Q_sigma P_sigma = I and D^{l+1} Q_sigma = Q_p D^l.
  * m_f > 1 (App. A.2, eq. definition-traces): the traces at F_{K,L} are (M_N^-1 D_N^T q_i)|_F on N = N(A_K) for every
    column q_i of P_{A_K} (extended by zero from A_K to N(A_K)), and the same from A_L. Each is scaled to unit 2-norm
    and projected by Pi_F = I - sigma^PV t^T / (t . sigma^PV), t the outflow functional of A_K through F, so that
    sigma^PV stays the only carrier of the net flux through F; the left singular vectors of the projected set with
    singular value > 1e-8 are kept (at most m_f - 1 and |F| - 1), each signed so that its first entry within 1e-6 of
    the largest magnitude is positive. Each is extended
    into A_K and A_L like sigma^PV (its net flux, hence its coarse divergence, is zero) and is numbered after the
    bubbles, interface by interface; its Q_sigma row is u^T Pi_F (u orthonormal), which keeps Q_sigma P_sigma = I and the commuting
    relation. Coarse boundary unknowns keep one trace.
Local Neumann problems are solved densely with the pressure null vector 1^l fixed by a bordering constraint.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import aggregation
from .tpfa import BC_INTERIOR, BC_DIRICHLET, flux_dofs

KIND_IFACE, KIND_BDRY, KIND_BUBBLE = 0, 1, 2
SVD_DROP = 1e-10
TRACE_DROP = 1e-8


@dataclass
class Level:
    n_cells: int
    m: np.ndarray                  # [n_cells] pressure unknowns per cell
    n_flux: int
    flux_kind: np.ndarray          # [n_flux] KIND_*
    flux_owner: np.ndarray         # [n_flux, 2] (c, d) c < d for interfaces; (c, -1) otherwise
    loc: list                      # per cell: sorted global flux ids of its local unknowns
    Mloc: list                     # per cell: static local flux matrix
    Dloc: list                     # per cell: m_c x n_loc divergence block
    w: list                        # per cell: Pi~ weights (m_c)
    vol: np.ndarray                # [n_cells] cell (aggregate) volume
    ones: np.ndarray               # the vector 1^l over the pressure unknowns
    face_ids: np.ndarray | None = None   # level 0 only: face id of each flux unknown

    @property
    def p_off(self):
        return np.concatenate([[0], np.cumsum(self.m)]).astype(np.int64)

    @property
    def n_p(self):
        return int(np.sum(self.m))

    def pdofs(self, cells):
        off = self.p_off
        return np.concatenate([np.arange(off[c], off[c + 1]) for c in cells]) if len(cells) else np.zeros(0, int)


@dataclass
class Transfer:
    agg_of: np.ndarray             # [n_cells fine level] -> coarse cell
    Pp: sp.csr_matrix              # n_p(l) x n_p(l+1), block diagonal
    Psigma: sp.csr_matrix          # n_flux(l) x n_flux(l+1)
    Qsigma: sp.csr_matrix          # n_flux(l+1) x n_flux(l)
    extra: dict = field(default_factory=dict)

    @property
    def Qp(self):
        return self.Pp.T.tocsr()


def level0(mesh):
    """The fine level in the cell-by-cell form of eq. fine-local-product-decomposition: Mloc[K] = diag(1/Ups_bar)."""
    dofs = flux_dofs(mesh)
    nf = dofs.size
    K = mesh.face_cells[dofs, 0].astype(np.int64)
    L = mesh.face_cells[dofs, 1].astype(np.int64)
    kind = np.where(mesh.face_bc[dofs] == BC_INTERIOR, KIND_IFACE, KIND_BDRY)
    owner = np.stack([K, np.where(kind == KIND_IFACE, L, -1)], 1)
    per_cell = [[] for _ in range(mesh.n_cells)]
    for j in range(nf):
        per_cell[K[j]].append((j, 0))
        if kind[j] == KIND_IFACE:
            per_cell[L[j]].append((j, 1))
    loc, Mloc, Dloc, w = [], [], [], []
    for c in range(mesh.n_cells):
        items = sorted(per_cell[c])
        ids = np.array([j for j, _ in items], dtype=np.int64)
        ups = np.array([mesh.half_trans[dofs[j], side] for j, side in items])
        loc.append(ids)
        Mloc.append(np.diag(1.0 / ups) if ids.size else np.zeros((0, 0)))
        Dloc.append(np.array([[(-1.0 if side == 0 else 1.0) for _, side in items]]).reshape(1, ids.size))
        w.append(np.ones(1))
    return Level(n_cells=mesh.n_cells, m=np.ones(mesh.n_cells, dtype=np.int64), n_flux=nf, flux_kind=kind,
                 flux_owner=owner, loc=loc, Mloc=Mloc, Dloc=Dloc, w=w,
                 vol=np.asarray(mesh.cell_volume, dtype=np.float64).copy(), ones=np.ones(mesh.n_cells),
                 face_ids=dofs)


def assemble_M(lev, scale=None):
    """sum_c scale_c W_c^T Mloc[c] W_c (eq. assemble), scale = 1 by default."""
    rows, cols, vals = [], [], []
    for c in range(lev.n_cells):
        ids = lev.loc[c]
        if ids.size == 0:
            continue
        s = 1.0 if scale is None else scale[c]
        r, cc = np.meshgrid(ids, ids, indexing="ij")
        rows.append(r.ravel())
        cols.append(cc.ravel())
        vals.append((s * lev.Mloc[c]).ravel())
    if not rows:
        return sp.csr_matrix((lev.n_flux, lev.n_flux))
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(lev.n_flux, lev.n_flux))
    M.sum_duplicates()
    return M


def assemble_D(lev):
    """D = sum_c rows_c Dloc[c] W_c over the pressure unknowns of each cell."""
    off = lev.p_off
    rows, cols, vals = [], [], []
    for c in range(lev.n_cells):
        ids = lev.loc[c]
        r, cc = np.meshgrid(np.arange(off[c], off[c + 1]), ids, indexing="ij")
        rows.append(r.ravel())
        cols.append(cc.ravel())
        vals.append(lev.Dloc[c].ravel())
    D = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(lev.n_p, lev.n_flux))
    D.sum_duplicates()
    return D


def internal_flux(lev, cells):
    """Flux unknowns whose owner cells all lie in `cells`: interfaces with both owners inside, and bubbles."""
    inside = np.zeros(lev.n_cells, dtype=bool)
    inside[np.asarray(cells, dtype=np.int64)] = True
    c0 = lev.flux_owner[:, 0]
    c1 = lev.flux_owner[:, 1]
    ok_if = (lev.flux_kind == KIND_IFACE) & inside[c0] & inside[np.maximum(c1, 0)] & (c1 >= 0)
    ok_bu = (lev.flux_kind == KIND_BUBBLE) & inside[c0]
    return np.where(ok_if | ok_bu)[0]


def _neumann_solve(Mss, Dps, ones_p, rhs_s, rhs_p):
    """Solve [M D^T; D 0][s; p] = [rhs_s; rhs_p] with ones_p^T p = 0 (bordering); return s."""
    ns, npp = Mss.shape[0], Dps.shape[0]
    A = np.zeros((ns + npp + 1, ns + npp + 1))
    A[:ns, :ns] = Mss
    A[:ns, ns:ns + npp] = Dps.T
    A[ns:ns + npp, :ns] = Dps
    A[ns:ns + npp, -1] = ones_p
    A[-1, ns:ns + npp] = ones_p
    b = np.concatenate([rhs_s, rhs_p, [0.0]])
    x = np.linalg.solve(A, b)
    return x[:ns]


def _saddle_solve(Mss, Dps, rhs_s, rhs_p):
    ns, npp = Mss.shape[0], Dps.shape[0]
    A = np.zeros((ns + npp, ns + npp))
    A[:ns, :ns] = Mss
    A[:ns, ns:] = Dps.T
    A[ns:, :ns] = Dps
    x = np.linalg.solve(A, np.concatenate([rhs_s, rhs_p]))
    return x[:ns]


def _sign_fix(u):
    i = int(np.argmax(np.abs(u)))
    return u if u[i] > 0 else -u


def _sign_fix_tie(u):
    """Sign of a kept trace: its first entry within 1e-6 (relative) of the largest magnitude is made positive, so
    that entries equal in exact arithmetic (mirror-symmetric interfaces) do not let rounding pick the sign."""
    a = np.abs(u)
    i = int(np.argmax(a >= (1.0 - 1e-6) * a.max()))
    return u if u[i] > 0 else -u


def coarsen(lev, target, modes, fine_vol, P0_prev, fine_agg_prev, flux_modes=1):
    """One coarsening step l -> l+1. Returns (coarse Level, Transfer, composed P to level 0, fine->coarse map).

    flux_modes: m_f, flux unknowns per coarse interface at most (1: sigma^PV alone).
    fine_vol: level-0 cell volumes; P0_prev: (P_p)^0_l (sparse, n_fine x n_p(l)); fine_agg_prev: level-0 cell ->
    level-l cell map.
    """
    # --- App. A.1: aggregates of the level-l cell graph (edges = interface unknowns) -----------------------
    ifc = np.where(lev.flux_kind == KIND_IFACE)[0]
    nbrs = aggregation.adjacency(lev.n_cells, lev.flux_owner[ifc])
    agg_of = aggregation.aggregate(lev.n_cells, nbrs, target)
    n_agg = int(agg_of.max()) + 1
    cells_of = [np.where(agg_of == a)[0] for a in range(n_agg)]
    M1 = assemble_M(lev).tocsr()
    D = assemble_D(lev).tocsr()
    Md = M1.toarray() if lev.n_flux <= 4000 else None

    def Msub(r, c):
        if Md is not None:
            return Md[np.ix_(r, c)]
        return M1[r][:, c].toarray()

    def Dsub(r, c):
        return D[r][:, c].toarray()

    # --- local eigenproblems on extended aggregates -> P_A = [q_PV, P_NPV] ------------------------------------
    PA = []
    eig_gap = []
    trace_src = []       # m_f > 1: (sN, M_N^-1 D_N^T [P_A extended by zero]) per aggregate, eq. definition-traces
    for a in range(n_agg):
        cA = cells_of[a]
        ext = set(cA.tolist())
        for c in cA:
            ext.update(nbrs[c])
        cN = np.array(sorted(ext), dtype=np.int64)
        pN = lev.pdofs(cN)
        sN = internal_flux(lev, cN)
        DN = Dsub(pN, sN)
        MN = Msub(sN, sN)
        LN = DN @ np.linalg.solve(MN, DN.T) if sN.size else np.zeros((pN.size, pN.size))
        LN = 0.5 * (LN + LN.T)
        lam, vec = np.linalg.eigh(LN)
        pA = lev.pdofs(cA)
        m = min(modes, pA.size)
        pos = np.searchsorted(pN, pA)
        V = vec[pos, :m]
        eig_gap.append(lam[m] - lam[m - 1] if m < lam.size else np.inf)
        q = lev.ones[pA] / np.linalg.norm(lev.ones[pA])
        V = V - np.outer(q, q @ V)
        cols = [q]
        if m > 1:
            U, S, _ = np.linalg.svd(V, full_matrices=False)
            if S.size and S[0] > 0:
                k = int(np.sum(S > SVD_DROP * S[0]))
                k = min(k, m - 1, pA.size - 1)
                for j in range(k):
                    cols.append(_sign_fix(U[:, j]))
        PA.append(np.stack(cols, 1))
        if flux_modes > 1:
            Qt = np.zeros((pN.size, PA[-1].shape[1]))
            Qt[pos] = PA[-1]
            trace_src.append((sN, np.linalg.solve(MN, DN.T @ Qt) if sN.size else np.zeros((0, Qt.shape[1]))))
    mc = np.array([P.shape[1] for P in PA], dtype=np.int64)
    coff = np.concatenate([[0], np.cumsum(mc)])
    rows, cols_, vals = [], [], []
    for a in range(n_agg):
        pA = lev.pdofs(cells_of[a])
        r, c = np.meshgrid(pA, np.arange(coff[a], coff[a + 1]), indexing="ij")
        rows.append(r.ravel())
        cols_.append(c.ravel())
        vals.append(PA[a].ravel())
    Pp = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols_))),
                       shape=(lev.n_p, int(coff[-1])))
    ones_c = Pp.T @ lev.ones

    # --- App. A.2: coarse flux space ----------------------------------------------------------------------------
    own = lev.flux_owner
    iface_pairs = {}
    for j in ifc:
        a, b = int(agg_of[own[j, 0]]), int(agg_of[own[j, 1]])
        if a != b:
            iface_pairs.setdefault((min(a, b), max(a, b)), []).append(int(j))
    pairs = sorted(iface_pairs)
    bdry = np.where(lev.flux_kind == KIND_BDRY)[0]
    bdry_of = [[] for _ in range(n_agg)]
    for j in bdry:
        bdry_of[int(agg_of[own[j, 0]])].append(int(j))
    bdry_aggs = [a for a in range(n_agg) if bdry_of[a]]
    int_of = [internal_flux(lev, cells_of[a]) for a in range(n_agg)]
    pd_of = [lev.pdofs(cells_of[a]) for a in range(n_agg)]

    def extend(a, Fd, sF):
        """eq. local_neumann_boundary_value_problem: extend trace sF (on unknowns Fd) into aggregate a."""
        ia, pa = int_of[a], pd_of[a]
        q = lev.ones[pa] / np.linalg.norm(lev.ones[pa])
        DaF = Dsub(pa, Fd) @ sF
        c_a = q @ DaF
        if ia.size == 0:
            return np.zeros(0), c_a
        rs = -Msub(ia, Fd) @ sF
        rp = c_a * q - DaF
        return _neumann_solve(Msub(ia, ia), Dsub(pa, ia), lev.ones[pa], rs, rp), c_a

    def extra_traces(a, b, Fd, sF, tvec):
        """m_f > 1: orthonormal traces on F beside sigma^PV, and the projection Pi_F (docstring of the module)."""
        cols = []
        for c in (a, b):
            sN, T = trace_src[c]
            pos = np.searchsorted(sN, Fd)
            assert np.all(sN[pos] == Fd)
            for i in range(T.shape[1]):
                v = T[pos, i]
                nv = np.linalg.norm(v)
                if nv > 0:
                    cols.append(v / nv)
        Pi = np.eye(Fd.size) - np.outer(sF, tvec) / (tvec @ sF)
        if not cols or Fd.size < 2:
            return [], Pi, np.zeros(0)
        U, S, _ = np.linalg.svd(Pi @ np.stack(cols, 1), full_matrices=False)
        k = min(int(np.sum(S > TRACE_DROP)), flux_modes - 1, Fd.size - 1)
        return [_sign_fix_tie(U[:, j]) for j in range(k)], Pi, S

    psi_cols = []        # (support ids, values)
    qrows = []           # (ids, coefficients)
    coarse_kind, coarse_owner = [], []
    sigma_pv = {}
    trace_sv = {}        # m_f > 1: singular values of the projected trace set per interface
    pending = []         # m_f > 1: the kept traces, numbered after the bubbles (interface by interface)
    for (a, b) in pairs:
        Fd = np.array(sorted(iface_pairs[(a, b)]), dtype=np.int64)
        U = np.concatenate([cells_of[a], cells_of[b]])
        iU = internal_flux(lev, U)
        pU = np.concatenate([pd_of[a], pd_of[b]])
        na2 = np.sum(lev.ones[pd_of[a]] ** 2)
        nb2 = np.sum(lev.ones[pd_of[b]] ** 2)
        fF = np.concatenate([-lev.ones[pd_of[a]] / na2, lev.ones[pd_of[b]] / nb2])
        sU = _neumann_solve(Msub(iU, iU), Dsub(pU, iU), lev.ones[pU], np.zeros(iU.size), fF)
        sF = sU[np.searchsorted(iU, Fd)]
        sigma_pv[(a, b)] = sF
        ea, _ = extend(a, Fd, sF)
        eb, _ = extend(b, Fd, sF)
        ids = np.concatenate([int_of[a], Fd, int_of[b]])
        v = np.concatenate([ea, sF, eb])
        psi_cols.append((ids, v))
        tvec = -(lev.ones[pd_of[a]] @ Dsub(pd_of[a], Fd))          # outflow of a through F
        qrows.append((Fd, tvec / (tvec @ sF)))
        coarse_kind.append(KIND_IFACE)
        coarse_owner.append((a, b))
        if flux_modes > 1:
            extras, Pi, sv = extra_traces(a, b, Fd, sF, tvec)
            trace_sv[(a, b)] = sv
            for u in extras:
                ea, _ = extend(a, Fd, u)
                eb, _ = extend(b, Fd, u)
                pending.append(((ids, np.concatenate([ea, u, eb])), (Fd, Pi.T @ u), (a, b)))
    for a in bdry_aggs:
        Bd = np.array(sorted(bdry_of[a]), dtype=np.int64)
        ia, pa = int_of[a], pd_of[a]
        ids_s = np.concatenate([ia, Bd])
        n2 = np.sum(lev.ones[pa] ** 2)
        s_all = _saddle_solve(Msub(ids_s, ids_s), Dsub(pa, ids_s), np.zeros(ids_s.size), -lev.ones[pa] / n2)
        sB = s_all[ia.size:]
        ea, _ = extend(a, Bd, sB)
        psi_cols.append((np.concatenate([ia, Bd]), np.concatenate([ea, sB])))
        tvec = -(lev.ones[pa] @ Dsub(pa, Bd))
        qrows.append((Bd, tvec / (tvec @ sB)))
        coarse_kind.append(KIND_BDRY)
        coarse_owner.append((a, -1))
    for a in range(n_agg):
        ia, pa = int_of[a], pd_of[a]
        Dfull = D[pa].toarray()
        for j in range(1, mc[a]):
            qj = PA[a][:, j]
            sb = _neumann_solve(Msub(ia, ia), Dsub(pa, ia), lev.ones[pa], np.zeros(ia.size), qj)
            psi_cols.append((ia, sb))
            row = qj @ Dfull
            nz = np.nonzero(row)[0]
            qrows.append((nz, row[nz]))
            coarse_kind.append(KIND_BUBBLE)
            coarse_owner.append((a, -1))
    for col, qr, ab in pending:
        psi_cols.append(col)
        qrows.append(qr)
        coarse_kind.append(KIND_IFACE)
        coarse_owner.append(ab)
    ncf = len(psi_cols)
    rows, cols_, vals = [], [], []
    for J, (ids, v) in enumerate(psi_cols):
        rows.append(ids)
        cols_.append(np.full(ids.size, J))
        vals.append(v)
    Psig = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols_))),
                         shape=(lev.n_flux, ncf))
    rows, cols_, vals = [], [], []
    for J, (ids, v) in enumerate(qrows):
        rows.append(np.full(ids.size, J))
        cols_.append(ids)
        vals.append(v)
    Qsig = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols_))),
                         shape=(ncf, lev.n_flux))

    # --- coarse operators: D^{l+1} = P_p^T D P_sigma, static local M (App. C), Pi~ weights ----------------------
    Dc = (Pp.T @ D @ Psig).tocsr()
    coarse_owner = np.array(coarse_owner, dtype=np.int64).reshape(-1, 2)
    coarse_kind = np.array(coarse_kind, dtype=np.int64)
    loc_c = [[] for _ in range(n_agg)]
    for J in range(ncf):
        loc_c[coarse_owner[J, 0]].append(J)
        if coarse_owner[J, 1] >= 0:
            loc_c[coarse_owner[J, 1]].append(J)
    loc_c = [np.array(sorted(x), dtype=np.int64) for x in loc_c]
    PsigT = Psig.tocsc()
    Mloc_c, Dloc_c, w_c = [], [], []
    P0 = (P0_prev @ Pp).tocsr()
    fine_agg = agg_of[fine_agg_prev]
    vol_c = np.zeros(n_agg)
    np.add.at(vol_c, agg_of, lev.vol)
    for a in range(n_agg):
        dofsA = np.unique(np.concatenate([lev.loc[c] for c in cells_of[a]]))
        MA = np.zeros((dofsA.size, dofsA.size))
        for c in cells_of[a]:
            pos = np.searchsorted(dofsA, lev.loc[c])
            MA[np.ix_(pos, pos)] += lev.Mloc[c]
        PsA = PsigT[:, loc_c[a]].tocsr()[dofsA].toarray()
        Mloc_c.append(PsA.T @ MA @ PsA)
        Dloc_c.append(Dc[coff[a]:coff[a + 1]][:, loc_c[a]].toarray())
        fcells = np.where(fine_agg == a)[0]
        w_c.append((fine_vol[fcells] @ P0[fcells][:, coff[a]:coff[a + 1]].toarray()) / vol_c[a])
    coarse = Level(n_cells=n_agg, m=mc, n_flux=ncf, flux_kind=coarse_kind, flux_owner=coarse_owner, loc=loc_c,
                   Mloc=Mloc_c, Dloc=Dloc_c, w=w_c, vol=vol_c, ones=ones_c)
    tr = Transfer(agg_of=agg_of, Pp=Pp, Psigma=Psig, Qsigma=Qsig,
                  extra=dict(PA=PA, sigma_pv=sigma_pv, pairs=pairs, eig_gap=np.array(eig_gap), Dc=Dc,
                             trace_sv=trace_sv))
    return coarse, tr, P0, fine_agg


@dataclass
class Hierarchy:
    levels: list
    transfers: list


def build(mesh, opts):
    """Levels 0..n_levels-1 with aggregate targets opts['agg_size'][l], modes opts['modes'][l] and flux unknowns per
    coarse interface opts['flux_modes'][l] (default 1)."""
    lev = level0(mesh)
    levels, transfers = [lev], []
    P0 = sp.identity(mesh.n_cells, format="csr")
    fagg = np.arange(mesh.n_cells)
    mf = opts.get("flux_modes", [1] * 8)
    for l in range(opts["n_levels"] - 1):
        lev, tr, P0, fagg = coarsen(lev, opts["agg_size"][l], opts["modes"][l], mesh.cell_volume, P0, fagg,
                                    flux_modes=int(mf[l]))
        levels.append(lev)
        transfers.append(tr)
    return Hierarchy(levels, transfers)
