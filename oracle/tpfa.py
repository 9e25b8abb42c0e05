"""Fine-level TPFA operators in FP64 (oracle; test infrastructure only).

Follows Sec. 2.1 of the paper:
  * eq. TPFA_flux: interior flux  sigma = -Ups_KL (p_L - p_K), Dirichlet flux sigma = -Ups_K,eps (g_D - p_K)
    (the printed comma "(g_D, - p_K)" is read as a minus sign), Neumann flux sigma = -|eps| g_N;
  * eq. half-transmissibility: Ups_i,eps = kappa(p_i) * Ups_bar_i,eps, Ups_KL the harmonic mean of the two halves;
  * eq. permeability_pressure_relationship: kappa(p) = exp(a p); the second kind (1 + p^2)^-1 is a workload's;
    the third is the static Richards' equation of Sec. 4.3 (Example 3): with p = psi + z, K(p) = K_hat(p - z) and
    eq. permeability_function_richards K_hat(psi) = K_0 alpha / (alpha + |psi|^beta), so kappa_K(p) = alpha /
    (alpha + |p - z_K|^beta) with K_0 in the transmissibilities and z_K the height of cell K (RichardsParams);
  * eq. FV_matrix and its definitions: the mixed matrices M(p) (diagonal), D, and the vectors g, [f];
  * Remark after eq. FV_matrix: the equivalent reduced cell-centred residual (eliminating sigma gives
    D M^-1 D^T p + D M^-1 g = -[f] for the mixed system as printed; the remark's sign on g is read from the mixed
    system, which is the authority).
The reduced residual used throughout is R_K(p) = (net outgoing flux of K over interior and Dirichlet faces) - [f]_K,
which equals minus the pressure row of the mixed residual with sigma eliminated.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

KAPPA_EXP, KAPPA_INV1P2, KAPPA_RICHARDS = 0, 1, 2
BC_INTERIOR, BC_DIRICHLET, BC_NEUMANN = 0, 1, 2


@dataclass
class RichardsParams:
    """Parameters of the Richards nonlinearity on one level: alpha, beta of eq. permeability_function_richards and
    the height z of every cell of that level (coarse levels: the volume-weighted aggregate mean, like Pi~ p)."""
    alpha: float
    beta: float
    z: np.ndarray


def kappa(p, kind, a):
    """kappa(p) = exp(a p) (eq. permeability_pressure_relationship), (1 + p^2)^-1, or, for the Richards kind,
    alpha / (alpha + |p - z|^beta) per cell (a: RichardsParams)."""
    p = np.asarray(p, dtype=np.float64)
    if kind == KAPPA_EXP:
        return np.exp(a * p)
    if kind == KAPPA_RICHARDS:
        psi = np.abs(p - a.z)
        return a.alpha / (a.alpha + psi ** a.beta)
    return 1.0 / (1.0 + p * p)


def dkappa(p, kind, a):
    """d kappa / dp, from the closed forms above."""
    p = np.asarray(p, dtype=np.float64)
    if kind == KAPPA_EXP:
        return a * np.exp(a * p)
    if kind == KAPPA_RICHARDS:
        psi = p - a.z
        apsi = np.abs(psi)
        den = a.alpha + apsi ** a.beta
        return -a.alpha * a.beta * np.sign(psi) * apsi ** (a.beta - 1.0) / (den * den)
    return -2.0 * p / (1.0 + p * p) ** 2


def flux_dofs(mesh):
    """Face ids that carry a flux unknown: interior and Dirichlet faces, in face order.

    Neumann faces have M = 1 and a zero column in D (eq. FV_matrix), so their flux is fixed by the data; they are
    folded into [f] and carry no unknown here.
    """
    return np.where(mesh.face_bc != BC_NEUMANN)[0]


def rhs_cell(mesh, f_cell, g_face):
    """[f]_K = |tau_K| f_K + sum over Neumann faces of K of |eps| g_N (definitions under eq. FV_matrix)."""
    rhs = mesh.cell_volume * np.asarray(f_cell, dtype=np.float64)
    neu = np.where(mesh.face_bc == BC_NEUMANN)[0]
    np.add.at(rhs, mesh.face_cells[neu, 0], mesh.face_area[neu] * g_face[neu])
    return rhs


def face_fluxes(mesh, kind, a, p, g_face):
    """sigma on every face (eq. TPFA_flux), oriented along n_K of the lower index K."""
    K = mesh.face_cells[:, 0]
    L = mesh.face_cells[:, 1]
    bc = mesh.face_bc
    sig = np.zeros(mesh.n_faces)
    kp = kappa(p, kind, a)
    it = np.where(bc == BC_INTERIOR)[0]
    hK = kp[K[it]] * mesh.half_trans[it, 0]
    hL = kp[L[it]] * mesh.half_trans[it, 1]
    ups = 1.0 / (1.0 / hK + 1.0 / hL)
    sig[it] = -ups * (p[L[it]] - p[K[it]])
    dr = np.where(bc == BC_DIRICHLET)[0]
    sig[dr] = -kp[K[dr]] * mesh.half_trans[dr, 0] * (g_face[dr] - p[K[dr]])
    ne = np.where(bc == BC_NEUMANN)[0]
    sig[ne] = -mesh.face_area[ne] * g_face[ne]
    return sig


def reduced_residual(mesh, kind, a, p, f_cell, g_face):
    """R_K(p) = sum of outgoing fluxes over interior + Dirichlet faces of K - [f]_K (eq. mass_balance_FV)."""
    p = np.asarray(p, dtype=np.float64)
    sig = face_fluxes(mesh, kind, a, p, g_face)
    out = np.zeros(mesh.n_cells)
    K = mesh.face_cells[:, 0]
    L = mesh.face_cells[:, 1]
    bc = mesh.face_bc
    it = np.where(bc == BC_INTERIOR)[0]
    dr = np.where(bc == BC_DIRICHLET)[0]
    np.add.at(out, K[it], sig[it])
    np.add.at(out, L[it], -sig[it])
    np.add.at(out, K[dr], sig[dr])
    return out - rhs_cell(mesh, f_cell, g_face)


def mixed_matrices(mesh, kind, a, p, f_cell, g_face):
    """M(p) (diagonal, over flux dofs), D (cells x flux dofs), g and [f] exactly as in eq. FV_matrix.

    Returns (M, D, g, f, dofs) with M and D scipy sparse and dofs the face ids of the flux unknowns.
    """
    dofs = flux_dofs(mesh)
    K = mesh.face_cells[dofs, 0]
    L = mesh.face_cells[dofs, 1]
    bc = mesh.face_bc[dofs]
    kp = kappa(p, kind, a)
    n = dofs.size
    mdiag = np.zeros(n)
    rows, cols, vals = [], [], []
    for j in range(n):
        if bc[j] == BC_INTERIOR:
            mdiag[j] = 1.0 / (kp[K[j]] * mesh.half_trans[dofs[j], 0]) + 1.0 / (kp[L[j]] * mesh.half_trans[dofs[j], 1])
            rows += [L[j], K[j]]
            cols += [j, j]
            vals += [1.0, -1.0]          # [D^T]_{j,:} = delta_L - delta_K
        else:
            mdiag[j] = 1.0 / (kp[K[j]] * mesh.half_trans[dofs[j], 0])
            rows += [K[j]]
            cols += [j]
            vals += [-1.0]               # Dirichlet: -delta_K
    D = sp.csr_matrix((vals, (rows, cols)), shape=(mesh.n_cells, n))
    g = np.where(bc == BC_DIRICHLET, g_face[dofs], 0.0)
    return sp.diags(mdiag).tocsr(), D, g, rhs_cell(mesh, f_cell, g_face), dofs


def reduced_jacobian(mesh, kind, a, p, g_face):
    """Exact dR/dp as a sparse matrix, differentiating the harmonic-mean transmissibility analytically."""
    p = np.asarray(p, dtype=np.float64)
    N = mesh.n_cells
    kp = kappa(p, kind, a)
    dkp = dkappa(p, kind, a)
    K = mesh.face_cells[:, 0]
    L = mesh.face_cells[:, 1]
    bc = mesh.face_bc
    rows, cols, vals = [], [], []
    it = np.where(bc == BC_INTERIOR)[0]
    k, l = K[it], L[it]
    hK = kp[k] * mesh.half_trans[it, 0]
    hL = kp[l] * mesh.half_trans[it, 1]
    ups = 1.0 / (1.0 / hK + 1.0 / hL)
    # d ups / d p_K = ups^2 / hK^2 * kappa'(p_K) Ups_bar_K
    dupsK = ups ** 2 / hK ** 2 * dkp[k] * mesh.half_trans[it, 0]
    dupsL = ups ** 2 / hL ** 2 * dkp[l] * mesh.half_trans[it, 1]
    dp = p[k] - p[l]
    # flux out of K: ups (p_K - p_L); into row K with +, into row L with -
    dF_dpK = ups + dupsK * dp
    dF_dpL = -ups + dupsL * dp
    rows += [k, k, l, l]
    cols += [k, l, k, l]
    vals += [dF_dpK, dF_dpL, -dF_dpK, -dF_dpL]
    dr = np.where(bc == BC_DIRICHLET)[0]
    kd = K[dr]
    vals.append(dkp[kd] * mesh.half_trans[dr, 0] * (p[kd] - g_face[dr]) + kp[kd] * mesh.half_trans[dr, 0])
    rows.append(kd)
    cols.append(kd)
    J = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    J.sum_duplicates()
    return J


def picard_diagonal(mesh, kind, a, p):
    """sum of the frozen-coefficient transmissibilities around each cell (interior + Dirichlet faces)."""
    kp = kappa(p, kind, a)
    K = mesh.face_cells[:, 0]
    L = mesh.face_cells[:, 1]
    bc = mesh.face_bc
    out = np.zeros(mesh.n_cells)
    it = np.where(bc == BC_INTERIOR)[0]
    ups = 1.0 / (1.0 / (kp[K[it]] * mesh.half_trans[it, 0]) + 1.0 / (kp[L[it]] * mesh.half_trans[it, 1]))
    np.add.at(out, K[it], ups)
    np.add.at(out, L[it], ups)
    dr = np.where(bc == BC_DIRICHLET)[0]
    np.add.at(out, K[dr], kp[K[dr]] * mesh.half_trans[dr, 0])
    return out
