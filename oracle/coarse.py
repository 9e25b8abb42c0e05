"""Level operators and the Picard step in FP64 (oracle; test only).

  * pbar(): Pi~ p, the volume-weighted aggregate mean of the fine-interpolated pressure (eq. pwc_projector),
    evaluated with the per-cell weights built by oracle.hierarchy;
  * operator(): A^l(x) = [M^l(Pi~ p) sigma + D^T p ; D sigma] (eq. structure), with M^l(Pi~ p) assembled cell by
    cell as sum_c W_c^T Mloc[c] W_c / kappa(pbar_c) (Prop. 1, eqs. local-product-decomposition and assemble);
  * picard_solve(): the frozen-coefficient saddle of eq. picardian_system, here with the FAS right-hand side,
    solved directly with a sparse LU;
  * n_matrix(), pi_matrix(), jacobian(), newton_update(): the coarse-level Newton linearization (Sec. 3.3.2):
    M(Pi~ p) sigma = N(sigma) kappa_inv(Pi~ p) with N(sigma) = sum_c W_c^T Mloc[c] (W_c sigma) e_c^T (Prop. 2,
    eq. definition-N), hence d r_sigma / dp = N(sigma) diag(d kappa_inv / d pbar) Pi~ + D^T (Prop. 3), and the
    Jacobian of eq. jacobian_matrix with the blocks of eq. easy_jacobian_matrix_terms, solved directly with a
    sparse LU (the paper uses GMRES: the system is not symmetric).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import hierarchy
from .tpfa import dkappa, kappa


def pbar(lev, p):
    off = lev.p_off
    return np.array([lev.w[c] @ p[off[c]:off[c + 1]] for c in range(lev.n_cells)])


def operator(lev, kind, a, sigma, p):
    """A^l(x) for x = (sigma, p); returns the concatenation [flux rows; pressure rows]."""
    s = 1.0 / kappa(pbar(lev, p), kind, a)
    M = hierarchy.assemble_M(lev, s)
    D = hierarchy.assemble_D(lev)
    return np.concatenate([M @ sigma + D.T @ p, D @ sigma])


def picard_solve(lev, kind, a, sigma, p, b):
    """Solve [M(Pi~ p) D^T; D 0] x_P = b with M frozen at the current iterate (eq. picardian_system)."""
    s = 1.0 / kappa(pbar(lev, p), kind, a)
    M = hierarchy.assemble_M(lev, s)
    D = hierarchy.assemble_D(lev)
    A = sp.bmat([[M, D.T], [D, None]]).tocsc()
    x = spla.spsolve(A, b)
    return x[:lev.n_flux], x[lev.n_flux:]


def pi_matrix(lev):
    """Pi~ as an n_cells x n_p matrix: row c holds the weights w_c on the pressure unknowns of cell c, so that
    pi_matrix(lev) @ p == pbar(lev, p)."""
    off = lev.p_off
    rows = np.concatenate([np.full(off[c + 1] - off[c], c) for c in range(lev.n_cells)])
    cols = np.arange(off[-1])
    vals = np.concatenate([np.asarray(lev.w[c], dtype=np.float64) for c in range(lev.n_cells)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(lev.n_cells, lev.n_p))


def n_matrix(lev, sigma):
    """N(sigma) of eq. definition-N (n_flux x n_cells): column c is W_c^T Mloc[c] W_c sigma, the static local product
    of cell c scattered to the global flux unknowns (Prop. 2)."""
    rows, cols, vals = [], [], []
    for c in range(lev.n_cells):
        ids = lev.loc[c]
        if ids.size == 0:
            continue
        rows.append(ids)
        cols.append(np.full(ids.size, c))
        vals.append(lev.Mloc[c] @ sigma[ids])
    if not rows:
        return sp.csr_matrix((lev.n_flux, lev.n_cells))
    N = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(lev.n_flux, lev.n_cells))
    N.sum_duplicates()
    return N


def jacobian(lev, kind, a, sigma, p):
    """The Jacobian of A^l at x = (sigma, p) (eq. jacobian_matrix): [[M(Pi~ p), d r_sigma / dp], [D, 0]] with
    d r_sigma / dp = N(sigma) diag(d kappa_inv / d pbar) Pi~ + D^T (Prop. 3), kappa_inv = 1 / kappa(pbar) (eq.
    definition_inverse_kappa_vector), whose derivative is -kappa'(pbar) / kappa(pbar)^2."""
    pb = pbar(lev, p)
    k = kappa(pb, kind, a)
    M = hierarchy.assemble_M(lev, 1.0 / k)
    D = hierarchy.assemble_D(lev)
    dkinv = -dkappa(pb, kind, a) / (k * k)
    E = (n_matrix(lev, sigma) @ sp.diags(dkinv) @ pi_matrix(lev) + D.T).tocsr()
    return sp.bmat([[M, E], [D, None]]).tocsc()


def newton_update(lev, kind, a, sigma, p, b):
    """The Newton update dx solving J(x) dx = -(A^l(x) - b) (eq. jacobian_system), by a sparse LU."""
    J = jacobian(lev, kind, a, sigma, p)
    r = operator(lev, kind, a, sigma, p) - b
    return -spla.spsolve(J, r)
