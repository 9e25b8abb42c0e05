"""Level operators and the Picard step in FP64 (oracle; test only).

  * pbar(): Pi~ p, the volume-weighted aggregate mean of the fine-interpolated pressure (eq. pwc_projector),
    evaluated with the per-cell weights built by oracle.hierarchy;
  * operator(): A^l(x) = [M^l(Pi~ p) sigma + D^T p ; D sigma] (eq. structure), with M^l(Pi~ p) assembled cell by
    cell as sum_c W_c^T Mloc[c] W_c / kappa(pbar_c) (Prop. 1, eqs. local-product-decomposition and assemble);
  * picard_solve(): the frozen-coefficient saddle of eq. picardian_system, here with the FAS right-hand side,
    solved directly with a sparse LU.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import hierarchy
from .tpfa import kappa


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
