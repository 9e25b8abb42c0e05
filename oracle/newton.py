"""The definitional fine solution p*: R(p*) = 0 in FP64 (oracle; test only).

R is the reduced TPFA residual (oracle.tpfa.reduced_residual, Sec. 2.1). Frozen-coefficient (Picard) steps with the
pressure-change clamp of Sec. 4.1 bring the iterate near the solution, then Newton steps with the exact Jacobian
finish it; every linear system is solved with a sparse direct LU. Each step is halved while the residual norm does
not decrease. This is a plain safeguarded iteration, not the paper's Algorithm 1: only its limit point is used.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import tpfa


def picard_matrix(mesh, kind, a, p):
    """A(kappa(p)): the TPFA matrix with transmissibilities frozen at p, so that A(kappa(p)) p - rhs = R(p)."""
    kp = tpfa.kappa(p, kind, a)
    K = mesh.face_cells[:, 0]
    L = mesh.face_cells[:, 1]
    it = np.where(mesh.face_bc == tpfa.BC_INTERIOR)[0]
    ups = 1.0 / (1.0 / (kp[K[it]] * mesh.half_trans[it, 0]) + 1.0 / (kp[L[it]] * mesh.half_trans[it, 1]))
    dr = np.where(mesh.face_bc == tpfa.BC_DIRICHLET)[0]
    rows = np.concatenate([K[it], L[it], K[it], L[it], K[dr]])
    cols = np.concatenate([L[it], K[it], K[it], L[it], K[dr]])
    vals = np.concatenate([-ups, -ups, ups, ups, kp[K[dr]] * mesh.half_trans[dr, 0]])
    A = sp.csr_matrix((vals, (rows, cols)), shape=(mesh.n_cells, mesh.n_cells))
    A.sum_duplicates()
    return A


def solve(mesh, kind, a, f_cell, g_face, p0=None, rtol=1e-14, atol=1e-300, maxit=300, dp_clamp=0.0,
          switch=1e-4):
    """Return (p*, history of ||R||_2). Picard steps until ||R|| <= switch ||R_0||, Newton afterwards."""
    p = np.zeros(mesh.n_cells) if p0 is None else np.array(p0, dtype=np.float64)
    r = tpfa.reduced_residual(mesh, kind, a, p, f_cell, g_face)
    r0 = np.linalg.norm(r)
    hist = [r0]
    for _ in range(maxit):
        nr = np.linalg.norm(r)
        if nr <= rtol * r0 or nr <= atol:
            break
        if nr > switch * r0:
            J = picard_matrix(mesh, kind, a, p).tocsc()
        else:
            J = tpfa.reduced_jacobian(mesh, kind, a, p, g_face).tocsc()
        dp = -spla.spsolve(J, r)
        mx = np.max(np.abs(dp))
        if dp_clamp > 0 and mx > dp_clamp:
            dp *= dp_clamp / mx
        if nr > switch * r0:
            # Picard phase: halve at most 4 times, accept the last trial (the rule of Algorithm 1, n_max = 4)
            s = 1.0
            for _ in range(5):
                pt = p + s * dp
                rt = tpfa.reduced_residual(mesh, kind, a, pt, f_cell, g_face)
                if np.all(np.isfinite(rt)) and np.linalg.norm(rt) < nr:
                    break
                s *= 0.5
            if not np.all(np.isfinite(rt)):
                break
        else:
            s = 1.0
            ok = False
            for _ in range(60):
                pt = p + s * dp
                rt = tpfa.reduced_residual(mesh, kind, a, pt, f_cell, g_face)
                if np.all(np.isfinite(rt)) and np.linalg.norm(rt) < nr:
                    ok = True
                    break
                s *= 0.5
            if not ok:
                break
        p, r = pt, rt
        hist.append(np.linalg.norm(r))
    return p, hist
