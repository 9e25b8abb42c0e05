"""Fixed-length Krylov iterations and the algebraic hybridization of Sec. 3.4 in FP64 (oracle; test only).

The paper solves the linear systems of its Picard and Newton steps inexactly with Krylov methods (Sec. 3.4: CG on
the symmetric systems, GMRES on the Newton systems; hybridization on the coarse levels). A Krylov iterate after k
steps from a zero start is fixed by the method's definition, whatever the implementation's recurrences, so these
plain versions give the values an inexact solve must reproduce step for step:

  * jacobi_pcg(): k steps of CG preconditioned by diag(A) (written as CG on S A S y = S b, dx = S y, S = diag(A)^-1/2);
  * bicgstab_scaled(): k steps of BiCGStab (van der Vorst) on S J S y = S b with S = diag(w)^1/2 and shadow residual
    r^ = r_0, dx = S y;
  * hybridized(): the frozen-coefficient coarse saddle of eq. picardian_system by the algebraic hybridization of
    eqs. hybridized-block-system and hybridized-system: the flux unknowns shared by two coarse cells are broken into
    one copy per cell, flux continuity copy(K) - copy(L) = 0 (K the first owner) is imposed by a multiplier lambda,
    H lambda = xi is solved by k steps of CG preconditioned by diag(H) (or exactly), and sigma, p are recovered cell
    by cell. Readings where the paper is silent: the flux data g of a shared unknown go to the copy of its first
    owner (the broken vector g^ of eq. hybridized-block-system), and the recovered flux of a shared unknown is that
    copy's value (after an exact solve both copies agree).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .tpfa import kappa
from . import coarse


def jacobi_pcg(A, b, k, tol=0.0):
    """At most k CG steps on S A S y = S b from y = 0 (S = diag(A)^-1/2), stopping once ||r|| <= tol ||r_0|| for the
    residual r of the scaled system (or when it has vanished to rounding); returns (dx = S y, steps taken)."""
    A = sp.csr_matrix(A)
    S = 1.0 / np.sqrt(A.diagonal())
    As = sp.diags(S) @ A @ sp.diags(S)
    y = np.zeros(b.size)
    r = S * b
    p = r.copy()
    rr = r @ r
    stop = tol * tol * rr
    it = 0
    while it < k and rr > 0.0 and rr > stop:
        q = As @ p
        pq = p @ q
        if not pq > 0.0:       # the residual vanished to rounding: the iterate is the solution
            break
        alpha = rr / pq
        y += alpha * p
        r -= alpha * q
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return S * y, it


def bicgstab_scaled(J, b, w, k, tol=0.0):
    """At most k BiCGStab steps on S J S y = S b from y = 0, S = diag(w)^1/2, shadow residual r^ = r_0, stopping once
    ||r|| <= tol ||r_0||; returns (dx = S y, steps taken). A breakdown (a zero inner product) ends the iteration with
    the current y."""
    J = sp.csr_matrix(J)
    S = np.sqrt(w)
    Js = sp.diags(S) @ J @ sp.diags(S)
    y = np.zeros(b.size)
    r = S * b
    rh = r.copy()
    p = r.copy()
    v = np.zeros(b.size)
    rho = rh @ r
    stop = tol * tol * rho
    it = 0
    while it < k and r @ r > 0.0 and r @ r > stop:
        v = Js @ p
        den = rh @ v
        if den == 0.0:
            break
        alpha = rho / den
        s = r - alpha * v
        t = Js @ s
        tt = t @ t
        omega = (t @ s) / tt if tt != 0.0 else 0.0
        y = y + alpha * p + omega * s
        r = s - omega * t
        rho_new = rh @ r
        it += 1
        if omega == 0.0 or rho == 0.0:
            break
        beta = (rho_new / rho) * (alpha / omega)
        rho = rho_new
        p = r + beta * (p - omega * v)
    return S * y, it


def _local_saddles(lev, kbar):
    """Per coarse cell c: the inverse of its local saddle [Mloc[c] / kappa_c, Dloc[c]^T; Dloc[c], 0] (Prop. 1)."""
    inv = []
    for c in range(lev.n_cells):
        nl, m = lev.loc[c].size, int(lev.m[c])
        A = np.zeros((nl + m, nl + m))
        A[:nl, :nl] = lev.Mloc[c] / kbar[c]
        A[:nl, nl:] = lev.Dloc[c].T
        A[nl:, :nl] = lev.Dloc[c]
        inv.append(np.linalg.inv(A))
    return inv


def hybridized(lev, kind, a, sigma, p, rhs, k=None, tol=0.0):
    """Solve [M(Pi~ p) D^T; D 0] dx = rhs (M frozen at the iterate (sigma, p), eq. picardian_system) by hybridization
    (module docstring); k = None solves H lambda = xi exactly, else at most k Jacobi-preconditioned CG steps from
    lambda = 0, stopping once ||xi - H lambda|| <= tol ||xi||. Returns (dx, CG steps)."""
    kbar = kappa(coarse.pbar(lev, p), kind, a)
    inv = _local_saddles(lev, kbar)
    nf = lev.n_flux
    own = lev.flux_owner
    shared = np.where(own[:, 1] >= 0)[0]               # interface unknowns: one multiplier each
    lam_of = -np.ones(nf, dtype=np.int64)
    lam_of[shared] = np.arange(shared.size)
    nlam = shared.size
    off = lev.p_off
    # broken right-hand side per cell, and the columns of C^T per cell (slot, multiplier, sign)
    rhat, cons = [], []
    for c in range(lev.n_cells):
        ids = lev.loc[c]
        r = np.concatenate([np.where(own[ids, 0] == c, rhs[ids], 0.0), rhs[nf + off[c]:nf + off[c + 1]]])
        rhat.append(r)
        cons.append([(u, lam_of[j], 1.0 if own[j, 0] == c else -1.0) for u, j in enumerate(ids) if lam_of[j] >= 0])
    H = np.zeros((nlam, nlam))
    xi = np.zeros(nlam)
    for c in range(lev.n_cells):
        x0 = inv[c] @ rhat[c]
        for (u, l, s) in cons[c]:
            xi[l] += s * x0[u]
            for (v, l2, s2) in cons[c]:
                H[l, l2] += s * s2 * inv[c][u, v]
    if nlam == 0:
        lam, it = np.zeros(0), 0
    elif k is None:
        lam, it = np.linalg.solve(H, xi), 0
    else:
        d = 1.0 / np.diag(H)
        lam = np.zeros(nlam)
        r = xi.copy()
        z = d * r
        q = z.copy()
        rz = r @ z
        stop = tol * tol * (xi @ xi)
        it = 0
        while it < k and r @ r > 0.0 and r @ r > stop:
            Hq = H @ q
            qHq = q @ Hq
            if not qHq > 0.0:  # the residual vanished to rounding: the iterate is the solution
                break
            alpha = rz / qHq
            lam += alpha * q
            r -= alpha * Hq
            z = d * r
            rz_new = r @ z
            q = z + (rz_new / rz) * q
            rz = rz_new
            it += 1
    dx = np.zeros(nf + lev.n_p)
    for c in range(lev.n_cells):
        rc = rhat[c].copy()
        for (u, l, s) in cons[c]:
            rc[u] -= s * lam[l]
        xc = inv[c] @ rc
        ids = lev.loc[c]
        first = own[ids, 0] == c
        dx[ids[first]] = xc[:ids.size][first]
        dx[nf + off[c]:nf + off[c + 1]] = xc[ids.size:]
    return dx, it
