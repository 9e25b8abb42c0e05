"""Linear multigrid preconditioner for the level-0 linear systems, in FP64 (oracle; test only).

Sec. 3.4: the paper solves the fine-level systems of its Picard and Newton steps with Krylov methods preconditioned
by AMG (BoomerAMG on the Schur complement S = D diag(M)^-1 E of eq. general-block-system). On the TPFA fine level M is
diagonal, so for the Picard step S is exactly the frozen TPFA matrix A of the reduced system. This build replaces AMG
by one linear V-cycle on the pressure spaces of the spectral hierarchy itself (the coarse spaces the FAS cycles use):
  * operators: A_0 = the frozen TPFA matrix, A_{l+1} = P_l^T A_l P_l with P_l = (P_p)^l_{l+1} (Galerkin products);
  * smoother on level l < L-1: `degree` steps of Chebyshev iteration for A_l x = b from x = 0, preconditioned by
    D_l^-1, with D_0 = diag(A_0) and D_l (l >= 1) the block diagonal of A_l over the pressure unknowns of each
    coarse cell; the Chebyshev interval is [lam / alpha, lam], lam = max_i sum_j |(D_l^-1 A_l)_ij|, a Gershgorin
    bound of the largest eigenvalue of D_l^-1 A_l (whose eigenvalues are real and positive);
  * V-cycle on level l: x = smooth(b); x += P_l Vcycle_{l+1}(P_l^T (b - A_l x)); x = smooth continued from x; the
    coarsest level is solved exactly;
  * levels: the hierarchy the FAS cycles use, coarsened further for the preconditioner alone when its coarsest level
    is large (extended_options: up to four more steps, aggregates of agg_size[l] cells (8 unless given), the last
    FAS step's modes, one flux unknown per interface), cut at the first level whose cell count times its largest
    mode count is at most MAX_COARSE (levels_for). Pre- and post-smoothing are the same polynomial, so the cycle is a symmetric
    positive definite operator B ~ A_0^-1 (the smoother converges in the energy norm: the interval covers the
    spectrum's top).
Chebyshev iteration (the three-term recurrence for the shifted and scaled Chebyshev polynomials on [lmin, lmax]):
theta = (lmax + lmin) / 2, delta = (lmax - lmin) / 2, sigma = theta / delta; rho_0 = 1 / sigma,
d_0 = D^-1 (b - A x) / theta, x += d_0; for k >= 1: rho_k = 1 / (2 sigma - rho_{k-1}),
d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) D^-1 (b - A x), x += d_k.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

ALPHA = 4.0       # Chebyshev interval [lam / ALPHA, lam]
DEGREES = (2, 2)  # smoothing steps before and after the coarse correction: level 0, levels >= 1
MAX_COARSE = 128  # the coarsest level the V-cycle solves directly has at most this many pressure unknowns (padded
                  # to the largest mode count of the level)


@dataclass
class MGLevel:
    A: sp.csr_matrix
    Dinv: sp.csr_matrix        # inverse of the (block) diagonal D_l
    lam: float                 # Gershgorin bound of the largest eigenvalue of D_l^-1 A_l


def _block_diag_inverse(A, blocks):
    """Inverse of the block diagonal of A over the index blocks (lists of indices)."""
    rows, cols, vals = [], [], []
    Ad = A.tocsr()
    for idx in blocks:
        B = Ad[idx][:, idx].toarray()
        Bi = np.linalg.inv(B)
        r, c = np.meshgrid(idx, idx, indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(Bi.ravel())
    n = A.shape[0]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def extended_options(opts):
    """Hierarchy options with the preconditioner's extra coarsening steps (module docstring)."""
    o = dict(opts)
    nl = int(opts["n_levels"])
    total = min(8, nl + 4)
    agg = list(opts["agg_size"]) + [8] * 8
    modes = list(opts["modes"]) + [2] * 8
    mf = list(opts.get("flux_modes", [1] * 8)) + [1] * 8
    mlast = modes[nl - 2] if nl >= 2 else modes[0]
    for l in range(max(nl - 1, 0), 8):
        agg[l] = agg[l] if agg[l] >= 2 else 8
        modes[l] = max(1, min(8, mlast))
        mf[l] = 1
    o.update(n_levels=total, agg_size=agg[:8], modes=modes[:8], flux_modes=mf[:8])
    return o


def levels_for(H):
    """The number of levels of H the V-cycle uses: the first level whose cells times largest mode count is at most
    MAX_COARSE ends it (0 if none)."""
    for L in range(2, len(H.levels) + 1):
        lev = H.levels[L - 1]
        if lev.n_cells * int(np.max(lev.m)) <= MAX_COARSE:
            return L
    return 0


def build(A0, H, n_levels=None):
    """The V-cycle's levels on the hierarchy H (oracle.hierarchy.Hierarchy) for the fine matrix A0; n_levels caps the
    number of levels (default: all of H)."""
    L = len(H.levels) if n_levels is None else min(n_levels, len(H.levels))
    levels = []
    A = sp.csr_matrix(A0, dtype=np.float64)
    for l in range(L):
        if l == 0:
            Dinv = sp.diags(1.0 / A.diagonal()).tocsr()
        else:
            lev = H.levels[l]
            off = lev.p_off
            Dinv = _block_diag_inverse(A, [np.arange(off[c], off[c + 1]) for c in range(lev.n_cells)])
        lam = float(np.max(np.abs(Dinv @ A).sum(axis=1)))
        levels.append(MGLevel(A, Dinv, lam))
        if l + 1 < L:
            P = H.transfers[l].Pp
            A = (P.T @ A @ P).tocsr()
    return levels


def chebyshev(lv, b, x, degree, alpha=ALPHA):
    """`degree` Chebyshev steps for lv.A x = b from x, preconditioned by lv.Dinv (module docstring)."""
    lmax = lv.lam
    lmin = lmax / alpha
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = x.copy()
    d = (lv.Dinv @ (b - lv.A @ x)) / theta
    x += d
    for _ in range(1, degree):
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (lv.Dinv @ (b - lv.A @ x))
        x += d
        rho = rho_new
    return x


def vcycle(levels, H, b, l=0, degrees=DEGREES, alpha=ALPHA):
    """B b: one V-cycle from level l for A_l x = b (module docstring)."""
    lv = levels[l]
    if l == len(levels) - 1:
        return np.linalg.solve(lv.A.toarray(), b)
    deg = degrees[0] if l == 0 else degrees[1]
    x = chebyshev(lv, b, np.zeros(b.size), deg, alpha)
    P = H.transfers[l].Pp
    x = x + P @ vcycle(levels, H, P.T @ (b - lv.A @ x), l + 1, degrees, alpha)
    return chebyshev(lv, b, x, deg, alpha)


def pcg(A, b, apply_B, k, tol=0.0, w=None):
    """At most k steps of preconditioned CG for A x = b from x = 0 (preconditioner apply_B), stopping once
    ||w (b - A x)|| <= tol ||w b|| (w = 1 by default; the level-0 solves use w = diag(A)^-1/2, the scaled residual of
    their Jacobi-preconditioned CG); returns (x, steps). Flexible form: beta = (r_new, z_new - z_old) / (r_old, z_old)
    (equal to the plain form for a fixed linear preconditioner)."""
    w = np.ones(b.size) if w is None else w
    x = np.zeros(b.size)
    r = b.copy()
    z = apply_B(r)
    p = z.copy()
    rz = r @ z
    stop = tol * tol * ((w * b) @ (w * b))
    it = 0
    while it < k and (w * r) @ (w * r) > stop:
        q = A @ p
        pq = p @ q
        if not pq > 0.0:
            break
        alpha = rz / pq
        x += alpha * p
        r_new = r - alpha * q
        z_new = apply_B(r_new)
        beta = (r_new @ (z_new - z)) / rz
        rz = r_new @ z_new
        r, z = r_new, z_new
        p = z + beta * p
        it += 1
    return x, it
