"""Backtracking (Algorithm 1), smoothers and the FAS V-cycle (Algorithm 2) in FP64 (oracle; test only).

Level 0 is evaluated in the equivalent reduced cell-centred form (Remark after eq. FV_matrix): its state is p, the
flux is the TPFA flux sigma(p) (eq. TPFA_flux), so the flux rows of the mixed fine residual vanish and the mixed
residual is [0; -R(p)]. Coarse levels are mixed, with the operators of oracle.coarse.

Algorithm 2, per level l (l = 0 finest):
  coarsest: up to `coarsest_steps` Picard smoothing steps, stopping once that level's residual is below
            `coarsest_tol` (default: the relative tolerance of the outer solve) times its initial value, or below
            the absolute tolerance;
  otherwise: pre-smooth; x^{l+1} = Q x^l; b^{l+1} = A^{l+1}(x^{l+1}) - R (A^l(x^l) - b^l) with R = P^T
            (eq. coarse_level_residual); recurse; x^l = Backtracking(x^l, P (y^{l+1} - x^{l+1})); post-smooth.
Smoothing on level 0 is, by default, one Picard step (Sec. 3.3.1): the frozen-coefficient system
A(kappa(p_k)) dp = -R(p_k), which is the mixed Picard system of eq. picardian_system with the diagonal M eliminated.
The alternative smoother ("jacobi") is nu damped nonlinear (point-Newton) Jacobi sweeps
p_K <- p_K - omega R_K / J~_KK with J~_KK = max(dR_K/dp_K, d_K / 2), d_K the frozen-coefficient diagonal.
The smoother "picard_newton" takes the Picard step while ||R(p_k)|| > newton_switch ||R(p_0)|| (p_0 the iterate the
solve started from) and a Newton step afterwards (Sec. 3.3.2 on level 0): J(p_k) dp = -R(p_k) with the exact
Jacobian of the reduced TPFA residual (the reduced form of eq. jacobian_system). A Newton step that leaves more than
NEWTON_KEEP = 1/2 of the residual it started from shows that the iterate is outside Newton's region of fast
convergence: the rest of the solve then takes Picard steps (the switch is not tried again).
Every update then passes through the pressure-change clamp (Sec. 4.1: max |dp| <= dp_clamp) and Algorithm 1. Smoothing on coarse levels is one Picard
step (Sec. 3.3.1) followed by the clamp (applied to the aggregate means Pi~ dp) and Algorithm 1; with the option
coarse_smoother = "newton" it is one Newton step instead (Sec. 3.3.2, Props. 2-3: the Jacobian of the coarse operator
assembled without visiting finer levels), with the same clamp and Algorithm 1.
Residual comparisons in Algorithm 1 use the Euclidean norm of the level residual, with a strict ">".
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse.linalg as spla

from . import coarse, newton, tpfa

NEWTON_KEEP = 0.5     # a Newton smoothing step must reduce the residual at least this much, else Picard from then on


def backtracking(res_norm, x, dx, r_x, nmax, theta):
    """Algorithm 1. res_norm(x) -> ||r(x)||; r_x = ||r(x)||. Returns (x + s dx, ||r(x + s dx)||, s, n).

    The algorithm presumes finite residual norms: a trial whose norm is not finite counts as +infinity, and if the
    trial it would return is not finite, x is returned unchanged (s = 0)."""
    fin = lambda v: v if np.isfinite(v) else np.inf
    s = 1.0
    n = 0
    r_s = fin(res_norm(x + s * dx))
    while r_s > r_x and n < nmax:
        r_half = fin(res_norm(x + 0.5 * s * dx))
        if r_half > theta * r_s:
            break
        s *= 0.5
        n += 1
        r_s = r_half
    if not np.isfinite(r_s):
        return x, r_x, 0.0, n
    return x + s * dx, r_s, s, n


def level_params(H, mesh, kind, a):
    """The nonlinearity's parameter on every level: `a` itself, except for the Richards kind, whose cell heights are
    carried to the coarse levels as volume-weighted aggregate means (the averaging of Pi~ p, eq. pwc_projector)."""
    L = len(H.levels)
    if kind != tpfa.KAPPA_RICHARDS:
        return [a] * L
    out = [a]
    z = np.asarray(a.z, dtype=np.float64)
    vol = np.asarray(mesh.cell_volume, dtype=np.float64)
    for l in range(L - 1):
        agg = H.transfers[l].agg_of
        na = int(agg.max()) + 1
        vz = np.bincount(agg, weights=vol * z, minlength=na)
        vol = np.bincount(agg, weights=vol, minlength=na)
        z = vz / vol
        out.append(tpfa.RichardsParams(a.alpha, a.beta, z))
    return out


@dataclass
class Stats:
    cycles: int = 0
    history: list = field(default_factory=list)
    early_exit: bool = False
    fine_evals: int = 0
    newton_steps: int = 0
    coarse_newton_steps: int = 0


class FAS:
    """FAS solver over an oracle hierarchy for one problem (mesh, kappa, data, options)."""

    def __init__(self, H, mesh, kind, a, f_cell, g_face, opts):
        self.H, self.mesh, self.kind, self.a = H, mesh, kind, a
        self.f, self.g, self.o = f_cell, g_face, opts
        self.dofs = tpfa.flux_dofs(mesh)
        self.stats = Stats()
        self.a_lev = level_params(H, mesh, kind, a)
        self.r0_ref = 0.0         # ||R(p_0)|| of the current solve (set by vcycle; 0: no Newton step)
        self.newton_off = False   # set once a Newton step reduced the residual by less than NEWTON_KEEP
        self.coarse_newton_now = False   # coarse_smoother = "picard_newton": Newton on the coarse levels this cycle

    # ---- level 0 (reduced form) --------------------------------------------------------------------------------
    def R(self, p):
        self.stats.fine_evals += 1
        return tpfa.reduced_residual(self.mesh, self.kind, self.a, p, self.f, self.g)

    def Rnorm(self, p):
        return float(np.linalg.norm(self.R(p)))

    def jacobi_diag(self, p):
        J = tpfa.reduced_jacobian(self.mesh, self.kind, self.a, p, self.g).diagonal()
        d = tpfa.picard_diagonal(self.mesh, self.kind, self.a, p)
        return np.maximum(J, 0.5 * d)

    def picard_matrix0(self, p):
        """The frozen-coefficient TPFA matrix A(kappa(p)) with A(kappa(p)) p - rhs(kappa(p)) = R(p)."""
        return newton.picard_matrix(self.mesh, self.kind, self.a, p)

    def newton_update0(self, p, Rp=None):
        """The level-0 Newton update: dp solving J(p) dp = -R(p), J the exact Jacobian of R (Sec. 3.3.2)."""
        Rp = self.R(p) if Rp is None else Rp
        J = tpfa.reduced_jacobian(self.mesh, self.kind, self.a, p, self.g).tocsc()
        return -spla.spsolve(J, Rp)

    def use_newton0(self, r_p):
        """picard_newton: Newton once ||R(p_k)|| <= newton_switch ||R(p_0)|| (r0_ref, set by the cycle)."""
        o = self.o
        return (o.get("smoother", "picard") == "picard_newton" and not self.newton_off
                and r_p <= o.get("newton_switch", 1e-3) * self.r0_ref)

    def smooth0(self, p, nu, r_p=None):
        """One smoothing step on level 0: a Picard step (Sec. 3.3.1, default), a Newton step (picard_newton, once
        the residual is below newton_switch times the initial one and while no Newton step of the solve has failed
        to halve the residual) or nu nonlinear Jacobi sweeps."""
        o = self.o
        smoother = o.get("smoother", "picard")
        newton_step = False
        if smoother in ("picard", "picard_newton"):
            Rp = self.R(p)
            r_p = float(np.linalg.norm(Rp)) if r_p is None else r_p
            newton_step = self.use_newton0(r_p)
            if newton_step:
                dp = self.newton_update0(p, Rp)
                self.stats.newton_steps += 1
            else:
                dp = -spla.spsolve(self.picard_matrix0(p).tocsc(), Rp)
        else:
            q = p.copy()
            for _ in range(nu):
                q = q - o["omega"] * self.R(q) / self.jacobi_diag(q)
            dp = q - p
        mx = np.max(np.abs(dp)) if dp.size else 0.0
        if o["dp_clamp"] > 0 and mx > o["dp_clamp"]:
            dp = dp * (o["dp_clamp"] / mx)
        r_p = self.Rnorm(p) if r_p is None else r_p
        pn, rn, _, _ = backtracking(self.Rnorm, p, dp, r_p, o["bt_nmax"], o["bt_theta"])
        if newton_step and not rn <= NEWTON_KEEP * r_p:
            self.newton_off = True
        return pn, rn

    def sigma0(self, p):
        return tpfa.face_fluxes(self.mesh, self.kind, self.a, p, self.g)[self.dofs]

    # ---- coarse levels (mixed) ---------------------------------------------------------------------------------
    def split(self, l, x):
        nf = self.H.levels[l].n_flux
        return x[:nf], x[nf:]

    def res(self, l, x, b):
        lev = self.H.levels[l]
        s, p = self.split(l, x)
        return coarse.operator(lev, self.kind, self.a_lev[l], s, p) - b

    def picard_smooth(self, l, x, b, r_x=None):
        lev = self.H.levels[l]
        o = self.o
        s, p = self.split(l, x)
        sP, pP = coarse.picard_solve(lev, self.kind, self.a_lev[l], s, p, b)
        dx = np.concatenate([sP, pP]) - x
        if o["dp_clamp"] > 0:
            mx = np.max(np.abs(coarse.pbar(lev, dx[lev.n_flux:])))
            if mx > o["dp_clamp"]:
                dx = dx * (o["dp_clamp"] / mx)
        nrm = lambda y: float(np.linalg.norm(self.res(l, y, b)))
        r_x = nrm(x) if r_x is None else r_x
        xn, rn, _, _ = backtracking(nrm, x, dx, r_x, o["bt_nmax"], o["bt_theta"])
        return xn, rn

    def newton_smooth(self, l, x, b, r_x=None):
        """One coarse Newton smoothing step (Sec. 3.3.2 on level l >= 1): the update of eq. jacobian_system with the
        Jacobian of Props. 2-3 (oracle.coarse.jacobian), then the clamp on Pi~ dp and Algorithm 1, as for Picard."""
        lev = self.H.levels[l]
        o = self.o
        s, p = self.split(l, x)
        dx = coarse.newton_update(lev, self.kind, self.a_lev[l], s, p, b)
        self.stats.coarse_newton_steps += 1
        if o["dp_clamp"] > 0:
            mx = np.max(np.abs(coarse.pbar(lev, dx[lev.n_flux:])))
            if mx > o["dp_clamp"]:
                dx = dx * (o["dp_clamp"] / mx)
        nrm = lambda y: float(np.linalg.norm(self.res(l, y, b)))
        r_x = nrm(x) if r_x is None else r_x
        xn, rn, _, _ = backtracking(nrm, x, dx, r_x, o["bt_nmax"], o["bt_theta"])
        return xn, rn

    def coarse_smooth(self, l, x, b, r_x=None):
        """The coarse smoothing step: Picard (default); with coarse_smoother = "newton", Newton (FAS-Newton on every
        coarse level, Sec. 3.3.2); with "picard_newton", Newton once the level-0 smoother has switched to Newton
        steps in this cycle (the fine residual below newton_switch times the initial one, no failed Newton step)."""
        cs = self.o.get("coarse_smoother", "picard")
        if cs == "newton" or (cs == "picard_newton" and self.coarse_newton_now):
            return self.newton_smooth(l, x, b, r_x)
        return self.picard_smooth(l, x, b, r_x)

    def coarsest(self, l, x, b):
        o = self.o
        r = float(np.linalg.norm(self.res(l, x, b)))
        r0 = r
        rel = o.get("coarsest_tol", 0.0) or o["tol_rel"]
        for _ in range(o["coarsest_steps"]):
            if r <= rel * r0 or r <= o["tol_abs"]:
                break
            x, r = self.coarse_smooth(l, x, b, r)
        return x

    def cycle_coarse(self, l, x, b):
        """Algorithm 2 on a mixed level l >= 1."""
        if l == len(self.H.levels) - 1:
            return self.coarsest(l, x, b)
        lev, tr, levc = self.H.levels[l], self.H.transfers[l], self.H.levels[l + 1]
        x, _ = self.coarse_smooth(l, x, b)
        s, p = self.split(l, x)
        r = self.res(l, x, b)
        rs, rp = r[:lev.n_flux], r[lev.n_flux:]
        xc = np.concatenate([tr.Qsigma @ s, tr.Qp @ p])
        bc = coarse.operator(levc, self.kind, self.a_lev[l + 1], xc[:levc.n_flux], xc[levc.n_flux:]) \
            - np.concatenate([tr.Psigma.T @ rs, tr.Pp.T @ rp])
        yc = self.cycle_coarse(l + 1, xc, bc)
        e = yc - xc
        dx = np.concatenate([tr.Psigma @ e[:levc.n_flux], tr.Pp @ e[levc.n_flux:]])
        nrm = lambda y: float(np.linalg.norm(self.res(l, y, b)))
        x, _, _, _ = backtracking(nrm, x, dx, nrm(x), self.o["bt_nmax"], self.o["bt_theta"])
        x, _ = self.coarse_smooth(l, x, b)
        return x

    def vcycle(self, p, r0):
        """One Algorithm 2 cycle from level 0. Returns (p, ||R(p)||, stopped_after_presmoothing)."""
        o = self.o
        H = self.H
        self.r0_ref = r0
        p, rn = self.smooth0(p, o["nu_pre"])
        if rn <= o["tol_rel"] * r0 or rn <= o["tol_abs"]:
            return p, rn, True
        self.coarse_newton_now = (not self.newton_off and rn <= o.get("newton_switch", 1e-3) * r0)
        if len(H.levels) == 1:
            p, rn = self.smooth0(p, o["nu_post"], rn)
            return p, rn, False
        tr, levc = H.transfers[0], H.levels[1]
        Rp = self.R(p)
        xc = np.concatenate([tr.Qsigma @ self.sigma0(p), tr.Qp @ p])
        # mixed fine residual is [0; -R(p)]; R r^0 = [0; P_p^T (-R(p))]
        bc = coarse.operator(levc, self.kind, self.a_lev[1], xc[:levc.n_flux], xc[levc.n_flux:]) \
            - np.concatenate([np.zeros(levc.n_flux), tr.Pp.T @ (-Rp)])
        yc = self.cycle_coarse(1, xc, bc)
        dp = tr.Pp @ (yc - xc)[levc.n_flux:]
        p, rn, _, _ = backtracking(self.Rnorm, p, dp, float(np.linalg.norm(Rp)), o["bt_nmax"], o["bt_theta"])
        p, rn = self.smooth0(p, o["nu_post"], rn)
        return p, rn, False

    def cascade(self, p):
        """Nonlinear cascadic start (Sec. 4.2, Example 2): the FAS coarse problems of Algorithm 2 are formed top-down
        at the current iterate; then, from the coarsest level up, each is solved nonlinearly by Picard smoothing steps
        (at most `coarsest_steps`, stopping like the coarsest solve of a cycle: `coarsest_tol`, else the relative
        tolerance of the solve) from the point its finer level
        projected, and its correction is carried to the finer level with Algorithm 1. Returns the new level-0
        iterate."""
        o, H = self.o, self.H
        L = len(H.levels)
        if L == 1:
            return p
        xs, bs, x0s = [None] * L, [None] * L, [None] * L
        tr, levc = H.transfers[0], H.levels[1]
        Rp = self.R(p)
        xs[1] = np.concatenate([tr.Qsigma @ self.sigma0(p), tr.Qp @ p])
        bs[1] = coarse.operator(levc, self.kind, self.a_lev[1], xs[1][:levc.n_flux], xs[1][levc.n_flux:]) \
            - np.concatenate([np.zeros(levc.n_flux), tr.Pp.T @ (-Rp)])
        for l in range(1, L - 1):
            lev, tr, levc = H.levels[l], H.transfers[l], H.levels[l + 1]
            s, q = self.split(l, xs[l])
            r = self.res(l, xs[l], bs[l])
            xs[l + 1] = np.concatenate([tr.Qsigma @ s, tr.Qp @ q])
            bs[l + 1] = coarse.operator(levc, self.kind, self.a_lev[l + 1], xs[l + 1][:levc.n_flux],
                                        xs[l + 1][levc.n_flux:]) \
                - np.concatenate([tr.Psigma.T @ r[:lev.n_flux], tr.Pp.T @ r[lev.n_flux:]])
        for l in range(1, L):
            x0s[l] = xs[l].copy()

        rel = o.get("coarsest_tol", 0.0) or o["tol_rel"]   # each level stops like the coarsest solve of a cycle

        def solve_level(l, x, b):
            r = float(np.linalg.norm(self.res(l, x, b)))
            r_in = r
            for _ in range(o["coarsest_steps"]):
                if r <= rel * r_in or r <= o["tol_abs"]:
                    break
                x, r = self.coarse_smooth(l, x, b, r)
            return x

        ys = [None] * L
        ys[L - 1] = solve_level(L - 1, xs[L - 1], bs[L - 1])
        for l in range(L - 2, 0, -1):
            tr, levc = H.transfers[l], H.levels[l + 1]
            e = ys[l + 1] - x0s[l + 1]
            dx = np.concatenate([tr.Psigma @ e[:levc.n_flux], tr.Pp @ e[levc.n_flux:]])
            nrm = lambda y, l=l: float(np.linalg.norm(self.res(l, y, bs[l])))
            x, _, _, _ = backtracking(nrm, xs[l], dx, nrm(xs[l]), o["bt_nmax"], o["bt_theta"])
            ys[l] = solve_level(l, x, bs[l])
        tr, levc = H.transfers[0], H.levels[1]
        dp = tr.Pp @ (ys[1] - x0s[1])[levc.n_flux:]
        p, _, _, _ = backtracking(self.Rnorm, p, dp, float(np.linalg.norm(Rp)), o["bt_nmax"], o["bt_theta"])
        return p

    def solve(self, p0=None, max_cycles=None, cascadic=False):
        """FAS cycles (Algorithm 2) from p0 until the relative / absolute tolerance; with cascadic=True the cycles
        start from the nonlinear cascadic iterate (cascade), the tolerance still relative to ||R(p0)||."""
        o = self.o
        p = np.zeros(self.mesh.n_cells) if p0 is None else np.array(p0, dtype=np.float64)
        self.newton_off = False
        r0 = self.Rnorm(p)
        if cascadic:
            p = self.cascade(p)
        rn = self.Rnorm(p)
        self.stats.history = [r0, rn] if cascadic else [r0]
        maxc = o["max_cycles"] if max_cycles is None else max_cycles
        for _ in range(maxc):
            if rn <= o["tol_rel"] * r0 or rn <= o["tol_abs"]:
                break
            p, rn, early = self.vcycle(p, r0)
            self.stats.cycles += 1
            self.stats.history.append(rn)
            if early:
                self.stats.early_exit = True
                break
        return p
