"""Thin ctypes binding of libnlmg.so (include/nlmg.h): argument marshalling only, every step runs in the library.

The library is built in-tree by paper_2005_01275_gb300.build; importing this module without it raises, there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libnlmg.so")

OK, EINVAL, ENOMEM, ENOCONV, EDIVERGED, ETIMEOUT, ECUDA, EUNSUPPORTED = range(8)
KAPPA_EXP, KAPPA_INV1P2 = 0, 1
SMOOTH_PICARD, SMOOTH_JACOBI, SMOOTH_PICARD_NEWTON = 0, 1, 2
_SMOOTHERS = {"picard": SMOOTH_PICARD, "jacobi": SMOOTH_JACOBI, "picard_newton": SMOOTH_PICARD_NEWTON}
PROJECT, RESTRICT, PROLONG = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOCONV", 4: "EDIVERGED", 5: "ETIMEOUT", 6: "ECUDA",
                7: "EUNSUPPORTED"}


class Mesh(C.Structure):
    _fields_ = [("n_cells", C.c_int32), ("cell_volume", C.POINTER(C.c_double)), ("n_faces", C.c_int32),
                ("face_cells", C.POINTER(C.c_int32)), ("half_trans", C.POINTER(C.c_double)),
                ("face_bc", C.POINTER(C.c_uint8)), ("face_area", C.POINTER(C.c_double))]


class Kappa(C.Structure):
    _fields_ = [("kind", C.c_int32), ("a", C.c_double)]


class Options(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("agg_size", C.c_int32 * 8), ("modes", C.c_int32 * 8),
                ("smoother", C.c_int32), ("nu_pre", C.c_int32), ("nu_post", C.c_int32), ("omega", C.c_double),
                ("bt_nmax", C.c_int32), ("bt_theta", C.c_double), ("dp_clamp", C.c_double),
                ("coarsest_steps", C.c_int32), ("coarsest_tol", C.c_double), ("lin_tol", C.c_double),
                ("lin_maxit", C.c_int32),
                ("coarse_lin_tol", C.c_double), ("lin_precision", C.c_int32),
                ("setup_threads", C.c_int32), ("max_sms", C.c_int32), ("newton_switch", C.c_double),
                ("newton_lin_tol", C.c_double), ("coarsest_lin_tol", C.c_double), ("flux_modes", C.c_int32 * 8),
                ("cascadic", C.c_int32), ("lin_precond", C.c_int32), ("mg_row_cells", C.c_int32),
                ("reserved", C.c_int32 * 2)]


class Report(C.Structure):
    _fields_ = [("cycles", C.c_int32), ("early_exit", C.c_int32), ("res0", C.c_double), ("res", C.c_double),
                ("solve_ms", C.c_double), ("fine_evals", C.c_int64), ("lin_iters", C.c_int64),
                ("kernel_launches", C.c_int64), ("lin_iters_level", C.c_int64 * 8),
                ("tol_tightened", C.c_int32), ("newton_steps", C.c_int32), ("history_len", C.c_int32),
                ("history", C.c_double * 64)]

    def as_dict(self):
        return dict(cycles=self.cycles, early_exit=bool(self.early_exit), res0=self.res0, res=self.res,
                    solve_ms=self.solve_ms, fine_evals=self.fine_evals, lin_iters=self.lin_iters,
                    kernel_launches=self.kernel_launches, lin_iters_level=list(self.lin_iters_level),
                    tol_tightened=self.tol_tightened, newton_steps=self.newton_steps,
                    history=list(self.history[:self.history_len]))


class ServerOptions(C.Structure):
    _fields_ = [("max_inflight", C.c_int32), ("mem_budget_bytes", C.c_size_t),
                ("setup_threads_per_request", C.c_int32), ("hierarchy_cache", C.c_int32)]


class RequestTimes(C.Structure):
    _fields_ = [("queue_ms", C.c_double), ("setup_ms", C.c_double), ("solve_ms", C.c_double),
                ("latency_ms", C.c_double), ("hierarchy_reused", C.c_int32)]


class LevelInfo(C.Structure):
    _fields_ = [("n_cells", C.c_int32), ("n_flux", C.c_int32), ("n_p", C.c_int32), ("n_lambda", C.c_int32),
                ("eig_host", C.c_int32)]


_lib = None

# every exported symbol of include/nlmg.h with (restype, argtypes)
_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int32)
SIGNATURES = {
    "nlmg_default_options": (None, [C.POINTER(Options)]),
    "nlmg_setup": (C.c_int, [C.POINTER(Mesh), C.POINTER(Kappa), C.POINTER(Options), C.POINTER(_P)]),
    "nlmg_setup_host": (C.c_int, [C.POINTER(Mesh), C.POINTER(Kappa), C.POINTER(Options), C.POINTER(_P)]),
    "nlmg_instance": (C.c_int, [_P, C.POINTER(Kappa), C.POINTER(_P)]),
    "nlmg_solve_many": (C.c_int, [_P, C.c_int32, _D, _D, _D, C.c_double, C.c_double, C.c_int32, C.c_int32, _D,
                                  C.POINTER(Report), _I]),
    "nlmg_solve_many_device": (C.c_int, [_P, C.c_int32, _P, _P, _P, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                         _P, C.POINTER(Report), _I]),
    "nlmg_set_options": (C.c_int, [_P, C.POINTER(Options)]),
    "nlmg_tune_sm_share": (C.c_int, [_P, C.c_int32, _D, _D, _I, _D]),
    "nlmg_set_data": (C.c_int, [_P, _D, _D]),
    "nlmg_solve": (C.c_int, [_P, _D, _D, _D, C.c_double, C.c_double, C.c_int32, _D, C.POINTER(Report)]),
    "nlmg_solve_device": (C.c_int, [_P, _P, _P, _P, C.c_double, C.c_double, C.c_int32, _P, C.POINTER(Report)]),
    "nlmg_solve_picard": (C.c_int, [_P, _D, _D, _D, C.c_double, C.c_double, C.c_int32, _D, C.POINTER(Report)]),
    "nlmg_solve_newton": (C.c_int, [_P, _D, _D, _D, C.c_double, C.c_double, C.c_int32, _D, C.POINTER(Report)]),
    "nlmg_fine_residual": (C.c_int, [_P, _D, _D]),
    "nlmg_fine_flux": (C.c_int, [_P, _D, _D]),
    "nlmg_level_apply": (C.c_int, [_P, C.c_int32, _D, _D]),
    "nlmg_transfer": (C.c_int, [_P, C.c_int32, C.c_int32, _D, _D]),
    "nlmg_picard_update": (C.c_int, [_P, C.c_int32, _D, _D, _D, _I]),
    "nlmg_newton_update": (C.c_int, [_P, _D, _D, _I]),
    "nlmg_precond_apply": (C.c_int, [_P, _D, _D, _D]),
    "nlmg_vcycle": (C.c_int, [_P, _D, C.c_double, _D, _D, _I]),
    "nlmg_level_info_get": (C.c_int, [_P, C.c_int32, C.POINTER(LevelInfo)]),
    "nlmg_get_aggregates": (C.c_int, [_P, C.c_int32, _I, _I]),
    "nlmg_get_transfer_dense": (C.c_int, [_P, C.c_int32, C.c_int32, _D]),
    "nlmg_server_default_options": (None, [C.POINTER(ServerOptions)]),
    "nlmg_server_create": (C.c_int, [C.POINTER(ServerOptions), C.POINTER(_P)]),
    "nlmg_server_submit": (C.c_int, [_P, C.POINTER(Mesh), C.POINTER(Kappa), C.POINTER(Options), _D, _D, C.c_double,
                                     C.c_double, C.c_int32, C.POINTER(C.c_uint64)]),
    "nlmg_server_poll": (C.c_int, [_P, C.c_uint64, C.c_int32, _D, C.POINTER(Report), C.POINTER(RequestTimes)]),
    "nlmg_server_destroy": (None, [_P]),
    "nlmg_profile": (C.c_int, [_P, C.c_int32]),
    "nlmg_profile_read": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int64), _D, _D, _D]),
    "nlmg_fine_residual_noalloc": (C.c_int, [_P, _P, _P, _P, _P]),
    "nlmg_measure_fp64": (C.c_int, [_D]),
    "nlmg_device_bytes": (C.c_int, [_P, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "nlmg_check_grid_barrier": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int64, _I]),
    "nlmg_server_request_bytes": (C.c_int, [C.POINTER(Mesh), C.POINTER(C.c_size_t)]),
    "nlmg_last_error": (C.c_char_p, [_P]),
    "nlmg_destroy": (None, [_P]),
}


def lib():
    """Load libnlmg.so (raises if it has not been built: there is no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libnlmg.so is not built: run paper_2005_01275_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class NlmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def _dp(a):
    return a.ctypes.data_as(_D)


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def default_options(**kw):
    o = Options()
    lib().nlmg_default_options(C.byref(o))
    for k, v in kw.items():
        if k in ("agg_size", "modes", "flux_modes"):
            arr = getattr(o, k)
            for i, x in enumerate(v[:8]):
                arr[i] = int(x)
        else:
            setattr(o, k, v)
    return o


def options_from_dict(d):
    """Options from the dictionary used by the synthetic problem configurations."""
    keep = {k: d[k] for k in ("n_levels", "agg_size", "modes", "nu_pre", "nu_post", "omega", "bt_nmax", "bt_theta",
                              "dp_clamp", "coarsest_steps", "coarsest_tol", "lin_tol", "lin_maxit", "coarse_lin_tol",
                              "lin_precision", "max_sms", "newton_switch", "newton_lin_tol", "coarsest_lin_tol",
                              "setup_threads", "flux_modes", "cascadic", "lin_precond", "mg_row_cells") if k in d}
    if "lin_tol" in d and "coarse_lin_tol" not in d:
        keep["coarse_lin_tol"] = d["lin_tol"]       # one tolerance given: use it on every level
    if "lin_tol" in d and "newton_lin_tol" not in d:
        keep["newton_lin_tol"] = d["lin_tol"]       # ... and for the Newton steps
    if "coarsest_lin_tol" not in d and ("coarse_lin_tol" in keep):
        keep["coarsest_lin_tol"] = keep["coarse_lin_tol"]   # ... and on the coarsest level
    if "smoother" in d:
        keep["smoother"] = _SMOOTHERS[d["smoother"]]
    return default_options(**keep)


class Context:
    """Owns one nlmg_ctx (hierarchy + device buffers)."""

    def __init__(self, mesh, kappa_kind, kappa_a, opts, device=True):
        L = lib()
        self._keep = dict(vol=_f64(mesh.cell_volume), fc=np.ascontiguousarray(mesh.face_cells, dtype=np.int32),
                          ht=_f64(mesh.half_trans), bc=np.ascontiguousarray(mesh.face_bc, dtype=np.uint8),
                          area=_f64(mesh.face_area))
        k = self._keep
        m = Mesh(mesh.n_cells, _dp(k["vol"]), int(k["fc"].shape[0]), k["fc"].ctypes.data_as(_I), _dp(k["ht"]),
                 k["bc"].ctypes.data_as(C.POINTER(C.c_uint8)), _dp(k["area"]))
        self.n_cells = int(mesh.n_cells)
        self.n_faces = int(k["fc"].shape[0])
        if isinstance(opts, dict):
            opts = options_from_dict(opts)
        self.opts = opts
        h = _P()
        fn = L.nlmg_setup if device else L.nlmg_setup_host
        st = fn(C.byref(m), C.byref(Kappa(int(kappa_kind), float(kappa_a))), C.byref(opts), C.byref(h))
        if st != OK:
            raise NlmgError(st, "setup failed: " + L.nlmg_last_error(None).decode())
        self.h = h

    def instance(self, kappa_kind=None, kappa_a=None):
        """A second context sharing this one's device hierarchy (own work buffers and stream)."""
        k = None if kappa_kind is None else C.byref(Kappa(int(kappa_kind), float(kappa_a)))
        h = _P()
        self._check(lib().nlmg_instance(self.h, k, C.byref(h)))
        other = Context.__new__(Context)
        other._keep, other.n_cells, other.n_faces, other.opts = self._keep, self.n_cells, self.n_faces, self.opts
        other._base = self
        other.h = h
        return other

    def set_options(self, **changes):
        """Change solver options (not the hierarchy ones) for the following solves."""
        o = Options.from_buffer_copy(self.opts)
        for k, v in changes.items():
            setattr(o, k, _SMOOTHERS[v] if k == "smoother" and isinstance(v, str) else v)
        self._check(lib().nlmg_set_options(self.h, C.byref(o)))
        self.opts = o

    def tune_sm_share(self, f_rows, g_rows):
        """Times the SM-share candidates on these rows; returns (best max_sms, solves/s per candidate)."""
        f = np.ascontiguousarray(f_rows, dtype=np.float64)
        g = np.ascontiguousarray(g_rows, dtype=np.float64)
        n = f.shape[0]
        best = C.c_int32(0)
        rates = np.zeros(4)
        self._check(lib().nlmg_tune_sm_share(self.h, n, _dp(f), _dp(g), C.byref(best), _dp(rates)))
        return best.value, rates

    def solve_many_device(self, n_rhs, f_ptr, g_ptr, p_ptr, tol_rel=1e-8, tol_abs=1e-10, max_cycles=50, n_streams=0):
        """nlmg_solve_many on device-resident rows (raw device pointers of [n_rhs][n_cells], [n_rhs][n_faces] and
        [n_rhs][n_cells] arrays); returns (list of report dicts, status array, overall status)."""
        reps = (Report * n_rhs)()
        sts = np.zeros(n_rhs, dtype=np.int32)
        st = lib().nlmg_solve_many_device(self.h, int(n_rhs), _P(f_ptr), _P(g_ptr), None, tol_rel, tol_abs,
                                          max_cycles, int(n_streams), _P(p_ptr), reps, sts.ctypes.data_as(_I))
        return [r.as_dict() for r in reps], sts, st

    def solve_many(self, f_rows, g_rows, x0_rows=None, tol_rel=1e-8, tol_abs=1e-10, max_cycles=50, n_streams=0,
                   allow_noconv=False):
        """Independent FAS solves of every row of f_rows [n_rhs, n_cells] / g_rows [n_rhs, n_faces]."""
        f = np.ascontiguousarray(f_rows, dtype=np.float64)
        g = np.ascontiguousarray(g_rows, dtype=np.float64)
        n = f.shape[0]
        if f.shape != (n, self.n_cells) or g.shape != (n, self.n_faces):
            raise ValueError("f_rows must be [n_rhs, n_cells] and g_rows [n_rhs, n_faces]")
        x0 = None if x0_rows is None else np.ascontiguousarray(x0_rows, dtype=np.float64).reshape(n, self.n_cells)
        out = np.zeros((n, self.n_cells))
        reps = (Report * max(n, 1))()
        sts = np.zeros(max(n, 1), np.int32)
        st = lib().nlmg_solve_many(self.h, n, _dp(f), _dp(g), None if x0 is None else _dp(x0), tol_rel, tol_abs,
                                   max_cycles, n_streams, _dp(out), reps, sts.ctypes.data_as(_I))
        if not (st == OK or (allow_noconv and st == ENOCONV)):
            self._check(st)
        return out, [reps[i].as_dict() for i in range(n)], sts[:n].copy()

    def _check(self, st):
        if st not in (OK,):
            raise NlmgError(st, lib().nlmg_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().nlmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- hierarchy export ---------------------------------------------------------------------------------
    def n_levels(self):
        return int(self.opts.n_levels)

    def level_info(self, l):
        out = LevelInfo()
        self._check(lib().nlmg_level_info_get(self.h, l, C.byref(out)))
        return dict(n_cells=out.n_cells, n_flux=out.n_flux, n_p=out.n_p, n_lambda=out.n_lambda,
                    eig_host=out.eig_host)

    def aggregates(self, l):
        nf = self.level_info(l)["n_cells"]
        nc = self.level_info(l + 1)["n_cells"]
        agg = np.zeros(nf, np.int32)
        m = np.zeros(nc, np.int32)
        self._check(lib().nlmg_get_aggregates(self.h, l, agg.ctypes.data_as(_I), m.ctypes.data_as(_I)))
        return agg, m

    def transfer_dense(self, l, which):
        a, b = self.level_info(l), self.level_info(l + 1)
        shape = {0: (a["n_p"], b["n_p"]), 1: (a["n_flux"], b["n_flux"]), 2: (b["n_flux"], a["n_flux"])}[which]
        out = np.zeros(shape)
        self._check(lib().nlmg_get_transfer_dense(self.h, l, which, _dp(out)))
        return out

    # ---- device calls ------------------------------------------------------------------------------------
    def set_data(self, f_cell, g_face):
        self._f = _f64(f_cell, self.n_cells)
        self._g = _f64(g_face, self.n_faces)
        self._check(lib().nlmg_set_data(self.h, _dp(self._f), _dp(self._g)))

    def fine_residual(self, p):
        p = _f64(p, self.n_cells)
        out = np.zeros(self.n_cells)
        self._check(lib().nlmg_fine_residual(self.h, _dp(p), _dp(out)))
        return out

    def fine_flux(self, p):
        p = _f64(p, self.n_cells)
        out = np.zeros(self.level_info(0)["n_flux"])
        self._check(lib().nlmg_fine_flux(self.h, _dp(p), _dp(out)))
        return out

    def _nx(self, l):
        if l == 0:
            return self.n_cells
        i = self.level_info(l)
        return i["n_flux"] + i["n_p"]

    def level_apply(self, l, x):
        x = _f64(x, self._nx(l))
        out = np.zeros_like(x)
        self._check(lib().nlmg_level_apply(self.h, l, _dp(x), _dp(out)))
        return out

    def transfer(self, l, op, vec):
        nin = self._nx(l + 1) if op == PROLONG else self._nx(l)
        nout = self._nx(l) if op == PROLONG else self._nx(l + 1)
        vec = _f64(vec, nin)
        out = np.zeros(nout)
        self._check(lib().nlmg_transfer(self.h, l, op, _dp(vec), _dp(out)))
        return out

    def picard_update(self, l, x, b=None):
        x = _f64(x, self._nx(l))
        b = np.zeros_like(x) if b is None else _f64(b, self._nx(l))
        out = np.zeros_like(x)
        it = C.c_int32(0)
        self._check(lib().nlmg_picard_update(self.h, l, _dp(x), _dp(b), _dp(out), C.byref(it)))
        return out, it.value

    def newton_update(self, p):
        """dx solving J(p) dx = -R(p) (level-0 Newton update by the persistent BiCGStab) and its iterations."""
        p = _f64(p, self.n_cells)
        out = np.zeros_like(p)
        it = C.c_int32(0)
        self._check(lib().nlmg_newton_update(self.h, _dp(p), _dp(out), C.byref(it)))
        return out, it.value

    def precond_apply(self, p, r):
        """z = B r, one V-cycle of the level-0 multigrid preconditioner at the frozen matrix A(kappa(p))."""
        p = _f64(p, self.n_cells)
        r = _f64(r, self.n_cells)
        out = np.zeros_like(p)
        self._check(lib().nlmg_precond_apply(self.h, _dp(p), _dp(r), _dp(out)))
        return out

    def vcycle(self, p, r0):
        p = _f64(p, self.n_cells)
        out = np.zeros_like(p)
        res = C.c_double(0)
        early = C.c_int32(0)
        self._check(lib().nlmg_vcycle(self.h, _dp(p), float(r0), _dp(out), C.byref(res), C.byref(early)))
        return out, res.value, bool(early.value)

    def solve(self, f_cell, g_face, x0=None, tol_rel=1e-8, tol_abs=1e-10, max_cycles=50, picard_only=False,
              allow_noconv=False, newton=False):
        f = _f64(f_cell, self.n_cells)
        g = _f64(g_face, self.n_faces)
        x0a = None if x0 is None else _f64(x0, self.n_cells)
        out = np.zeros(self.n_cells)
        rep = Report()
        fn = lib().nlmg_solve_newton if newton else (lib().nlmg_solve_picard if picard_only else lib().nlmg_solve)
        st = fn(self.h, _dp(f), _dp(g), None if x0a is None else _dp(x0a), tol_rel, tol_abs, max_cycles, _dp(out),
                C.byref(rep))
        if not (st == OK or (allow_noconv and st == ENOCONV)):
            self._check(st)
        return out, rep.as_dict(), st

    def profile(self, enable):
        self._check(lib().nlmg_profile(self.h, 1 if enable else 0))

    def profile_read(self, kernel):
        n = C.c_int64(0)
        ms = C.c_double(0)
        by = C.c_double(0)
        fl = C.c_double(0)
        self._check(lib().nlmg_profile_read(self.h, kernel, C.byref(n), C.byref(ms), C.byref(by), C.byref(fl)))
        return n.value, ms.value, by.value, fl.value

    def solve_ptr(self, f_ptr, g_ptr, p_ptr, tol_rel=1e-8, tol_abs=1e-10, max_cycles=50):
        """Host-pointer solve (e.g. pinned torch tensors): the library copies inputs in and p out."""
        rep = Report()
        st = lib().nlmg_solve(self.h, C.cast(f_ptr, _D), C.cast(g_ptr, _D), None, tol_rel, tol_abs, max_cycles,
                              C.cast(p_ptr, _D), C.byref(rep))
        return rep.as_dict(), st

    def fine_residual_noalloc(self, p_ptr, r_ptr, norm2_ptr, stream_ptr=0):
        """Allocation-free residual on caller device buffers (raw device pointers); enqueued on stream_ptr."""
        st = lib().nlmg_fine_residual_noalloc(self.h, _P(p_ptr), _P(r_ptr), _P(norm2_ptr),
                                               _P(stream_ptr) if stream_ptr else None)
        return st

    def last_error(self):
        return lib().nlmg_last_error(self.h).decode()

    def device_bytes(self):
        """(shared, own) device bytes held by this context."""
        a, b = C.c_size_t(0), C.c_size_t(0)
        self._check(lib().nlmg_device_bytes(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def check_grid_barrier(self, blocks, absent_block, spin_limit):
        """Runs the bounded grid barrier alone (one block may stay away); returns (status, blocks that passed)."""
        n = C.c_int32(0)
        st = lib().nlmg_check_grid_barrier(self.h, int(blocks), int(absent_block), int(spin_limit), C.byref(n))
        return st, n.value

    def solve_device(self, f_ptr, g_ptr, x0_ptr, p_ptr, tol_rel=1e-8, tol_abs=1e-10, max_cycles=50):
        """Device-resident solve on raw device pointers (ints), e.g. torch tensor.data_ptr()."""
        rep = Report()
        st = lib().nlmg_solve_device(self.h, _P(f_ptr), _P(g_ptr), _P(x0_ptr) if x0_ptr else None, tol_rel,
                                     tol_abs, max_cycles, _P(p_ptr), C.byref(rep))
        return rep.as_dict(), st


class Server:
    """Continuous-batching request loop of the library (nlmg_server_*)."""

    def __init__(self, max_inflight=8, mem_budget_bytes=16 << 30, setup_threads_per_request=2, hierarchy_cache=None):
        o = ServerOptions()
        lib().nlmg_server_default_options(C.byref(o))
        o.max_inflight = max_inflight
        o.mem_budget_bytes = mem_budget_bytes
        o.setup_threads_per_request = setup_threads_per_request
        if hierarchy_cache is not None:
            o.hierarchy_cache = hierarchy_cache
        h = _P()
        st = lib().nlmg_server_create(C.byref(o), C.byref(h))
        if st != OK:
            raise NlmgError(st, "server create failed")
        self.h = h
        self._sizes = {}

    def submit(self, mesh, kappa_kind, kappa_a, opts, f_cell, g_face, tol_rel=1e-8, tol_abs=1e-10, max_cycles=60):
        fc = np.ascontiguousarray(mesh.face_cells, dtype=np.int32)
        vol, ht, area = _f64(mesh.cell_volume), _f64(mesh.half_trans), _f64(mesh.face_area)
        bc = np.ascontiguousarray(mesh.face_bc, dtype=np.uint8)
        f, g = _f64(f_cell), _f64(g_face)
        m = Mesh(mesh.n_cells, _dp(vol), int(fc.shape[0]), fc.ctypes.data_as(_I), _dp(ht),
                 bc.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(area))
        if isinstance(opts, dict):
            opts = options_from_dict(opts)
        t = C.c_uint64(0)
        st = lib().nlmg_server_submit(self.h, C.byref(m), C.byref(Kappa(int(kappa_kind), float(kappa_a))),
                                      C.byref(opts), _dp(f), _dp(g), tol_rel, tol_abs, max_cycles, C.byref(t))
        if st != OK:
            raise NlmgError(st, "submit failed")
        self._sizes[t.value] = mesh.n_cells
        return t.value

    def poll(self, ticket, wait_ms=0):
        """Returns None if not done, else (p, report dict, times dict, status)."""
        p = np.zeros(self._sizes[ticket])
        rep = Report()
        tm = RequestTimes()
        st = lib().nlmg_server_poll(self.h, ticket, int(wait_ms), _dp(p), C.byref(rep), C.byref(tm))
        if st == ETIMEOUT:
            return None
        del self._sizes[ticket]
        return p, rep.as_dict(), dict(queue_ms=tm.queue_ms, setup_ms=tm.setup_ms, solve_ms=tm.solve_ms,
                                      latency_ms=tm.latency_ms, hierarchy_reused=bool(tm.hierarchy_reused)), st

    def close(self):
        if getattr(self, "h", None):
            lib().nlmg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def request_bytes(mesh):
    """Device bytes the request loop reserves for a request on this mesh before admitting it."""
    fc = np.ascontiguousarray(mesh.face_cells, dtype=np.int32)
    vol, ht, area = _f64(mesh.cell_volume), _f64(mesh.half_trans), _f64(mesh.face_area)
    bc = np.ascontiguousarray(mesh.face_bc, dtype=np.uint8)
    m = Mesh(mesh.n_cells, _dp(vol), int(fc.shape[0]), fc.ctypes.data_as(_I), _dp(ht),
             bc.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(area))
    v = C.c_size_t(0)
    st = lib().nlmg_server_request_bytes(C.byref(m), C.byref(v))
    if st != OK:
        raise NlmgError(st, "request_bytes failed")
    return v.value


def measure_fp64_gflops():
    """FP64 FMA throughput of the current device (GFLOP/s) from the library's synthetic kernel."""
    v = C.c_double(0)
    st = lib().nlmg_measure_fp64(C.byref(v))
    if st != OK:
        raise NlmgError(st, "fp64 measurement failed")
    return v.value
