#!/usr/bin/env python
"""Benchmark: FAS solves of the 64^3 channelized TPFA problem on GB300, through the C ABI.

The headline (`value`) is the batched mixed form the metric names: one step = 32 right-hand sides of the workload
(per row its own Dirichlet data and smooth source) solved from p = 0 to relative residual 1e-8 (FP64 residuals and
convergence tests) on 8 contexts of one hierarchy, the level-0 Krylov solves preconditioned by the FP32 multigrid
V-cycle; device-resident inputs; the hierarchy is built once before timing. Beside it, `plain_fp64`: one right-hand
side at a time on one FP64 context (Jacobi-preconditioned persistent kernels), and the ratio. Level-0 smoothing is
Picard steps, then Newton steps once the residual is below 1e-3 of the initial one. Further sections: Picard
smoothing throughout, single-level baselines, the request loop, the 1M-cell Voronoi workload, the 256^3 workload
(`--cfg5`), and the FP64 CPU oracle on a bounded sample. Prints one JSON line. `--impl reference` times the oracle
instead (on a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s to rel. residual 1e-8 (batched mixed vs plain FP64); V-cycle DOF/s"
SMOOTHER_TEXT = {"picard": "FP64 Picard smoothing",
                 "picard_newton": "FP64 Picard-then-Newton level-0 smoothing (switch at 1e-3)"}


def workload_name(scale, smoother):
    return ("chan3d_%d: %d^3 hexahedral TPFA, channelized K over 6 decades, kappa = exp(2 p), 3-level FAS "
            "(aggregates 64 then 8, 4 modes), %s, tol 1e-8" % (scale, scale, SMOOTHER_TEXT[smoother]))
SAMPLE_SCALE = 16          # side of the reference arm's per-step sample of the same generator
CPU_SAMPLE_SCALE = 24      # side of the cpu_baseline sample


# DRAM bytes (read + write) per launch on the 64^3 workload with the default options, from ncu captures of the
# kernels as they are now (averaged over the launches of one solve where they differ): valid for that kernel, that
# workload and those options only, else the traffic is reported as null.
DRAM_BYTES_64 = {0: 23.102e6,     # kp_fine_cg_reg<double, 4>, mean of the 8 launches of a solve
                 1: 25.362e6,     # kp_coarse_step<double>, mean of the 15 launches (10 on level 1, 5 coarsest solves)
                 3: 25.216e6}     # kp_fine_bicgstab, mean of the 3 launches

KERNELS = {0: ("kp_fine_cg_reg<double, 4> (persistent register-resident pipelined Jacobi-scaled CG of the level-0 "
               "Picard step)", "kp_fine_cg* (level-0 Picard CG)"),
           1: ("kp_coarse_step<double> (fused coarse Picard step: coarse operator evaluations, pipelined hybridized "
               "CG, clamp and Algorithm 1 in one persistent launch)",) * 2,
           3: ("kp_fine_bicgstab (persistent FP64 BiCGStab of the level-0 Newton step)",) * 2,
           5: ("level-0 CG preconditioned by the multigrid V-cycle (per-step Galerkin setup, then one CUDA graph "
               "with a device-side while loop: FP64 CG vectors, FP32 V-cycle kernels)",) * 2,
           6: ("level-0 BiCGStab of the Newton step preconditioned by the multigrid V-cycle (setup and CUDA "
               "graphs as for the CG)",) * 2}


def roofline(prof, dev_ms, fp64_peak, hbm_peak, hbm_kind, default_case):
    """The roofline object of the kernel with the largest share of the solve time among the persistent kernels
    (0 level-0 CG, 1 + 4 coarse step: intermediate levels and the coarsest solve, 3 level-0 BiCGStab): FP64
    arithmetic against the measured FMA rate (at 64^3 the kernels' vectors live in L2), with the memory view
    beside it."""
    def add(a, b):
        return tuple(x + y for x, y in zip(a, b))
    kern = {0: prof[0], 1: add(prof[1], prof[4]), 3: prof[3], 5: prof[5], 6: prof[6]}
    kid = max((k for k in kern if kern[k][0]), key=lambda k: kern[k][1])
    n, ms, by, fl = kern[kid]
    avg_ms = ms / n
    gfs = fl / (avg_ms / 1e3) / 1e9
    gbs = by / (avg_ms / 1e3) / 1e9
    traffic = DRAM_BYTES_64.get(kid) if default_case else None
    if kid in (5, 6):   # memory-streaming FP32 kernels: the HBM roofline
        out = {"bound": "hbm", "kernel": KERNELS[kid][0], "achieved": gbs, "peak": hbm_peak, "peak_kind": hbm_kind,
               "unit": "GB/s", "frac": gbs / hbm_peak, "traffic": None,
               "traffic_note": "no capture of this kernel in this configuration", "bytes_per_launch": by,
               "avg_launch_us": avg_ms * 1e3, "launches": n, "share_of_solve": ms / dev_ms if dev_ms else None,
               "others": {}}
    else:
        out = None
    if out is None:
      out = {"bound": "alu", "kernel": KERNELS[kid][0 if default_case else 1], "achieved": gfs, "peak": fp64_peak,
           "peak_kind": "measured FP64 FMA throughput (nlmg_measure_fp64, independent FMA chains)",
           "unit": "GFLOP/s", "frac": gfs / fp64_peak, "traffic": traffic,
           "traffic_note": "DRAM read + write bytes per launch from ncu captures of this kernel on this workload" if
           traffic is not None else "no capture of this kernel in this configuration",
           "flops_per_launch": fl, "bytes_per_launch": by, "avg_launch_us": avg_ms * 1e3, "launches": n,
           "memory_view": {"achieved_GBs": gbs, "peak_GBs": hbm_peak, "peak_kind": hbm_kind, "frac": gbs / hbm_peak},
           "share_of_solve": ms / dev_ms if dev_ms else None, "others": {}}
    names = {0: "level0_cg", 1: "kp_coarse_step_intermediate_levels", 2: "k_residual", 3: "kp_fine_bicgstab",
             4: "kp_coarse_step_coarsest_solve", 5: "level0_mg_pcg", 6: "level0_mg_bicgstab"}
    for k in (0, 1, 2, 3, 4, 5, 6):
        if k == kid or not prof[k][0]:
            continue
        n, ms, by, fl = prof[k]
        avg = ms / n / 1e3
        out["others"][names[k]] = {"launches": n, "avg_us": avg * 1e6, "share_of_solve": ms / dev_ms if dev_ms else None,
                                   "GB/s": by / avg / 1e9, "GFLOP/s": fl / avg / 1e9 if fl else None}
    return out


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), "nlmg_bench_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
            sm = [float(r[1]) for r in rows]
            mx = float(rows[0][2])
            reasons = set()
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for r in rows:
                for k, nme in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nme)
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                    "samples": len(rows)}
        except Exception as e:  # no nvidia-smi
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "error": str(e)[:80]}


def _cpu_seconds():
    import resource
    ru = resource.getrusage(resource.RUSAGE_SELF)
    return ru.ru_utime + ru.ru_stime


def oracle_sample(smoother, scale, solves):
    """Times the FP64 oracle on the scale^3 instance of the same generator: the hierarchy once (setup), then
    `solves` FAS solves from p = 0 to relative residual 1e-8 (each timed). Returns the setup and solve wall times,
    the cycles, the cell count and the host threads the solves kept busy (CPU time / wall time)."""
    from synth.grids import problem_config
    from oracle import fas, hierarchy
    pr = problem_config("chan3d_64", scale=scale)
    pr.opts = dict(pr.opts, smoother=smoother)
    t0 = time.perf_counter()
    H = hierarchy.build(pr.mesh, pr.opts)
    setup_s = time.perf_counter() - t0
    times, cycles, cpu, wall = [], [], 0.0, 0.0
    for _ in range(solves):
        S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, pr.opts)
        c0 = _cpu_seconds()
        t0 = time.perf_counter()
        S.solve()
        times.append(time.perf_counter() - t0)
        cpu += _cpu_seconds() - c0
        wall += times[-1]
        cycles.append(S.stats.cycles)
    threads = max(1, int(round(cpu / wall))) if wall > 0 else 1
    return {"setup_s": setup_s, "solve_s": times, "cycles": cycles, "cells": pr.mesh.n_cells, "threads": threads}


def cpu_baseline_dict(full_cells, smoother):
    """The oracle measured on a bounded sample of the workload: the 24^3 instance of the same generator (13,824
    cells), median of 3 solves; solves/s scaled to the full mesh by the ratio of cell counts (the oracle's cost grows
    at least linearly in the cells, so the scaling favours the CPU)."""
    m = oracle_sample(smoother, CPU_SAMPLE_SCALE, 3)
    med = statistics.median(m["solve_s"])
    return {"value": (m["cells"] / full_cells) / med, "unit": "solves/s", "cores": m["threads"],
            "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": "FP64 oracle (numpy/scipy, sparse LU solves; its BLAS free to use every host core) on the "
                      "%d^3 instance of the same generator (%d cells, %s cycles): median solve %.2f s of 3, hierarchy "
                      "setup %.2f s (separate, not in the rate); solves/s scaled to %d cells by the cell ratio" %
                      (CPU_SAMPLE_SCALE, m["cells"], "/".join(str(c) for c in m["cycles"]), med, m["setup_s"],
                       full_cells),
            "measured": {"cells": m["cells"], "solve_s": m["solve_s"], "setup_s": m["setup_s"],
                         "cycles": m["cycles"], "threads_busy": m["threads"]}}


def serving_requests(n, seed=4, lo=4096, hi=262144):
    """Requests shaped like the serving workload: sizes log-uniform in [lo, hi] cells, 2D or 3D by a fair coin,
    each with its own log-normal K (sigma 1, correlation 4 cells), Dirichlet data g_L ~ U[0.5, 1.5],
    g_R ~ U[-0.5, 0.5], kappa = exp(a p) with a ~ U[0.5, 2]."""
    import numpy as np
    from synth.grids import cartesian_mesh, lognormal_field, default_options
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        cells = float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        if rng.uniform() < 0.5:
            side = int(round(cells ** 0.5))
            shape = (side, side)
            opts = default_options(n_levels=3, agg_size=[16, 8], modes=[2, 2])
        else:
            side = int(round(cells ** (1.0 / 3.0)))
            shape = (side, side, side)
            opts = default_options(n_levels=3, agg_size=[64, 8], modes=[4, 4])
        K = lognormal_field(shape, 1.0, 4.0, seed=1000 + seed * 97 + i)
        mesh = cartesian_mesh(shape, K)
        a = float(rng.uniform(0.5, 2.0))
        opts["dp_clamp"] = float(np.log(1.5) / a)
        g = np.zeros(mesh.n_faces)
        d = np.where(mesh.face_bc == 1)[0]
        g[d] = np.where(mesh.face_cells[d, 0] % shape[0] == 0, rng.uniform(0.5, 1.5), rng.uniform(-0.5, 0.5))
        out.append((mesh, a, opts, np.zeros(mesh.n_cells), g))
    return out


def _serve(nlmg, reqs, arrivals=None, hierarchy_cache=8):
    """Submits the requests (at the given arrival offsets in seconds, else all at once) to the library's request
    loop and collects latency (submit -> result), setup and solve times."""
    import numpy as np
    srv = nlmg.Server(max_inflight=8, mem_budget_bytes=32 << 30, setup_threads_per_request=2,
                      hierarchy_cache=hierarchy_cache)
    t0 = time.perf_counter()
    tickets = []
    for i, (m, a, o, f, g) in enumerate(reqs):
        if arrivals is not None:
            wait = t0 + arrivals[i] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
        tickets.append(srv.submit(m, 0, a, o, f, g))
    lat, solve_ms, setup_ms, ok, reused = [], [], [], 0, 0
    for t in tickets:
        p, rep, tm, st = srv.poll(t, wait_ms=600000)
        ok += st == 0
        lat.append(tm["latency_ms"])
        solve_ms.append(tm["solve_ms"])
        setup_ms.append(tm["setup_ms"])
        reused += bool(tm["hierarchy_reused"])
    makespan = time.perf_counter() - t0
    srv.close()
    lat = np.array(lat)
    return {"ok": int(ok), "solves_per_s": len(reqs) / makespan, "makespan_s": makespan,
            "p50_latency_ms": float(np.percentile(lat, 50)), "p99_latency_ms": float(np.percentile(lat, 99)),
            "mean_setup_ms": float(np.mean(setup_ms)), "mean_solve_ms": float(np.mean(solve_ms)),
            "hierarchies_reused": int(reused)}


def run_serving(nlmg, n, smoother, n_seq=48, n_reuse=24):
    """The request loop (FP32 inner CG in the FP64 FAS, up to 8 requests in flight): a burst of n requests of their
    own meshes (sizes log-uniform in 4k-256k cells), then the same requests arriving as a Poisson stream at 0.8 of
    the burst's throughput, then n_reuse requests on one mesh and K with their own nonlinearity parameter and data
    (hierarchy reuse). Against: the first n_seq requests one at a time on a plain FP64 context each, setup included
    and excluded (a sample: the whole stream one by one would take minutes)."""
    import numpy as np
    from synth.grids import cartesian_mesh, lognormal_field, default_options, multi_rhs_rows
    t0 = time.perf_counter()
    gen = serving_requests(n)
    reqs = [(m, a, dict(o, lin_precision=1, smoother=smoother), f, g) for m, a, o, f, g in gen]
    gen_s = time.perf_counter() - t0
    burst = _serve(nlmg, reqs)
    rng = np.random.default_rng(7)
    rate = 0.8 * burst["solves_per_s"]
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n))
    poisson = _serve(nlmg, reqs, arrivals=arrivals)
    poisson["arrival_rate_per_s"] = rate
    seq_solve_ms, seq_total_s = 0.0, 0.0
    n_seq = min(n_seq, n)
    for m, a, o, f, g in gen[:n_seq]:
        t1 = time.perf_counter()
        ctx = nlmg.Context(m, 0, a, dict(o, smoother=smoother))
        _, rep, st = ctx.solve(f, g, max_cycles=60)
        seq_total_s += time.perf_counter() - t1
        seq_solve_ms += rep["solve_ms"]
        ctx.close()
    # one reservoir: a 40^3 mesh and K, per request its own kappa = exp(a p), clamp and data
    side = 40
    mesh = cartesian_mesh((side,) * 3, lognormal_field((side,) * 3, 1.0, 4.0, seed=11))
    F, G = multi_rhs_rows(mesh, n_reuse, seed=12)
    alphas = rng.uniform(0.5, 2.0, n_reuse)
    base = default_options(n_levels=3, agg_size=[64, 8], modes=[4, 4], lin_precision=1, smoother=smoother)
    shared = [(mesh, float(a), dict(base, dp_clamp=float(np.log(1.5) / a)), F[i], G[i]) for i, a in enumerate(alphas)]
    reuse = _serve(nlmg, shared)
    no_reuse = _serve(nlmg, shared, hierarchy_cache=0)
    sizes = np.array([r[0].n_cells for r in reqs])
    return {"requests": n, "sizes_cells": {"min": int(sizes.min()), "median": int(np.median(sizes)),
                                           "mean": int(sizes.mean()), "max": int(sizes.max()),
                                           "three_d": int(sum(len(r[0].shape) == 3 for r in reqs))},
            "generate_s": gen_s, "burst": burst, "poisson": poisson,
            "sequential_fp64_sample": {
                "requests": n_seq, "mean_cells": int(sizes[:n_seq].mean()),
                "solves_per_s_incl_setup": n_seq / seq_total_s,
                "solves_per_s_excl_setup": n_seq / (seq_solve_ms / 1e3),
                "what": "the first requests of the stream one after the other, each on its own plain FP64 context"},
            "one_mesh_with_hierarchy_reuse": reuse, "one_mesh_without_reuse": no_reuse,
            "one_mesh_requests": n_reuse,
            "what": "each request its own mesh and hierarchy (sizes log-uniform 4k-256k cells, 2D/3D) unless noted; "
                    "latency = submit -> result; FP32 CG inside the FP64 FAS; max 8 in flight, admission by the "
                    "estimated device bytes against a 32 GiB budget; level-0 smoother: " + smoother}


def run_baselines(nlmg, pr, ctx):
    """The single-level solvers the paper compares FAS with (Sec. 2.2), on the same problem and GPU: Picard steps
    (frozen-coefficient CG to lin_tol, clamp, Algorithm 1) and Newton steps (exact Jacobian, GMRES(30), clamp,
    Algorithm 1), each from p = 0 to relative residual 1e-8 or its iteration cap; one timed solve each."""
    out = {}
    for name, kw, cap in (("picard", dict(picard_only=True), 400), ("newton", dict(newton=True), 15)):
        try:
            _, rep, st = ctx.solve(pr.f_cell, pr.g_face, max_cycles=cap, allow_noconv=True, **kw)
            out[name] = {"status": nlmg.STATUS_NAMES.get(int(st), str(st)), "iterations": rep["cycles"],
                         "ms": rep["solve_ms"], "solves_per_s": 1e3 / rep["solve_ms"] if rep["solve_ms"] else None,
                         "rel_residual": rep["res"] / rep["res0"] if rep["res0"] else None,
                         "lin_iters": rep["lin_iters"], "cap": cap}
        except nlmg.NlmgError as e:
            out[name] = {"status": "error", "what": str(e)[:160], "cap": cap}
    # single-level Picard and FAS with the same multigrid-preconditioned level-0 CG (the paper's single-level solvers
    # use AMG-preconditioned Krylov methods): one context set up with lin_precond = 1, one timed solve after a warm-up
    try:
        mctx = nlmg.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, dict(pr.opts, lin_precond=1))
        for name, kw, cap in (("picard_mg", dict(picard_only=True), 400), ("fas_mg", {}, 60)):
            mctx.solve(pr.f_cell, pr.g_face, max_cycles=cap, allow_noconv=True, **kw)
            _, rep, st = mctx.solve(pr.f_cell, pr.g_face, max_cycles=cap, allow_noconv=True, **kw)
            out[name] = {"status": nlmg.STATUS_NAMES.get(int(st), str(st)), "iterations": rep["cycles"],
                         "ms": rep["solve_ms"], "solves_per_s": 1e3 / rep["solve_ms"] if rep["solve_ms"] else None,
                         "rel_residual": rep["res"] / rep["res0"] if rep["res0"] else None,
                         "lin_iters": rep["lin_iters"], "cap": cap}
        mctx.close()
    except Exception as e:   # a comparison section: reported, never fatal to the bench line
        out["picard_mg"] = {"status": "error", "what": str(e)[:160]}
    out["what"] = ("single-level solvers from p = 0 on the same workload and GPU (the FAS line is the bench value); "
                   "a Newton iteration from p = 0 is outside its region of fast convergence on this channelized case; "
                   "picard_mg and fas_mg: single-level Picard and FAS, both with the multigrid-preconditioned level-0 "
                   "CG (lin_precond = 1)")
    return out


def run_multi_rhs(nlmg, pr, ctx, n_rhs, n_streams):
    """n_rhs right-hand sides on the bench mesh and its hierarchy: one plain FP64 context solving them one after the
    other, against nlmg_solve_many on n_streams contexts of the same hierarchy, in FP64 and with the FP32 inner CG,
    each with the library's default SM share and with the share chosen by nlmg_tune_sm_share on the first n_streams
    rows. Host buffers in and out in every variant (wall clock per batch)."""
    import numpy as np
    from synth.grids import multi_rhs_rows
    F, G = multi_rhs_rows(pr.mesh, n_rhs, seed=5)
    mctx = ctx.instance()
    mctx.set_options(lin_precision=1)
    ns = min(n_streams, n_rhs)
    ctx.solve_many(F[:ns], G[:ns], max_cycles=60, n_streams=n_streams)      # creates the instances
    mctx.solve_many(F[:ns], G[:ns], max_cycles=60, n_streams=n_streams)
    t0 = time.perf_counter()
    seq = [ctx.solve(F[r], G[r], max_cycles=60) for r in range(n_rhs)]
    t_seq = time.perf_counter() - t0
    out = {"rhs": n_rhs, "streams": n_streams, "sequential_fp64_solves_per_s": n_rhs / t_seq}
    for name, c in (("fp64", ctx), ("mixed", mctx)):
        best, rates = c.tune_sm_share(F[:ns], G[:ns])
        for mode, sms in (("default", 0), ("tuned", best)):
            c.set_options(max_sms=sms)
            t0 = time.perf_counter()
            P, reps, sts = c.solve_many(F, G, max_cycles=60, n_streams=n_streams)
            dt = time.perf_counter() - t0
            diff = max(float(np.linalg.norm(P[r] - seq[r][0]) / np.linalg.norm(seq[r][0])) for r in range(n_rhs))
            out["many_%s_%s" % (name, mode)] = {
                "solves_per_s": n_rhs / dt, "max_sms": sms, "ok": int(np.sum(sts == 0)),
                "max_rel_diff_vs_sequential_fp64": diff,
                "max_rel_residual": max(r["res"] / r["res0"] for r in reps)}
        out["tuner_%s" % name] = {"candidates_max_sms": "all, 1/2, 1/4, 1/8 of the SMs",
                                  "solves_per_s": [float(x) for x in rates], "best_max_sms": best}
        c.set_options(max_sms=0)
    out["cycles_per_solve"] = float(np.mean([r[1]["cycles"] for r in seq]))
    out["what"] = ("right-hand sides share the mesh, K and the hierarchy (per row: Dirichlet value on x = 0 and a "
                   "smooth source); sequential = one context on all SMs, one row after the other; many = "
                   "nlmg_solve_many; default share = SMs / min(streams, 4); tuned = nlmg_tune_sm_share on the first "
                   "rows; host buffers in and out; wall clock per batch; all at relative residual 1e-8")
    mctx.close()
    return out


def run_voronoi(nlmg, n_side, steps, smoother, fp64_peak=None, hbm_peak=None, hbm_kind=None):
    """Unstructured workload: clipped Voronoi mesh of a jittered n_side^3 lattice, ln K ~ N(0, 2^2) correlated over 4
    spacings, kappa = (1 + p^2)^-1, p = 1 on x = 0 and 0 on x = 1, 4-level FAS (aggregates 64 then 8, 4 modes).
    FP64 and FP32-inner-CG solves; each solution's FP64 residual is recomputed by the library's residual call (the
    GPU tests check that call against the oracle). The FP64 solve is also timed with the other level-0 smoother."""
    import numpy as np
    from synth.grids import voronoi_problem
    t0 = time.perf_counter()
    pr = voronoi_problem(n_side)
    t_mesh = time.perf_counter() - t0
    opts = dict(pr.opts, n_levels=4, agg_size=[64, 8, 8], modes=[4, 4, 4])
    t0 = time.perf_counter()
    ctx = nlmg.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, opts)
    t_setup = time.perf_counter() - t0
    out = {"cells": int(pr.mesh.n_cells), "faces": int(pr.mesh.n_faces), "mesh_s": t_mesh, "setup_s": t_setup,
           "levels": [ctx.level_info(l) for l in range(4)]}
    ctx.set_data(pr.f_cell, pr.g_face)
    r0 = np.linalg.norm(ctx.fine_residual(np.zeros(pr.mesh.n_cells)))
    p64 = None
    other = "picard" if smoother != "picard" else "picard_newton"
    for key, prec, sm in (("fp64", 0, smoother), ("mixed", 1, smoother), ("fp64_" + other, 0, other)):
        ctx.set_options(lin_precision=prec, smoother=sm)
        ctx.solve(pr.f_cell, pr.g_face, max_cycles=80)
        ms, rep, p = [], None, None
        if key == "fp64":
            ctx.profile(True)
        for _ in range(steps):
            p, rep, st = ctx.solve(pr.f_cell, pr.g_face, max_cycles=80)
            ms.append(rep["solve_ms"])
        if key == "fp64":
            prof = {k: ctx.profile_read(k) for k in (0, 1, 2, 3, 4, 5, 6)}
            ctx.profile(False)
            if fp64_peak:
                out["roofline"] = roofline(prof, float(np.sum(ms)), fp64_peak, hbm_peak, hbm_kind, False)
        r = np.linalg.norm(ctx.fine_residual(p))
        d = {"solves_per_s": 1e3 / np.mean(ms), "ms_per_solve": float(np.mean(ms)), "cycles": rep["cycles"],
             "newton_steps": rep["newton_steps"], "lin_iters_level": rep["lin_iters_level"][:4],
             "tol_tightened": rep["tol_tightened"], "rel_residual_recomputed": float(r / r0), "smoother": sm}
        if key == "fp64":
            p64 = p
        else:
            d["rel_diff_vs_fp64_solution"] = float(np.linalg.norm(p - p64) / np.linalg.norm(p64))
        out[key] = d
    ctx.close()
    return out


def run_reference(args, rank):
    """The oracle as the reference arm: each step is one FP64 oracle FAS solve of the 16^3 instance of the same
    generator (hierarchy built once, before the warm-up), timed on the host; ms_per_step is that measured time and
    the solves/s are scaled to the 64^3 mesh by the ratio of cell counts."""
    if rank != 0:
        return 0
    from synth.grids import problem_config
    from oracle import fas, hierarchy
    pr = problem_config("chan3d_64", scale=SAMPLE_SCALE)
    pr.opts = dict(pr.opts, smoother=args.smoother)
    t0 = time.perf_counter()
    H = hierarchy.build(pr.mesh, pr.opts)
    setup_s = time.perf_counter() - t0
    full = 64 ** 3

    def step():
        S = fas.FAS(H, pr.mesh, pr.kappa_kind, pr.kappa_a, pr.f_cell, pr.g_face, pr.opts)
        t0 = time.perf_counter()
        S.solve()
        return time.perf_counter() - t0, S.stats.cycles

    for _ in range(args.warmup):
        step()
    ts, cyc = [], []
    c0 = _cpu_seconds()
    for _ in range(args.steps):
        t, c = step()
        ts.append(t)
        cyc.append(c)
    threads = max(1, int(round((_cpu_seconds() - c0) / sum(ts))))
    ms_step = sum(ts) / len(ts) * 1e3
    value = (pr.mesh.n_cells / full) / (ms_step / 1e3)
    sample = ("each step one FP64 oracle FAS solve of the %d^3 instance of the same generator (%d cells, %d cycles), "
              "hierarchy (%.2f s) excluded; ms_per_step is the measured time per sample solve; solves/s scaled to "
              "%d cells by the cell ratio" % (SAMPLE_SCALE, pr.mesh.n_cells, cyc[-1], setup_s, full))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(64, args.smoother), "cells": full, "sample_cells": pr.mesh.n_cells},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "host_cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest of the ranks' values of x (the slowest replica sets the job's time); x itself without
    torch.distributed."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, steps, max_ms):
    """Whole-job solves/s of `world` independent replicas that each ran `steps` solves, the slowest in max_ms."""
    return world * steps / (max_ms / 1e3)


def run_batched(nlmg, pr, args, world, dist, dev, flush, local_rank):
    """The headline: the batched mixed form. One step = args.batch right-hand sides of the workload (per row its own
    Dirichlet value and smooth source, synth.grids.multi_rhs_rows) solved to relative residual 1e-8 by
    nlmg_solve_many_device on args.batch_streams contexts of one hierarchy, level-0 Krylov solves preconditioned by
    the FP32 multigrid V-cycle inside FP64 iterations. Device-resident rows; each step timed with a synchronize on
    both sides (the contexts run on their own streams); the L2 flush before each step is outside its span. e2e: the
    same batches through nlmg_solve_many with host arrays (pinned), copies in and out inside the timed span."""
    import numpy as np
    import torch
    from synth.grids import multi_rhs_rows
    N, NF = pr.mesh.n_cells, pr.mesh.n_faces
    t0 = time.perf_counter()
    bctx = nlmg.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, dict(pr.opts, lin_precond=1))
    setup_s = time.perf_counter() - t0
    F, G = multi_rhs_rows(pr.mesh, args.batch, seed=5)
    f_d = torch.from_numpy(F).to(dev)
    g_d = torch.from_numpy(G).to(dev)
    p_d = torch.zeros_like(f_d)

    def step():
        reps, sts, st = bctx.solve_many_device(args.batch, f_d.data_ptr(), g_d.data_ptr(), p_d.data_ptr(),
                                               n_streams=args.batch_streams, max_cycles=60)
        if st != nlmg.OK:
            raise RuntimeError("batched step failed: %s" % nlmg.STATUS_NAMES.get(int(st), st))
        return reps

    for _ in range(args.warmup):
        step()
    bctx.profile(True)
    times, all_reps = [], []
    with Clocks(local_rank) as clk:
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            all_reps += step()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t1)
        if dist is not None:
            dist.barrier()
    prof = {k: bctx.profile_read(k) for k in range(8)}
    bctx.profile(False)
    span = max_over_ranks(sum(times), dist, dev)
    # the first context's rows: its kernels' event time against the solve time of the rows it ran
    prof_dev_ms = sum(v[1] for k, v in prof.items() if k in (1, 2, 4, 5, 6, 7))
    # end to end: host rows in, solutions out
    Fh = np.ascontiguousarray(F)
    Gh = np.ascontiguousarray(G)
    e2e_t = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        P, reps_h, sts = bctx.solve_many(Fh, Gh, max_cycles=60, n_streams=args.batch_streams)
        e2e_t.append(time.perf_counter() - t1)
    e2e_s = max_over_ranks(sum(e2e_t), dist, dev)
    rr = [r["res"] / r["res0"] for r in all_reps]
    ms_step = span / args.steps * 1e3
    detail = {"value": world * args.steps * args.batch / span, "unit": "solves/s", "ms_per_step": ms_step,
              "ms_per_solve": ms_step / args.batch, "cycles_per_solve": float(np.mean([r["cycles"] for r in all_reps])),
              "max_rel_residual": float(max(rr)), "newton_steps_per_solve":
                  float(np.mean([r["newton_steps"] for r in all_reps])),
              "lin_iters_level0_per_solve": float(np.mean([r["lin_iters_level"][0] for r in all_reps])),
              "step_times_s": [round(t, 4) for t in times]}
    return {"value": world * args.steps * args.batch / span, "ms_per_step": ms_step, "setup_s": setup_s,
            "prof": prof, "prof_dev_ms": prof_dev_ms, "detail": detail, "clocks": clk.summary(),
            "gpu_launches": int(sum(r["kernel_launches"] for r in all_reps)),
            "e2e": {"value": world * len(e2e_t) * args.batch / e2e_s, "unit": "solves/s",
                    "h2d_bytes_per_step": 8 * args.batch * (N + NF), "d2h_bytes_per_step": 8 * args.batch * N}}


def run_cfg5(nlmg, args, fp64_peak, hbm_peak, hbm_kind):
    """The 256^3 channelized workload (16.8M cells, 8 decades, 5 levels of 64- then 8-cell aggregates, 6 modes):
    plain FP64 (one context, Jacobi-preconditioned persistent Krylov kernels, one row) against the batched mixed form
    (args.cfg5 rows of synth.grids.multi_rhs_rows on two contexts, FP32 multigrid V-cycle with BF16 transfers inside
    FP64 Krylov iterations), device-resident rows. Every row's relative residual is recomputed in FP64 by the library's residual
    call; the mixed row 0 is compared with the FP64 one."""
    import numpy as np
    import torch
    from synth.grids import problem_config, multi_rhs_rows
    out = {}
    try:
        t0 = time.perf_counter()
        pr = problem_config("chan3d_256")
        F, G = multi_rhs_rows(pr.mesh, args.cfg5, seed=5)
        out["generate_s"] = time.perf_counter() - t0
        N = pr.mesh.n_cells
        t0 = time.perf_counter()
        ctx = nlmg.Context(pr.mesh, pr.kappa_kind, pr.kappa_a,
                           dict(pr.opts, smoother=args.smoother, lin_precond=1))
        out["setup_s"] = time.perf_counter() - t0
        out["cells"] = N
        out["device_bytes_shared_own"] = list(ctx.device_bytes())
        dev = torch.device("cuda", torch.cuda.current_device())
        f_d = torch.from_numpy(F).to(dev)
        g_d = torch.from_numpy(G).to(dev)
        p_d = torch.zeros_like(f_d)
        p0 = torch.zeros(N, dtype=torch.float64, device=dev)
        # plain FP64: Jacobi-preconditioned persistent kernels, row 0
        ctx.set_options(lin_precond=0)
        rep, st = ctx.solve_device(f_d[0].data_ptr(), g_d[0].data_ptr(), 0, p0.data_ptr(), 1e-8, 1e-10, 80)
        out["plain_fp64"] = {"solves_per_s": 1e3 / rep["solve_ms"], "ms": rep["solve_ms"], "cycles": rep["cycles"],
                             "status": int(st), "rel_residual": rep["res"] / rep["res0"],
                             "lin_iters_level": rep["lin_iters_level"][:5]}
        # batched mixed: FP32 V-cycle with BF16 transfers (FP32 accumulation) inside FP64 Krylov iterations
        ctx.set_options(lin_precond=1, lin_precision=2)
        ctx.profile(True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        reps, sts, st = ctx.solve_many_device(args.cfg5, f_d.data_ptr(), g_d.data_ptr(), p_d.data_ptr(),
                                              n_streams=2, max_cycles=80)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t1
        prof = {k: ctx.profile_read(k) for k in range(8)}
        ctx.profile(False)
        res = []
        for r in range(args.cfg5):
            ctx.set_data(F[r], G[r])
            rv = ctx.fine_residual(p_d[r].cpu().numpy())
            r0 = ctx.fine_residual(np.zeros(N))
            res.append(float(np.linalg.norm(rv) / np.linalg.norm(r0)))
        diff = float(torch.linalg.norm(p_d[0] - p0) / torch.linalg.norm(p0))
        out["batched_mixed"] = {"solves_per_s": args.cfg5 / dt, "rows": args.cfg5, "streams": 2, "wall_s": dt,
                                "ok": int(np.sum(sts == 0)), "cycles": [r["cycles"] for r in reps],
                                "ms_per_row": [round(r["solve_ms"], 1) for r in reps],
                                "rel_residual_recomputed_fp64": res,
                                "rel_diff_row0_vs_plain_fp64": diff,
                                "lin_iters_level": reps[0]["lin_iters_level"][:5]}
        out["batched_vs_plain_fp64"] = (args.cfg5 / dt) / out["plain_fp64"]["solves_per_s"]
        dev_ms = sum(v[1] for k, v in prof.items() if k in (1, 2, 4, 5, 6, 7))
        out["roofline"] = roofline(prof, dev_ms, fp64_peak, hbm_peak, hbm_kind, False)
        out["what"] = ("synthetic stand-in of the paper's refinement study shape; plain FP64 measured on row 0 alone, "
                       "the batch on every row; relative residuals recomputed by the library's FP64 residual")
        ctx.close()
    except Exception as e:   # the section is reported, not fatal to the bench line
        out["error"] = str(e)[:300]
    return out


def run_vcycle_probe(side):
    """The multigrid preconditioner alone on the channelized generator of the 256^3 workload at side^3 (5 levels,
    6 modes): three applications of one V-cycle (the kernels a launch list captures), then the time of one iteration of
    the preconditioned level-0 CG (CUDA events: the slope between 2 and 22 iterations at a fixed frozen matrix). One
    JSON line."""
    import numpy as np
    from paper_2005_01275_gb300 import build, nlmg
    from synth.grids import problem_config
    build.build()
    t0 = time.perf_counter()
    pr = problem_config("chan3d_256", scale=side)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ctx = nlmg.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, dict(pr.opts, lin_precond=1))
    setup_s = time.perf_counter() - t0
    ctx.set_data(pr.f_cell, pr.g_face)
    rng = np.random.default_rng(1)
    p = rng.uniform(0, 1, pr.mesh.n_cells)
    for _ in range(3):
        z = ctx.precond_apply(p, rng.uniform(-1, 1, pr.mesh.n_cells))
    per = {}
    for k in (2, 22):
        ctx.set_options(lin_tol=1e-30, lin_maxit=k)
        ctx.picard_update(0, p)
        ctx.profile(True)
        for _ in range(3):
            ctx.picard_update(0, p)
        n, ms, by, fl = ctx.profile_read(5)
        ctx.profile(False)
        per[k] = (ms / n, by / n)
    us = (per[22][0] - per[2][0]) / 20 * 1e3
    byt = (per[22][1] - per[2][1]) / 20
    print(json.dumps({"vcycle_probe": {"side": side, "cells": int(pr.mesh.n_cells), "generate_s": gen_s,
                                       "setup_s": setup_s, "levels": [ctx.level_info(l) for l in range(ctx.n_levels())],
                                       "us_per_cg_iteration": us, "bytes_per_cg_iteration": byt,
                                       "GBs": byt / (us / 1e6) / 1e9, "z_norm": float(np.linalg.norm(z))}}))
    ctx.close()
    return 0


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2005_01275_gb300 import build, nlmg
    build.build()
    from synth.grids import problem_config
    pr = problem_config("chan3d_64", scale=args.scale)
    pr.opts = dict(pr.opts, smoother=args.smoother)
    N = pr.mesh.n_cells
    if args.lin_tol is not None:
        pr.opts["lin_tol"] = args.lin_tol
    if args.coarse_lin_tol is not None:
        pr.opts["coarse_lin_tol"] = args.coarse_lin_tol
    if args.flux_modes != 1:
        pr.opts["flux_modes"] = [args.flux_modes] * 8
    if args.cascadic:
        pr.opts["cascadic"] = 1
    t0 = time.perf_counter()
    ctx = nlmg.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, pr.opts)
    setup_s = time.perf_counter() - t0
    dev = torch.device("cuda", local_rank)
    f_d = torch.from_numpy(pr.f_cell).to(dev)
    g_d = torch.from_numpy(pr.g_face).to(dev)
    p_d = torch.zeros(N, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    torch.cuda.synchronize()

    def solve_dev():
        rep, st = ctx.solve_device(f_d.data_ptr(), g_d.data_ptr(), 0, p_d.data_ptr(), 1e-8, 1e-10, 60)
        if st != nlmg.OK:
            raise RuntimeError("solve failed with status %d: %s" % (st, rep))
        return rep

    for _ in range(args.warmup):
        solve_dev()
    # timed region: K device-resident solves, L2 flushed between steps (outside each step's event pair)
    ctx.profile(True)
    reps = []
    with Clocks(local_rank) as clk:
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        w0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            reps.append(solve_dev())
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        wall = time.perf_counter() - w0
    clocks = clk.summary()
    prof = {k: ctx.profile_read(k) for k in (0, 1, 2, 3, 4, 5, 6)}
    ctx.profile(False)
    dev_ms = max_over_ranks(sum(r["solve_ms"] for r in reps), dist, dev)
    picard = None
    if args.smoother != "picard" and args.compare_picard:
        # the same timed loop with Picard steps throughout, for comparison
        ctx.set_options(smoother="picard")
        solve_dev()
        preps = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            preps.append(solve_dev())
        ctx.set_options(smoother=args.smoother)
        pms = max_over_ranks(sum(r["solve_ms"] for r in preps), dist, dev)
        picard = {"value": replica_throughput(world, args.steps, pms), "unit": "solves/s",
                  "ms_per_step": pms / args.steps, "cycles_per_solve": sum(r["cycles"] for r in preps) / len(preps),
                  "lin_iters_level": preps[-1]["lin_iters_level"][:3],
                  "what": "the same solves with Picard steps on level 0 throughout (Sec. 3.3.1 smoother)"}
    one_coarsest = None
    if args.compare_picard:
        # the same timed loop with one Picard step on the coarsest level instead of up to 10
        ctx.set_options(coarsest_steps=1)
        solve_dev()
        creps = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            creps.append(solve_dev())
        ctx.set_options(coarsest_steps=pr.opts.get("coarsest_steps", 10))
        cms = max_over_ranks(sum(r["solve_ms"] for r in creps), dist, dev)
        one_coarsest = {"value": replica_throughput(world, args.steps, cms), "unit": "solves/s",
                        "ms_per_step": cms / args.steps,
                        "cycles_per_solve": sum(r["cycles"] for r in creps) / len(creps),
                        "what": "the same solves with one Picard step on the coarsest level (coarsest_steps = 1) "
                                "instead of the paper's up to 10"}
    # end to end through the host-pointer C-ABI call: H2D of f and g from pinned memory, D2H of p
    f_h = torch.from_numpy(pr.f_cell).pin_memory()
    g_h = torch.from_numpy(pr.g_face).pin_memory()
    p_h = torch.zeros(N, dtype=torch.float64).pin_memory()
    e2e_t = []
    for _ in range(max(1, args.steps)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        rep, st = ctx.solve_ptr(f_h.data_ptr(), g_h.data_ptr(), p_h.data_ptr())
        e2e_t.append(time.perf_counter() - t1)
        if st != nlmg.OK:
            raise RuntimeError("e2e solve failed %d" % st)
    e2e_s = max_over_ranks(sum(e2e_t), dist, dev)
    head = run_batched(nlmg, pr, args, world, dist, dev, flush, local_rank)
    if rank != 0:
        dist.destroy_process_group()
        return 0
    peak, peak_kind = _peaks()
    ms_step = dev_ms / args.steps
    cycles = sum(r["cycles"] for r in reps) / len(reps)
    value = replica_throughput(world, args.steps, dev_ms)
    fp64_peak_gflops = nlmg.measure_fp64_gflops()
    default_case = (args.scale == 64 and args.lin_tol is None and args.coarse_lin_tol is None and
                    args.smoother == "picard_newton")
    roof = roofline(prof, dev_ms, fp64_peak_gflops, peak, peak_kind, default_case)
    mixed = None
    if args.mixed:
        mopts = dict(pr.opts, lin_precision=1)
        mctx = nlmg.Context(pr.mesh, pr.kappa_kind, pr.kappa_a, mopts)
        pm_d = torch.zeros(N, dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            mctx.solve_device(f_d.data_ptr(), g_d.data_ptr(), 0, pm_d.data_ptr(), 1e-8, 1e-10, 60)
        mms, mrep = 0.0, None
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            mrep, st = mctx.solve_device(f_d.data_ptr(), g_d.data_ptr(), 0, pm_d.data_ptr(), 1e-8, 1e-10, 60)
            if st != nlmg.OK:
                raise RuntimeError("mixed solve failed %d" % st)
            mms += mrep["solve_ms"]
        diff = float(torch.linalg.norm(pm_d - p_d) / torch.linalg.norm(p_d))
        mixed = {"value": world * args.steps / (mms / 1e3), "unit": "solves/s", "ms_per_step": mms / args.steps,
                 "cycles_per_solve": mrep["cycles"], "rel_residual": mrep["res"] / mrep["res0"],
                 "rel_diff_vs_fp64_solution": diff, "lin_iters_level": mrep["lin_iters_level"][:3],
                 "what": "same FP64 FAS (residuals, transfers, coarse operators, convergence test in FP64); the CG "
                         "solves inside the Picard steps in FP32 (tolerances floored at 1e-6); the Newton steps' "
                         "BiCGStab stays FP64"}
    walls = {}

    def timed(name, fn):
        t1 = time.perf_counter()
        r = fn()
        walls[name] = round(time.perf_counter() - t1, 1)
        return r

    baselines = timed("single_level_baselines", lambda: run_baselines(nlmg, pr, ctx)) \
        if (args.baselines and world == 1) else None
    multi = timed("multi_rhs", lambda: run_multi_rhs(nlmg, pr, ctx, args.multi_rhs, args.streams)) \
        if (args.multi_rhs > 0 and world == 1) else None
    serving = timed("serving", lambda: run_serving(nlmg, args.serving, args.smoother)) \
        if (args.serving > 0 and world == 1) else None
    voronoi = timed("voronoi", lambda: run_voronoi(nlmg, args.voronoi, max(1, min(5, args.steps // 2)), args.smoother,
                                                   fp64_peak_gflops, peak, peak_kind)) \
        if (args.voronoi > 0 and world == 1) else None
    cpu = timed("cpu_baseline", lambda: cpu_baseline_dict(N, args.smoother)) if (args.cpu_baseline and world == 1) \
        else None
    cfg5 = timed("cfg5", lambda: run_cfg5(nlmg, args, fp64_peak_gflops, peak, peak_kind)) \
        if (args.cfg5 > 0 and world == 1) else None
    head_roof = roofline(head["prof"], head["prof_dev_ms"], fp64_peak_gflops, peak, peak_kind, False)
    head_roof["measured_on"] = ("the batch's first context (it solves its share of the rows on its own stream, "
                                "side by side with the other contexts); share_of_solve relative to its rows")
    plain_fp64 = {
        "value": value, "unit": "solves/s", "ms_per_step": ms_step, "steps": args.steps,
        "what": "one right-hand side at a time on one FP64 context (Jacobi-preconditioned persistent Krylov kernels), "
                "device-resident data, CUDA-event time per solve",
        "vcycle_dof_per_s": N * cycles * world / (ms_step / 1e3),
        "cycles_per_solve": cycles,
        "lin_iters_per_solve": sum(r["lin_iters"] for r in reps) / len(reps),
        "lin_iters_level": reps[-1]["lin_iters_level"][:3],
        "wall_s_timed_region": wall,
        "roofline": roof,
        "clocks": clocks,
        "e2e": {"value": world * len(e2e_t) / e2e_s, "unit": "solves/s",
                "h2d_bytes_per_step": 8 * (N + len(pr.g_face)), "d2h_bytes_per_step": 8 * N},
        "gpu_launches": int(sum(r["kernel_launches"] for r in reps))}
    line = {
        "metric": METRIC, "value": head["value"], "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.scale, args.smoother) + "; batched mixed: %d right-hand sides per "
                               "step (Dirichlet data and smooth sources per row) on %d contexts of one hierarchy, level-0 "
                               "Krylov solves preconditioned by the FP32 multigrid V-cycle inside FP64 iterations" %
                               (args.batch, args.batch_streams),
                   "cells": N, "rhs_per_step": args.batch, "streams": args.batch_streams, "smoother": args.smoother,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "256 MiB buffer written before every step, outside the step's timed span",
                   "setup_s": round(head["setup_s"], 3), "lin_tol": ctx.opts.lin_tol,
                   "flux_modes": args.flux_modes, "cascadic": int(args.cascadic),
                   "coarse_lin_tol": ctx.opts.coarse_lin_tol, "lin_precond": 1},
        "batched_vs_plain_fp64": head["value"] / value,
        "plain_fp64": plain_fp64,
        "batched": head["detail"],
        "cycles_per_solve": head["detail"]["cycles_per_solve"],
        "roofline": head_roof,
        "picard_smoother": picard,
        "one_coarsest_step": one_coarsest,
        "single_level_baselines": baselines,
        "mixed": mixed,
        "multi_rhs": multi,
        "serving": serving,
        "voronoi": voronoi,
        "cpu_baseline": cpu,
        "cfg5": cfg5,
        "section_wall_s": walls,
        "e2e": head["e2e"],
        "gpu_launches": head["gpu_launches"],
        "clocks": head["clocks"],
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nlmg", choices=["nlmg", "reference"])
    ap.add_argument("--scale", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--lin-tol", type=float, default=None, help="level-0 CG tolerance (default: library's)")
    ap.add_argument("--coarse-lin-tol", type=float, default=None, help="coarse CG tolerance")
    ap.add_argument("--no-mixed", dest="mixed", action="store_false", help="skip the FP32-CG variant")
    ap.add_argument("--serving", type=int, default=512, help="requests in the serving run (0 = skip)")
    ap.add_argument("--multi-rhs", type=int, default=16, help="right-hand sides in the multi-RHS run (0 = skip)")
    ap.add_argument("--streams", type=int, default=8, help="contexts (streams) of the multi-RHS solve")
    ap.add_argument("--smoother", default="picard_newton", choices=["picard", "picard_newton"],
                    help="level-0 smoother (Picard-then-Newton by default)")
    ap.add_argument("--no-baselines", dest="baselines", action="store_false",
                    help="skip the single-level Picard and Newton solves")
    ap.add_argument("--no-compare-picard", dest="compare_picard", action="store_false",
                    help="skip the timed loop with Picard steps throughout")
    ap.add_argument("--flux-modes", type=int, default=1,
                    help="m_f, flux unknowns per coarse interface at most, on every coarsening step (default 1)")
    ap.add_argument("--cascadic", action="store_true",
                    help="start every solve from the nonlinear cascadic iterate (Sec. 4.2)")
    ap.add_argument("--batch", type=int, default=32, help="right-hand sides per step of the batched headline")
    ap.add_argument("--batch-streams", type=int, default=8, help="contexts (streams) of the batched headline")
    ap.add_argument("--cfg5", type=int, default=8,
                    help="rows of the 256^3 batched section (0 = skip); its plain FP64 reference is one row")
    ap.add_argument("--voronoi", type=int, default=100,
                    help="lattice side of the unstructured Voronoi section (100 = 1M cells, the default; 0 = skip)")
    ap.add_argument("--vcycle", type=int, default=0,
                    help="only time the multigrid-preconditioned level-0 CG on the 256^3 generator at this side "
                         "(per iteration, and three V-cycle applications): the command the V-cycle launch lists use")
    args = ap.parse_args()
    if args.vcycle > 0:
        return run_vcycle_probe(args.vcycle)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus if "RANK" in os.environ else 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank)
    return run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
