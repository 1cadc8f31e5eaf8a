#!/usr/bin/env python
"""Benchmark of the slab residual inside the per-slab GMRES solve on one GB300.

Workload (default): 64^3 uniform affine hexahedra on [0,1]^3, p = 4, q = 3,
eps and mu element-wise U[1,4] (PCG64 seeds 1307, 1308), slab-start state
U[-1,1] (seed 1310), PEC, J = 0, dt = h/(2p+1).  Elements are numbered along
the Z-order curve.

One step = one slab solve: GMRES(10) right-preconditioned by the
time-derivative terms, FP64, to 1e-9 relative residual, restarted from the
same slab-start state every step (the state is reset by a device copy), so
every step does the same work.  It runs every row of the hot path: temporal
contraction, mass, volume curl, face traces and lift (the residual kernels),
the preconditioner, the Krylov dot products and updates, and the slab-end
extraction and energy.

value = residual GDoF/s = (trial DoF per slab = 6 (q+1)(p+1)^3 per element)
        x (residual applies per step) / (seconds per step), summed over GPUs.

Inputs (6.3 GB of coefficients) are far larger than the 129 MB L2, so no L2
flush is needed between steps.  --impl reference times the CPU oracle on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "residual GDoF/s + %roofline, mixed vs FP64 @1e-9 rel; slab solves/s; p99 ms"


def hbm_peak():
    """Measured copy bandwidth of this machine's GPUs (GB/s) from MEASURED_PEAKS.json beside this
    file, else the fallback figure of 6,800 GB/s; returns (value, source)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "hbm_gbs of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "6,800 GB/s of fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=64, help="elements per direction")
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--q", type=int, default=3)
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the extra legs")
    ap.add_argument("--legs", default="hp_batch,curved,serving,inexact,dissipative,time_refinement,cavity_plain",
                    help="comma-separated extra legs to run (also, opt-in: serving_full = the full serving "
                         "stream, 512 requests with n up to 48, both precisions; tm11_hp = the hp experiment of "
                         "Sec. 6.1.1; iteration_study = GMRES iterations of the Sec. 5.3 resonator vs tolerance "
                         "and initial guess; curved_slabs = 50 mixed slab solves on 32^3 trilinear hexes, p = 3, 5, "
                         "7, Gaussian J)")
    ap.add_argument("--profile-case", default=None, choices=["apply", "curved", "solve", "hp"],
                    help="run a small fixed case for a profiler and exit (no JSON line): 'apply' = --steps "
                         "residual applies on --n^3 bricks (p, q), 'curved' = the same on trilinear hexes "
                         "(q = p - 1), 'solve' = --steps slab solves of the bench workload, 'hp' = --steps "
                         "residual applies on the hp_batch mesh (2:1 octree, uneven p and q; --n ignored)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "mixed"],
                    help="precision of --profile-case")
    ap.add_argument("--reorth", type=int, default=0, help="second Gram-Schmidt pass (DGKS test); off by default: same iteration count and accuracy on this workload")
    return ap.parse_args()


def workload(n, p, q):
    from paper_1307_5310_gb300 import meshgen

    m = meshgen.box_mesh(n, p=p, q=q, order="morton")
    meshgen.random_materials(m, 1307, 1308)
    return m


def flops_per_element(p, q):
    """Algorithmic flops of one residual apply per element (both fields), split by kernel.

    prep : y = B u (nnzB per point) and the folded face traces (one pass per axis, 2 comps)
    apply: mass (1 FMA per entry), volume curl (6 terms x nnzD per line), folded lift.
    """
    n = p + 1
    n2, n3 = n * n, n ** 3
    nnzB = 2 if q == 1 else 2 * q + 1
    nnzD = n * n // 4
    prep = 2 * (3 * n3 * nnzB + 3 * 2 * q * n3)
    apply = 2 * (3 * q * n3 + 6 * q * n2 * nnzD + 3 * 2 * q * n3)
    return 2 * prep, 2 * apply


def linop_bytes_per_element(p, q, es=4):
    """Algorithmic HBM bytes per element of one Krylov-operator apply A P^{-1} v (no slab-start
    mode, no load): read v, write A P^{-1} v, the six preconditioner factors and neighbour ids."""
    n3 = (p + 1) ** 3
    return es * (6 * q * n3 + 6 * q * n3) + 6 * es + 6 * 4


def fp32_krylov_kernel(p, q):
    """Name of the kernel of the mixed solve's FP32 operator A P^{-1} v on uniform bricks, by the
    launcher's shared-memory rule (residual.cuh: fused_smem <= 64 KB, fused_kry_smem <= 74 KB)."""
    n3, n2 = (p + 1) ** 3, (p + 1) ** 2
    fused = 4 * (12 * q * n3 + 24 * q * n2)
    kry = ((fused + 15) & ~15) + 4 * 12 * ((q * n3 + 6) & ~3)
    if fused > 64 * 1024:
        return f"k_prep<float,{p},{q}> + k_apply<float,{p},{q}>"
    return f"k_fused_kry<{p},{q}>" if kry <= 74 * 1024 else f"k_fused<float,{p},{q},1>"


def bytes_per_element(p, q, es=8):
    """Algorithmic HBM bytes of one apply per element: read U, write R, eps/mu."""
    n3 = (p + 1) ** 3
    return es * (6 * (q + 1) * n3 + 6 * q * n3) + 16


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _oracle_worker(task):
    """One process of the CPU baseline: the oracle's residual on its share of the elements of
    an 8^3 block of the workload, in chunks, until the time budget is spent."""
    p, q, elems, budget = task
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"  # one thread per process: the pool already covers the cores
    from oracle import stdg
    from paper_1307_5310_gb300 import meshgen

    n = 8
    m = meshgen.box_mesh(n, hi=(n / 64.0,) * 3, p=p, q=q)
    meshgen.random_materials(m, 1307, 1308)
    U = meshgen.random_coeffs(m, 1309)
    dt = (1.0 / 64) / (2 * p + 1)
    o = stdg.Oracle(m)
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < budget:  # cycles over the share until the budget is spent
        k = done % len(elems)
        chunk = elems[k:k + 4]
        o.residual(U, 0.0, dt, elems=chunk)
        done += len(chunk)
    return done, time.perf_counter() - t0


def cpu_baseline(p, q, target_s=15.0, pool=None):
    """The CPU oracle, as it stands, on an 8^3 block of the workload (PEC on the block boundary),
    spread over the host cores by a spawned process pool (elements dealt round-robin)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    workers = max(1, min(os.cpu_count() or 1, 64))
    own = pool is None
    if own:
        pool = cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"))
    try:
        elems = list(range(8 ** 3))
        tasks = [(p, q, elems[w::workers], target_s) for w in range(workers)]
        res = list(pool.map(_oracle_worker, tasks))
    finally:
        if own:
            pool.shutdown()
    done = sum(d for d, _ in res)
    t = max(w for _, w in res)
    dof = done * 6 * (q + 1) * (p + 1) ** 3
    return {"value": dof / t / 1e9, "unit": "GDoF/s", "cores": workers, "kind": "oracle",
            "sample": f"residual of {done} element evaluations over an 8^3 block of the workload (h=1/64, p={p}, "
                      f"q={q}, PEC on the block boundary), numpy FP64 full tensor quadrature, {workers} spawned "
                      f"processes (one per host core, one thread of work each), {t:.1f} s"}, t


def run_reference(args):
    import concurrent.futures as cf
    import multiprocessing as mp

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    workers = max(1, min(os.cpu_count() or 1, 64))
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as pool:
        base, _ = cpu_baseline(args.p, args.q, target_s=2.0, pool=pool)
        vals = []
        for _ in range(args.warmup):
            cpu_baseline(args.p, args.q, target_s=2.0, pool=pool)
        for _ in range(args.steps):
            b, t = cpu_baseline(args.p, args.q, target_s=6.0, pool=pool)
            vals.append((b["value"], t))
    v = statistics.median(x for x, _ in vals)
    tms = statistics.median(t for _, t in vals) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GDoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"affine {args.n}^3 bricks p={args.p} q={args.q}",
                       "sample": "8^3 block per step", "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": v, "unit": "GDoF/s", "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": v, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_solve(s, u_init, dt, steps, warmup, barrier):
    """Time `steps` slab solves from the same start state; returns timings and counters."""
    import torch

    reps = []

    def step():
        s.set_state(u_init)
        rc, rep = s.slab_solve(dt)
        reps.append((rc, rep))

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    s.profile(True)
    l0 = s.launch_count()
    reps.clear()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms = []
    e0.record()
    for _ in range(steps):
        a = time.perf_counter()
        step()
        torch.cuda.synchronize()
        step_ms.append((time.perf_counter() - a) * 1e3)
    e1.record()
    torch.cuda.synchronize()
    barrier()
    prof = s.profile_read()
    s.profile(False)
    return {"ms": e0.elapsed_time(e1) / steps, "step_ms": step_ms, "launches": s.launch_count() - l0,
            "prof": prof, "iterations": statistics.mean(r["iterations"] for _, r in reps),
            "restarts": statistics.mean(r["restarts"] for _, r in reps),
            "rel_residual": max(r["rel_residual"] for _, r in reps), "rc": [rc for rc, _ in reps]}


def curved_flops_per_element(p, q):
    """Algorithmic flops of one curved apply per element (both fields): the O(p^5)
    sum-factorised mass replaces the affine mass term."""
    n, nq = p + 1, p + 2
    fl_prep, fl_apply = flops_per_element(p, q)
    affine_mass = 2 * 2 * (3 * q * n ** 3)
    mass = 2 * 2 * q * (6 * (n ** 3 * nq + n ** 2 * nq ** 2 + n * nq ** 3) + 9 * nq ** 3)
    return fl_prep, fl_apply - affine_mass, mass


def time_applies(s, m, dt, prec, reps=5, warm=2):
    """CUDA-event time (ms) of one of `reps` residual applies through the C ABI on device buffers
    (no per-kernel profile: uneven meshes then run their class kernels side by side)."""
    import torch

    from paper_1307_5310_gb300 import stm

    dtp = torch.float64 if prec == stm.STM_FP64 else torch.float32
    U = torch.empty(s.n_trial, dtype=dtp, device="cuda").uniform_(-1, 1)
    R = torch.empty(s.n_test, dtype=dtp, device="cuda")
    for _ in range(warm):
        s.residual_apply(U, R, 0.0, dt, prec=prec)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        s.residual_apply(U, R, 0.0, dt, prec=prec)
    e1.record()
    torch.cuda.synchronize()
    del U, R
    return e0.elapsed_time(e1) / reps


def leg_hp_batch(fp64_peak):
    """2:1 corner-refined octree, 203,736 elements, p ~ U{1..7}, q ~ U{1..4}, eps ~ {1, 2.25, 4}."""
    import numpy as np

    from paper_1307_5310_gb300 import meshgen, stm

    m = meshgen.corner_octree_mesh(50, [0.45, 0.2])
    meshgen.random_hp(m, 1307)
    p, q = m["p"].astype(np.int64), m["q"].astype(np.int64)
    dof = int(np.sum(6 * (q + 1) * (p + 1) ** 3))
    fl = sum(sum(flops_per_element(int(pp), int(qq))) for pp, qq in zip(p, q))
    s = stm.Slab(m, tol=1e-9, max_it=400, reorth=False)
    dt = (1.0 / 200) / 15
    ms64 = time_applies(s, m, dt, stm.STM_FP64)
    ms32 = time_applies(s, m, dt, stm.STM_FP32)
    by32 = sum(bytes_per_element(int(pp), int(qq), 4) for pp, qq in zip(p, q))
    ach = fl / (ms64 / 1e3) / 1e12
    s.close()
    return {"workload": "2:1 corner octree 203,736 elements, p~U{1..7}, q~U{1..4}, eps~{1,2.25,4}, all "
                        f"{len(set(zip(p.tolist(), q.tolist())))} (p,q) classes + 2:1 transfers per apply",
            "elements": int(m["hex"].shape[0]), "hanging_rows": int(m["hang"].shape[0]), "dof": dof,
            "fp64": {"ms_per_apply": ms64, "gdofs": dof / (ms64 / 1e3) / 1e9,
                     "roofline": {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                                  "frac": ach / fp64_peak}},
            "fp32": {"ms_per_apply": ms32, "gdofs": dof / (ms32 / 1e3) / 1e9,
                     "roofline": {"bound": "hbm", "achieved": by32 / (ms32 / 1e3) / 1e9, "peak": hbm_peak()[0],
                                  "unit": "GB/s", "frac": by32 / (ms32 / 1e3) / 1e9 / hbm_peak()[0],
                                  "peak_source": hbm_peak()[1]}}}


def leg_curved(fp64_peak):
    """32^3 trilinear hexes (vertices moved by 0.1 h sin sin sin), p in {3, 5, 7}, q = p - 1."""
    from paper_1307_5310_gb300 import meshgen, stm

    out = {}
    for p in (3, 5, 7):
        q = p - 1
        m = meshgen.box_mesh(32, p=p, q=q, perturb=0.1, order="morton")
        meshgen.random_materials(m, 1307, 1308)
        s = stm.Slab(m)
        ne = m["hex"].shape[0]
        dt = (1.0 / 32) / (2 * p + 1)
        ms64 = time_applies(s, m, dt, stm.STM_FP64, reps=3)
        ms32 = time_applies(s, m, dt, stm.STM_FP32, reps=3)
        fp, fa, fm = curved_flops_per_element(p, q)
        ach = (fp + fa + fm) * ne / (ms64 / 1e3) / 1e12
        dof = ne * 6 * (q + 1) * (p + 1) ** 3
        out[f"p{p}"] = {"ms_fp64": ms64, "ms_fp32": ms32, "gdofs_fp64": dof / (ms64 / 1e3) / 1e9,
                        "gdofs_fp32": dof / (ms32 / 1e3) / 1e9, "flops_per_element": fp + fa + fm,
                        "roofline_fp64": {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                                          "frac": ach / fp64_peak}}
        s.close()
    return out


def leg_inexact():
    """Exact vs inexact slab solves for a TM_mm mode in the PEC unit cube, 8^3 bricks,
    p = q = 1..6, dt = h/(2p+1), m = 1, 1, 2, 2, 3, 3, the step counts of the paper's
    resonator experiment (Sec. 5.3).  The inexact run stops each slab on its share of the
    guaranteed bound eta_it, with target 0.1 x the discretisation error of the exact run (exact:
    relative residual 1e-14); its iteration error is measured against the exact run."""
    import numpy as np

    from paper_1307_5310_gb300 import meshgen, stm

    steps = {1: 189, 2: 315, 3: 220, 4: 283, 5: 213, 6: 252}
    out = {}
    for p in range(1, 7):
        mm = (p + 1) // 2
        E, H, _ = tm_mode(mm)
        m = meshgen.box_mesh(8, p=p, q=p)
        dt = (1.0 / 8) / (2 * p + 1)
        N = steps[p]
        T = N * dt
        aux = stm.Slab(m)
        aux.set_initial(lambda x: E(x, T), lambda x: H(x, T))
        uex, _ = aux.get_state()

        def err(u):
            aux.set_state(u)
            return math.sqrt(2.0 * aux.energy())

        def run(**kw):
            s = stm.Slab(m, max_it=4000, **kw)
            s.set_initial(lambda x: E(x, 0.0), lambda x: H(x, 0.0))
            it, eta2 = 0, 0.0
            torch_sync()
            a = time.perf_counter()
            for _ in range(N):
                rc, rep = s.slab_solve(dt)
                if rc != stm.STM_OK:
                    raise RuntimeError(f"slab solve returned {rc}")
                it += rep["iterations"]
                eta2 += rep["eta2"]
            torch_sync()
            ms = (time.perf_counter() - a) * 1e3
            u, _ = s.get_state()
            s.close()
            return u, it / N, math.sqrt(eta2), ms

        ue, it_e, _, ms_e = run(tol=1e-14)  # "exact": the tolerance whose counts match the paper's (R30)
        e_T = err(ue - uex)
        ui, it_i, eta, ms_i = run(eta_tol=0.1 * e_T, t_final=T)
        ur = ue  # the discrete solution (to 1e-14) the iteration error is measured against
        d = err(ui - ur)
        out[f"p{p}"] = {"steps": N, "m": mm, "N_it": it_e, "N_it_inexact": it_i, "speedup_iterations": it_e / it_i,
                        "speedup_time": ms_e / ms_i, "ms_exact": ms_e, "ms_inexact": ms_i, "e_T": e_T,
                        "e_T_inexact": err(ui - uex), "eta_it": eta, "iteration_error": d,
                        "I_eff": eta / d if d > 0 else None}
        aux.close()
    out["workload"] = ("TM_mm mode, PEC unit cube, 8^3 bricks, p=q=1..6, dt=h/(2p+1), exact = FP64 GMRES(10) to "
                       "1e-14, inexact = eta_it stopping with eta_tol = 0.1 e(T) of the exact run, iteration error "
                       "vs the exact run")
    return out


def tm_mode(mm, xy_only=True):
    """The TM_mm cavity mode of the PEC box (Sec. 6.1.1 with m = n = mm): E = sin(mm pi x)
    sin(mm pi y) cos(w t) e_z, H from mu H_t = -curl E, w = pi sqrt(2) mm (eps = mu = 1)."""
    import numpy as np

    w = math.pi * math.sqrt(2.0) * mm

    def E(x, t):
        z = np.zeros(x.shape[0])
        return np.stack([z, z, np.sin(mm * math.pi * x[:, 0]) * np.sin(mm * math.pi * x[:, 1]) * math.cos(w * t)], 1)

    def H(x, t):
        f = -math.sin(w * t) / w * mm * math.pi
        return np.stack([f * np.sin(mm * math.pi * x[:, 0]) * np.cos(mm * math.pi * x[:, 1]),
                         -f * np.cos(mm * math.pi * x[:, 0]) * np.sin(mm * math.pi * x[:, 1]),
                         np.zeros(x.shape[0])], 1)

    return E, H, w


def leg_tm11_hp(periods=20, p_mins=(1, 2, 3, 4)):
    """The hp experiment of Sec. 6.1.1: the TM_11 mode in [0,1] x [0,1] x [0,1/5] on 5 x 5 x 1
    hexahedra; from the boundary ring to the centre the elements take N_K = 1, 2, 4 local time
    steps and degrees p = q = p_min, p_min + 1, p_min + 2.  Slab dt = h / (2 p_min + 1) with
    h = 1/5.  Reports the spatial L2 error at the slab ends once per period, and the
    L2(0,T; L2) error from those samples (trapezoid rule), for each p_min."""
    import numpy as np

    from paper_1307_5310_gb300 import meshgen, stm

    E, H, w = tm_mode(1)
    T_per = 2 * math.pi / w
    out = {"workload": f"TM_11 in [0,1]^2 x [0,0.2], 5x5x1 hexahedra, rings N_K = 1/2/4 and p = q = p_min + "
                       f"0/1/2, PEC, dt = 0.2/(2 p_min + 1), {periods} periods, FP64 GMRES(10) to 1e-10",
           "runs": {}}
    for pm in p_mins:
        m = meshgen.box_mesh(5, 5, 1, hi=(1.0, 1.0, 0.2), p=1, q=1)
        cen = m["vert"][m["hex"]].mean(axis=1)
        i, j = np.floor(cen[:, 0] * 5).astype(int), np.floor(cen[:, 1] * 5).astype(int)
        ring = np.minimum(np.minimum(i, j), np.minimum(4 - i, 4 - j))
        m["p"] = (pm + ring).astype(np.uint8)
        m["q"] = (pm + ring).astype(np.uint8)
        m["nk"] = np.array([1, 2, 4])[ring].astype(np.uint8)
        dt = 0.2 / (2 * pm + 1)
        steps_per = max(1, int(round(T_per / dt)))
        dt = T_per / steps_per  # whole periods
        s = stm.Slab(m, tol=1e-10, max_it=4000, reorth=False)
        aux = stm.Slab(m)
        s.set_initial(lambda x: E(x, 0.0), lambda x: H(x, 0.0))

        def err(t):
            aux.set_initial(lambda x: E(x, t), lambda x: H(x, t))
            ue, _ = aux.get_state()
            u, _ = s.get_state()
            aux.set_state(u - ue)
            return math.sqrt(2.0 * aux.energy())

        errs, its = [err(0.0)], 0
        torch_sync()
        a = time.perf_counter()
        for k in range(periods):
            for _ in range(steps_per):
                rc, rep = s.slab_solve(dt)
                if rc != stm.STM_OK:
                    raise RuntimeError(f"slab solve returned {rc}")
                its += rep["iterations"]
            errs.append(err((k + 1) * T_per))
        torch_sync()
        ms = (time.perf_counter() - a) * 1e3
        l2l2 = math.sqrt(sum(0.5 * (errs[k] ** 2 + errs[k + 1] ** 2) * T_per for k in range(periods)))
        out["runs"][f"p_min{pm}"] = {"dt": dt, "slabs": periods * steps_per, "dofs": int(s.n_trial),
                                     "gmres_iterations_per_slab": its / (periods * steps_per),
                                     "error_per_period": errs, "l2_l2_error": l2l2, "ms": ms}
        s.close()
        aux.close()
    e = [out["runs"][f"p_min{pm}"]["l2_l2_error"] for pm in p_mins]
    out["log10_error_slope_per_p"] = float(np.polyfit(np.array(p_mins, float), np.log10(e), 1)[0])
    return out


def leg_iteration_study(slabs=40):
    """GMRES(10) iterations per slab of the resonator of Sec. 5.3 (TM_mm mode, 8^3 bricks,
    p = q = 1..6, dt = h/(2p+1), m = 1,1,2,2,3,3) for stop tolerances 1e-8 ... 1e-14 of the
    relative true residual, from the initial guess u_1 = u_0 and from zero; the paper's exact
    solves take 7.9, 24, 25, 20, 22, 18 iterations per slab."""
    from paper_1307_5310_gb300 import meshgen, stm

    out = {"paper_N_it": {"p1": 7.9, "p2": 24.0, "p3": 25.0, "p4": 20.0, "p5": 22.0, "p6": 18.0},
           "workload": f"TM_mm mode, PEC unit cube, 8^3 bricks, p=q, dt=h/(2p+1), first {slabs} slabs, FP64 "
                       "GMRES(10) right-preconditioned, stop on ||R(U^k)|| <= tol ||R(unknowns 0)||"}
    for p in range(1, 7):
        mm = (p + 1) // 2
        E, H, _ = tm_mode(mm)
        m = meshgen.box_mesh(8, p=p, q=p)
        dt = (1.0 / 8) / (2 * p + 1)
        row = {}
        for zero in (False, True):
            for tol in (1e-8, 1e-10, 1e-12, 1e-14):
                s = stm.Slab(m, tol=tol, max_it=4000, reorth=False, zero_guess=zero)
                s.set_initial(lambda x: E(x, 0.0), lambda x: H(x, 0.0))
                it = 0
                for _ in range(slabs):
                    rc, rep = s.slab_solve(dt)
                    it += rep["iterations"]
                s.close()
                row[f"{'zero' if zero else 'u0'}_tol{tol:g}"] = it / slabs
        out[f"p{p}"] = row
    return out


def torch_sync():
    import torch

    torch.cuda.synchronize()


def _solve_ms(s, u0, dt, reps=2):
    """Mean wall time of `reps` slab solves from the same state (synchronous C-ABI calls)."""
    out = []
    for k in range(reps + 1):
        s.set_state(u0)
        torch_sync()
        a = time.perf_counter()
        rc, rep = s.slab_solve(dt)
        torch_sync()
        if k > 0:
            out.append(((time.perf_counter() - a) * 1e3, rep["iterations"], rc))
    return statistics.mean(o[0] for o in out), out[-1][1], out[-1][2]


def leg_cavity_plain():
    """The plain-method configuration: PEC unit cube, 4^3 affine hexes, eps = mu = 1, J = 0,
    p = 2, q = 1, E0 = (0, 0, sin pi x sin pi y), H0 = 0, 20 slabs of dt = 0.05, FP64 slab solves
    to 1e-12 relative residual; timed per slab, with the energy drift and the error against the
    analytic cavity mode at t = 1."""
    import numpy as np

    from paper_1307_5310_gb300 import meshgen, stm

    m = meshgen.box_mesh(4, p=2, q=1)
    E, H, _ = tm_mode(1)
    out = {"workload": "PEC unit cube, 4^3 bricks, p=2, q=1, TM_11 initial data, 20 slabs of dt=0.05, FP64 "
                       "GMRES(10) to 1e-12 (20,736 DoF per slab)"}
    for per in (1, 8):
        s = stm.Slab(m, tol=1e-12, restart=10, max_it=2000, reorth=False, cycles_per_launch=per)
        s.set_initial(lambda x: E(x, 0.0), lambda x: H(x, 0.0))
        s.slab_solve(0.05)  # warm-up: graph capture
        s.set_initial(lambda x: E(x, 0.0), lambda x: H(x, 0.0))
        e0 = s.energy()
        torch_sync()
        times, its = [], 0
        for _ in range(20):
            a = time.perf_counter()
            rc, rep = s.slab_solve(0.05)
            torch_sync()
            times.append((time.perf_counter() - a) * 1e3)
            its += rep["iterations"]
        u, t = s.get_state()
        aux = stm.Slab(m)
        aux.set_initial(lambda x: E(x, t), lambda x: H(x, t))
        ue, _ = aux.get_state()
        aux.set_state(u - ue)
        err = math.sqrt(2.0 * aux.energy())
        aux.close()
        times.sort()
        out[f"cycles_per_launch_{per}"] = {
            "ms_per_slab_median": statistics.median(times), "ms_per_slab_p99": times[-1],
            "slab_solves_per_s": 1e3 / statistics.mean(times), "gmres_iterations_per_slab": its / 20,
            "energy_drift_rel": abs(s.energy() - e0) / e0, "l2_error_vs_mode_at_t1": err}
        s.close()
    return out


def leg_curved_slabs(slabs=50, ps=(3, 5, 7)):
    """The curved configuration as stated: 32^3 trilinear hexes (vertices moved by 0.1 h sin sin
    sin), p in {3, 5, 7}, q = p - 1, eps = mu = 1, a Gaussian current pulse (width 0.05, centre of
    the domain, Gaussian in time), dt = h/(2p+1), `slabs` mixed-precision slab solves (FP32
    inner GMRES with the mass term on the tensor cores, FP64 outer refinement) to 1e-9."""
    from paper_1307_5310_gb300 import meshgen, stm

    out = {"workload": f"32^3 trilinear hexes (0.1 h sin sin sin), q = p - 1, Gaussian J (sigma_x = 0.05 at the "
                       f"centre, z-directed, sigma_t = 0.05, t0 = 0.2), dt = h/(2p+1), {slabs} mixed slab solves "
                       "to 1e-9 relative residual"}
    for p in ps:
        q = p - 1
        m = meshgen.box_mesh(32, p=p, q=q, perturb=0.1, order="morton")
        dt = (1.0 / 32) / (2 * p + 1)
        s = stm.Slab(m, precision=stm.STM_MIXED, tol=1e-9, max_it=400, reorth=False)
        s.set_source_gauss([dict(centre=(0.5, 0.5, 0.5), dir=(0.0, 0.0, 1.0), sigma_x=0.05, t0=0.2, sigma_t=0.05,
                                 amp=1.0)])
        dof = s.n_trial
        torch_sync()
        a = time.perf_counter()
        its, worst = 0, 0.0
        for _ in range(slabs):
            rc, rep = s.slab_solve(dt)
            its += rep["iterations"]
            worst = max(worst, rep["rel_residual"])
        torch_sync()
        ms = (time.perf_counter() - a) * 1e3 / slabs
        out[f"p{p}"] = {"ms_per_slab": ms, "slab_solves_per_s": 1e3 / ms, "dof_per_slab": int(dof),
                        "inner_iterations_per_slab": its / slabs, "max_rel_residual": worst,
                        "energy_at_end": rep["energy"]}
        s.close()
        torch_sync()
    return out


def leg_dissipative(fp64_peak):
    """The bench workload (64^3 bricks, p=4, q=3) with the dissipative term D_h of Sec. 4.2, c = 1."""
    import numpy as np

    from paper_1307_5310_gb300 import stm

    n, p, q = 64, 4, 3
    m = workload(n, p, q)
    ne = m["hex"].shape[0]
    dt = (1.0 / n) / (2 * p + 1)
    dof = ne * 6 * (q + 1) * (p + 1) ** 3
    s = stm.Slab(m, c_diss=1.0, tol=1e-9, max_it=400, reorth=False)
    ms64 = time_applies(s, m, dt, stm.STM_FP64, reps=3)
    ms32 = time_applies(s, m, dt, stm.STM_FP32, reps=3)
    u0 = np.random.Generator(np.random.PCG64(1310)).uniform(-1, 1, s.n_state)
    sol64, it64, rc64 = _solve_ms(s, u0, dt, reps=1)
    s.close()
    smx = stm.Slab(m, c_diss=1.0, precision=stm.STM_MIXED, tol=1e-9, max_it=400, reorth=False)
    solmx, itmx, rcmx = _solve_ms(smx, u0, dt, reps=1)
    smx.close()
    fp, fa = flops_per_element(p, q)
    fd = 2 * 3 * 2 * q * (p + 1) ** 2 * 6  # per line: two jumps, two alpha scalings, two combinations
    ach = (fp + fa + fd) * ne / (ms64 / 1e3) / 1e12
    by32 = (bytes_per_element(p, q, 4) + 24 * 4) * ne  # + the 24 alpha coefficients per element
    return {"workload": "64^3 bricks, p=4, q=3, eps/mu U[1,4], PEC, dt=h/9, c_diss=1",
            "fp64": {"ms_per_apply": ms64, "gdofs": dof / (ms64 / 1e3) / 1e9,
                     "roofline": {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                                  "frac": ach / fp64_peak, "flops_per_element": fp + fa + fd}},
            "fp32": {"ms_per_apply": ms32, "gdofs": dof / (ms32 / 1e3) / 1e9, "kernel": f"k_fused<float,{p},{q},0,1>",
                     "roofline": {"bound": "hbm", "achieved": by32 / (ms32 / 1e3) / 1e9, "peak": hbm_peak()[0],
                                  "unit": "GB/s", "frac": by32 / (ms32 / 1e3) / 1e9 / hbm_peak()[0],
                                  "bytes_per_element": by32 / ne, "peak_source": hbm_peak()[1]}},
            "slab_solve_fp64": {"ms": sol64, "iterations": it64, "rc": rc64},
            "slab_solve_mixed": {"ms": solmx, "iterations": itmx, "rc": rcmx}}


def leg_time_refinement(fp64_peak):
    """48^3 bricks, p=3, q=2, N_K ~ U{1,2,4} per element (local refinement in time, Sec. 2.2)."""
    import numpy as np

    from paper_1307_5310_gb300 import meshgen, stm

    n, p, q = 48, 3, 2
    m = meshgen.box_mesh(n, p=p, q=q, order="morton")
    meshgen.random_materials(m, 1307, 1308)
    meshgen.random_nk(m, 1309, (1, 2, 4))
    nk = m["nk"].astype(np.int64)
    ne = m["hex"].shape[0]
    dt = (1.0 / n) / (2 * p + 1)
    dof = int(np.sum(6 * (nk * q + 1) * (p + 1) ** 3))
    s = stm.Slab(m, tol=1e-9, max_it=400, reorth=False)
    ms64 = time_applies(s, m, dt, stm.STM_FP64, reps=3)
    ms32 = time_applies(s, m, dt, stm.STM_FP32, reps=3)
    u0 = np.random.Generator(np.random.PCG64(1310)).uniform(-1, 1, s.n_state)
    sol64, it64, rc64 = _solve_ms(s, u0, dt, reps=1)
    s.close()
    smx = stm.Slab(m, precision=stm.STM_MIXED, tol=1e-9, max_it=400, reorth=False)
    solmx, itmx, rcmx = _solve_ms(smx, u0, dt, reps=1)
    smx.close()
    fl = int(np.sum(nk)) * sum(flops_per_element(p, q))  # per sub-interval the work of a q-mode element
    ach = fl / (ms64 / 1e3) / 1e12
    by32 = int(np.sum(nk)) * bytes_per_element(p, q, 4)
    return {"workload": "48^3 bricks, p=3, q=2, N_K~U{1,2,4} (PCG64 1309), eps/mu U[1,4], PEC, dt=h/7",
            "elements": ne, "dof": dof, "classes": "(p,q,N_K) = (3,2,1|2|4)",
            "fp64": {"ms_per_apply": ms64, "gdofs": dof / (ms64 / 1e3) / 1e9,
                     "roofline": {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                                  "frac": ach / fp64_peak}},
            "fp32": {"ms_per_apply": ms32, "gdofs": dof / (ms32 / 1e3) / 1e9,
                     "roofline": {"bound": "hbm", "achieved": by32 / (ms32 / 1e3) / 1e9, "peak": hbm_peak()[0],
                                  "unit": "GB/s", "frac": by32 / (ms32 / 1e3) / 1e9 / hbm_peak()[0],
                                  "peak_source": hbm_peak()[1]}},
            "slab_solve_fp64": {"ms": sol64, "iterations": it64, "rc": rc64},
            "slab_solve_mixed": {"ms": solmx, "iterations": itmx, "rc": rcmx}}


def serving_stream(n_req, n_max, rate=50.0, seed=1311):
    """The request stream of the serving workload: Poisson arrivals (mean `rate` req/s), n^3
    unit-cube bricks with n log-uniform in [8, n_max] (multiples of 4), p ~ U{2..6},
    q ~ U{1..3}, 1-4 eps/mu boxes U[1,4], 1-3 Gaussian pulses, cavity or scattering, 10 slabs
    of dt = h/(2p+1) each."""
    import numpy as np

    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, n_req)
    reqs = []
    for k in range(n_req):
        n = int(4 * round(np.exp(rng.uniform(np.log(8), np.log(n_max))) / 4))
        p, q = int(rng.integers(2, 7)), int(rng.integers(1, 4))
        boxes = []
        for _ in range(int(rng.integers(1, 5))):
            a = rng.uniform(0, 0.7, 3)
            b = a + rng.uniform(0.1, 0.3, 3)
            boxes.append(tuple(a) + tuple(np.minimum(b, 1.0)) + (rng.uniform(1, 4), rng.uniform(1, 4)))
        srcs = []
        for _ in range(int(rng.integers(1, 4))):
            d = rng.normal(size=3)
            srcs.append(dict(centre=tuple(rng.uniform(0.2, 0.8, 3)), dir=tuple(d / np.linalg.norm(d)), sigma_x=0.05,
                             t0=0.2, sigma_t=0.05, amp=1.0))
        kind = int(rng.integers(0, 2))
        reqs.append(dict(n=n, p=p, q=q, n_slabs=10, dt=(1.0 / n) / (2 * p + 1), kind=kind, boxes=boxes,
                         sources=srcs if kind == 1 else srcs[:1]))
    return reqs, np.cumsum(gaps)


def run_stream(reqs, arrivals, precision, workers=16):
    """Submit the stream at its arrival times to a server and wait for every result."""
    from paper_1307_5310_gb300 import stm

    srv = stm.Server(workers=workers, precision=precision, tol=1e-9, max_it=2000)
    t0 = time.perf_counter()
    tickets = []
    for k, r in enumerate(reqs):
        while time.perf_counter() - t0 < float(arrivals[k]):
            time.sleep(0.0005)
        tickets.append(srv.submit(**r))
    res = [srv.wait(t)[0] for t in tickets]
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat = sorted(r["latency_ms"] for r in res if r["status"] >= 0)
    solves = 10 * len(lat)
    return {"achieved_req_per_s": len(lat) / wall, "completed": st["completed"], "failed": st["failed"],
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "slab_solves_per_s": solves / wall, "wall_s": wall,
            "peak_admitted_gb": st["peak_admitted_bytes"] / 1e9,
            "max_rel_residual": max(r["max_rel_residual"] for r in res),
            "gmres_iterations": int(sum(r["iterations"] for r in res))}


def leg_serving(n_req=48, n_max=24, rate=50.0, seed=1311):
    """The serving workload in mixed precision and in plain FP64 (same stream, same 1e-9
    target): solves/s, latency percentiles, and the mixed-over-FP64 throughput ratio."""
    from paper_1307_5310_gb300 import stm

    reqs, arrivals = serving_stream(n_req, n_max, rate, seed)
    out = {"requests": n_req, "offered_req_per_s": rate, "workers": 16,
           "workload": f"Poisson stream (mean {rate:g} req/s) of {n_req} requests; n^3 unit-cube bricks, n "
                       f"log-uniform in [8,{n_max}] (x4), p~U{{2..6}}, q~U{{1..3}}, 1-4 eps/mu boxes U[1,4], "
                       "1-3 Gaussian pulses, cavity or scattering, 10 slabs each to 1e-9 relative residual"}
    for name, prec in (("mixed", stm.STM_MIXED), ("fp64", stm.STM_FP64)):
        out[name] = run_stream(reqs, arrivals, prec)
    out["mixed_over_fp64_solves_per_s"] = out["mixed"]["slab_solves_per_s"] / out["fp64"]["slab_solves_per_s"]
    return out


def dist_max(v, device="cuda"):
    """Maximum of v over all ranks of the default process group (v itself without one):
    the job's time is its slowest replica's."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return v
    t = torch.tensor([v], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, ms_max):
    """Units per second of the whole job: every replica processes units_per_rank, the job
    ends with the slowest replica (weak scaling, no data-path collective)."""
    return world * units_per_rank / (ms_max / 1e3)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1307_5310_gb300 import stm

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(v):
        return dist_max(v, "cuda")

    m = workload(args.n, args.p, args.q)
    ne = m["hex"].shape[0]
    h = 1.0 / args.n
    dt = h / (2 * args.p + 1)
    n3 = (args.p + 1) ** 3
    dof_slab = ne * 6 * (args.q + 1) * n3
    rng = np.random.Generator(np.random.PCG64(1310))
    u_host = torch.from_numpy(rng.uniform(-1, 1, ne * 6 * n3)).pin_memory()
    u_init = u_host.cuda()
    torch.cuda.synchronize()

    # ---- FP64 slab solve: the timed step --------------------------------------------------
    s = stm.Slab(m, tol=args.tol, restart=10, max_it=400, reorth=bool(args.reorth))
    clk = Clocks(local)
    r64 = measure_solve(s, u_init, dt, args.steps, args.warmup, barrier)
    clocks = clk.stop()
    ms = max_over_ranks(r64["ms"])
    prof = r64["prof"]
    applies = prof["k_apply_fp64"][1] / args.steps
    value = whole_job_rate(world, dof_slab * applies, ms) / 1e9
    u64 = torch.empty_like(u_init)
    s.get_state(u64)

    fl_prep, fl_apply = flops_per_element(args.p, args.q)
    apply_ms = prof["k_apply_fp64"][0] / max(1, prof["k_apply_fp64"][1])
    prep_ms = prof["k_prep_fp64"][0] / max(1, prof["k_prep_fp64"][1])
    sm_mhz = clocks["sm_mhz"] or 2070.0
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp64_peak = 4.0 * sms * sm_mhz * 1e6 / 1e12  # 2 FP64 FMA / clock / SM
    ach = fl_apply * ne / (apply_ms / 1e3) / 1e12
    # DRAM bytes per k_apply launch from one ncu capture of the 32^3 case (1.936 GB read + 0.572 GB
    # written), scaled by the element count to this workload; valid for p=4, q=3 on 64^3 only
    traffic = 2.507e9 * ne / 32 ** 3 if (args.n, args.p, args.q) == (64, 4, 3) else None
    try:  # context: the FP64 FMA rate this GPU reaches in a register-only kernel, measured live
        probe = stm.fp64_probe()
    except Exception:  # reported as missing, never replaced
        probe = None
    roofline = {"kernel": f"k_apply<double,{args.p},{args.q}>", "bound": "alu", "achieved": ach, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": ach / fp64_peak, "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, 32^3 capture x 8 (bytes)",
                "peak_source": f"FP64 pipe: 2 FMA/clock/SM x {sms} SMs (device property) x median SM clock under "
                               "load (of derived)",
                "launch_ms": apply_ms,
                "fp64_probe_tflops": probe, "frac_of_probe": (ach / probe) if probe else None,
                "prep": {"kernel": f"k_prep<double,{args.p},{args.q}>", "launch_ms": prep_ms,
                         "achieved": fl_prep * ne / (prep_ms / 1e3) / 1e12,
                         "frac": fl_prep * ne / (prep_ms / 1e3) / 1e12 / fp64_peak},
                # the whole FP64 residual apply (both launches, the flop model of both)
                "combined": {"kernels": f"k_prep + k_apply <double,{args.p},{args.q}>",
                             "launch_ms": prep_ms + apply_ms,
                             "achieved": (fl_prep + fl_apply) * ne / ((prep_ms + apply_ms) / 1e3) / 1e12,
                             "frac": (fl_prep + fl_apply) * ne / ((prep_ms + apply_ms) / 1e3) / 1e12 / fp64_peak}}

    # ---- end to end through the C ABI with pinned host buffers ---------------------------------
    hb_in, hb_out = stm.HostBuffer(u_host.numel()), stm.HostBuffer(u_host.numel())
    uh, oh = hb_in.array, hb_out.array
    uh[:] = u_host.numpy()
    s.set_state(uh)
    s.slab_solve(dt)
    s.get_state(oh)
    barrier()
    t0 = time.perf_counter()
    parts = [0.0, 0.0, 0.0]
    per_step = []
    for _ in range(args.steps):
        a = time.perf_counter()
        s.set_state(uh)
        b = time.perf_counter()
        s.slab_solve(dt)
        c_ = time.perf_counter()
        s.get_state(oh)
        d = time.perf_counter()
        parts[0] += b - a
        parts[1] += c_ - b
        parts[2] += d - c_
        per_step.append([round((b - a) * 1e3, 2), round((c_ - b) * 1e3, 2), round((d - c_) * 1e3, 2)])
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps)
    e2e = {"value": whole_job_rate(world, dof_slab * applies, e2e_ms) / 1e9, "unit": "GDoF/s",
           "h2d_bytes_per_step": int(uh.nbytes), "d2h_bytes_per_step": int(oh.nbytes), "ms_per_step": e2e_ms,
           "path": "stm_set_state (host) + stm_slab_solve + stm_get_state (host), buffers from stm_host_alloc",
           "ms_set_solve_get": [x * 1e3 / args.steps for x in parts], "ms_set_solve_get_per_step": per_step}

    # tight FP64 reference solution of the same slab for the accuracy statement
    s.close()
    sref = stm.Slab(m, tol=1e-12, restart=10, max_it=2000, reorth=True)
    sref.set_state(u_init)
    sref.slab_solve(dt)
    uref = torch.empty_like(u_init)
    sref.get_state(uref)
    sref.close()
    err64 = float(torch.linalg.norm(u64 - uref) / torch.linalg.norm(uref))

    # ---- mixed precision: FP32 inner GMRES, FP64 refinement ----------------------------------
    mixed = None
    try:
        smx = stm.Slab(m, precision=stm.STM_MIXED, tol=args.tol, restart=10, max_it=400, reorth=bool(args.reorth))
        rmx = measure_solve(smx, u_init, dt, args.steps, args.warmup, barrier)
        umx = torch.empty_like(u_init)
        smx.get_state(umx)
        msx = max_over_ranks(rmx["ms"])
        pm = rmx["prof"]
        ap64, ap32 = pm["k_apply_fp64"][1] / args.steps, pm["k_apply_fp32"][1] / args.steps
        mixed = {"ms_per_solve": msx, "slab_solves_per_s": world / (msx / 1e3),
                 "gdofs": whole_job_rate(world, dof_slab * (ap64 + ap32), msx) / 1e9,
                 "fp64_applies": ap64, "fp32_applies": ap32, "inner_iterations": rmx["iterations"],
                 "outer_refinements": rmx["restarts"], "rel_residual": rmx["rel_residual"],
                 "rel_err_vs_fp64_ref": float(torch.linalg.norm(umx - uref) / torch.linalg.norm(uref)),
                 "speedup_vs_fp64": ms / msx, "gpu_launches": rmx["launches"]}
        # FP32 residual kernel (single pass): HBM roofline
        k32 = pm["k_apply_fp32"]
        k32_ms = k32[0] / max(1, k32[1])
        by = linop_bytes_per_element(args.p, args.q, 4) * ne  # the solve's FP32 applies are A P^{-1} v
        # DRAM bytes per k_fused_kry launch: one ncu capture inside the 32^3 mixed solve (347.0 MB read +
        # 260.7 MB written), scaled by the element count; p=4, q=3 only
        kry43 = (args.p, args.q) == (4, 3)
        traffic32 = 607.7e6 * ne / 32 ** 3 if kry43 else None
        traffic32_src = ("ncu dram__bytes_read.sum + dram__bytes_write.sum, 32^3 mixed-solve capture x "
                         f"{ne / 32 ** 3:g} (bytes)") if kry43 else None
        mixed["fp32_kernel"] = {"kernel": fp32_krylov_kernel(args.p, args.q), "launch_ms": k32_ms,
                                "gdofs": dof_slab / (k32_ms / 1e3) / 1e9,
                                "roofline": {"bound": "hbm", "achieved": by / (k32_ms / 1e3) / 1e9, "peak": hbm_peak()[0],
                                             "unit": "GB/s", "frac": by / (k32_ms / 1e3) / 1e9 / hbm_peak()[0],
                                             "traffic": traffic32, "traffic_source": traffic32_src,
                                             "peak_source": hbm_peak()[1]}}
        smx.close()
    except Exception as ex:  # reported, never replaced by another path
        mixed = {"error": repr(ex)}

    extra = {}
    if not args.no_extra:
        for name, fn in (("hp_batch", lambda: leg_hp_batch(fp64_peak)), ("curved", lambda: leg_curved(fp64_peak)),
                         ("serving", leg_serving), ("serving_full", lambda: leg_serving(512, 48)),
                         ("inexact", leg_inexact), ("tm11_hp", leg_tm11_hp),
                         ("cavity_plain", leg_cavity_plain), ("curved_slabs", leg_curved_slabs),
                         ("iteration_study", leg_iteration_study),
                         ("dissipative", lambda: leg_dissipative(fp64_peak)),
                         ("time_refinement", lambda: leg_time_refinement(fp64_peak))):
            if name not in args.legs.split(","):
                continue
            try:
                extra[name] = fn()
            except Exception as ex:  # reported, never replaced by another path
                extra[name] = {"error": repr(ex)}
            torch.cuda.empty_cache()

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu, _ = cpu_baseline(args.p, args.q)
        lat = sorted(r64["step_ms"])
        line = {
            "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"affine {args.n}^3 bricks on [0,1]^3, p={args.p}, q={args.q}, eps/mu U[1,4], "
                                   f"PEC, dt=h/(2p+1); step = one FP64 slab solve (GMRES(10), tol {args.tol:g})",
                       "elements": ne, "dof_per_slab": dof_slab, "parallelism": f"replicas x{world}",
                       "reorth": bool(args.reorth), "l2": "inputs larger than L2 (6.3 GB coefficients)"},
            "residual_applies_per_step": applies, "gmres_iterations_per_step": r64["iterations"],
            "slab_solves_per_s": world / (ms / 1e3), "rel_err_vs_fp64_ref": err64,
            "latency_ms": {"p50": statistics.median(lat),
                           "p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]},
            "roofline": roofline, "mixed": mixed, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clocks, "gpu_launches": r64["launches"],
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_profile_case(args):
    """Small fixed workloads for profiler captures (the same seeds as the bench legs)."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1307_5310_gb300 import meshgen, stm

    n, p = args.n, args.p
    if args.profile_case == "solve":
        m = workload(n, p, args.q)
        prec = {"fp64": stm.STM_FP64, "mixed": stm.STM_MIXED}[args.precision]
        s = stm.Slab(m, precision=prec, tol=args.tol, max_it=400, reorth=bool(args.reorth))
        u = torch.from_numpy(np.random.Generator(np.random.PCG64(1310)).uniform(-1, 1, s.n_state)).cuda()
        for _ in range(args.steps):
            s.set_state(u)
            rc, rep = s.slab_solve(1.0 / n / (2 * p + 1))
        torch.cuda.synchronize()
        print("ok", rc, rep)
        return
    if args.profile_case == "hp":
        m = meshgen.corner_octree_mesh(50, [0.45, 0.2])
        meshgen.random_hp(m, 1307)
        n, p = 200, 7  # dt = (1/200)/15, the hp_batch leg's
    else:
        q = p - 1 if args.profile_case == "curved" else args.q
        m = meshgen.box_mesh(n, p=p, q=q, order="morton", perturb=0.1 if args.profile_case == "curved" else 0.0)
        meshgen.random_materials(m, 1307, 1308)
    s = stm.Slab(m)
    dtp = torch.float64 if args.precision == "fp64" else torch.float32
    U = torch.empty(s.n_trial, dtype=dtp, device="cuda").uniform_(-1, 1)
    R = torch.empty(s.n_test, dtype=dtp, device="cuda")
    prec = stm.STM_FP64 if args.precision == "fp64" else stm.STM_FP32
    for _ in range(args.steps):
        s.residual_apply(U, R, 0.0, 1.0 / n / (2 * p + 1), prec=prec)
    torch.cuda.synchronize()
    print("ok", float(R.abs().sum()))


def main():
    args = parse()
    if args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
