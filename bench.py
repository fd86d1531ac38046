#!/usr/bin/env python
"""Benchmark of the batched chi0 path: Sternheimer solves per second on one GB300.

Workload (default "pdep_L16_48"): one block application of the symmetrised
response chi0bar = v^1/2 chi0 v^1/2 to 64 perturbations on the 48^3 Gaussian-well
model (L = 16 bohr, ecut 7.75 Ha, N_pw = 4169, N_rho = 33833, 64 occupied states),
i.e. 4096 Sternheimer systems, in the mixed path (FP32 CG, FP64 refinement to
cg_tol 1e-10, which keeps drho within 1e-8 of the FP64 oracle).  A step is one
such block apply: perturbations to real space, right-hand sides, P_c, the
batched CG, refinement, and drho.

Printed: one JSON line (rank 0).  `value` is device time with inputs resident in
HBM (CUDA events on the launching stream, L2 flushed between steps outside the
timed interval); `e2e` is the same metric through the host-pointer entry point
with pinned host buffers (copies inside the timed region).  `--impl reference`
times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "pdep_L16_48": dict(config="pdep_L16_48", n_pert=64, pert_seed=5, cg_tol=1e-10,
                        desc="chibar0 block apply, 64 perturbations x 64 occupied states = 4096 "
                             "Sternheimer systems, 48^3 grid, N_pw=4169, N_rho=33833, mixed FP32/FP64"),
    "serve_L16_48": dict(config="pdep_L16_48", n_pert=16, pert_seed=5, cg_tol=1e-10,
                         desc="served stream on the 48^3 model: chibar0 requests of 4-16 perturbations "
                              "(256-1024 Sternheimer systems), Poisson arrivals (seed 6) at 0.3/0.6/0.9 of "
                              "the measured closed-loop capacity, merged into batched applies"),
    "serve_mixed": dict(config=None, n_pert=128, pert_seed=0, cg_tol=1e-10,
                        desc="served mixed stream: one seeded system per grid of {32,48,64}^3 (cell "
                             "N/3 bohr, ecut 9 Ha, N_v = 4 x wells drawn up to what the cell holds, "
                             "0-8 KB atoms) and the 96^3 KB model (N_v 256), one context each; Poisson arrivals (seed 7) at 0.7 of the "
                             "measured capacity of chibar0 requests (80 %, 16-128 perturbations) and "
                             "PDEP Davidson requests (20 %, 16-64 eigenpairs, dav_tol 1e-8) on a system "
                             "drawn uniformly; mixed FP32/FP64, continuously batched"),
    "dyson_P64_W32": dict(config=None, n_pert=64, pert_seed=32, cg_tol=0.0,
                          desc="Dyson step (1 - chibar0)^-1 chibar0 for 32 imaginary frequencies of a "
                               "64 x 64 PDEP-basis chibar0 (negative semidefinite, spectrum in [-8, 0])"),
    "g0_L16_48": dict(config="pdep_L16_48", n_pert=64, pert_seed=41, cg_tol=0.0,
                      desc="G0 Lanczos chains of H for I^SR on the 48^3 model: 64 basis vectors x the 4 "
                           "highest occupied states = 256 chains of 32 steps (FP64, full "
                           "reorthogonalisation), residues and resolvent matrices at 16 complex "
                           "frequencies"),
    "spin_L16_48": dict(config="pdep_L16_48", n_pert=64, pert_seed=5, cg_tol=1e-10,
                        desc="spin-polarised chibar0 block apply on the 48^3 model: channels with wells "
                             "split by +-0.2 Ha, 64 up + 62 down occupied states x 64 perturbations = "
                             "8064 Sternheimer systems, one context per channel (f_s = 1) run "
                             "concurrently, mixed FP32/FP64"),
    "kb_L24_96": dict(config="kb_L24_96", n_pert=256, pert_seed=5, cg_tol=1e-10,
                      desc="chibar0 block apply on the 96^3 model with Kleinman-Bylander projectors: "
                           "256 perturbations x 256 occupied states = 65536 Sternheimer systems, "
                           "N_pw=30095, N_rho=240417, 64 atoms x (well + s,p projectors) = 256 "
                           "projectors, mixed FP32/FP64, device-memory chunks of whole perturbations"),
    "chi0w_L10_24": dict(config="chi0_L10_24", n_pert=32, pert_seed=24, cg_tol=1e-10,
                         desc="full-frequency chibar0 on the 24^3 model: 32 perturbations x 4 occupied states x "
                              "32 Gauss-Legendre imaginary frequencies on [0, 50 Ha] = 4096 complex-shifted "
                              "Sternheimer systems (COCG batched over frequencies, mixed FP32/FP64), and Lanczos "
                              "chains of 64 steps for every (v, pdep) pair (128 chains) with chi0 in the basis at "
                              "the same frequencies"),
    "qp_L10_24": dict(config="chi0_L10_24", n_pert=32, pert_seed=94, cg_tol=0.0,
                      desc="quasiparticle energies of the 4 occupied states of the 24^3 model (Eq. e_qp by secant "
                           "on Sigma_X + I^SR + R): 32 basis vectors (seeded, scaled by 2), chi0 and G0 chains of 16 steps, 16 "
                           "Gauss-Legendre nodes on [0, 20 Ha], eta 0.1 Ha, e_F at mid-gap, FP64 path"),
    "chi0_L10_24": dict(config="chi0_L10_24", n_pert=8, pert_seed=2, cg_tol=1e-10,
                        desc="chi0 apply, 8 perturbations x 4 occupied states = 32 Sternheimer systems, "
                             "24^3 grid, N_pw=515, N_rho=4337, mixed FP32/FP64"),
}


METRIC = "Sternheimer solves/s at 1e-8 rel err vs FP64 oracle; p50/p99 request latency"


def line_config(args, wl, tensor_cores, world):
    """The config object of the block-apply line (both arms)."""
    mixed = args.precision == "mixed"
    return {"workload": args.workload, "desc": wl["desc"], "cg_tol": wl["cg_tol"], "precision": args.precision,
            "fp64_passes": ("float-float" if args.fp64_emulation else "native FP64") if mixed else "n/a",
            "pc_fp32": "tcgen05 3xTF32" if tensor_cores else "CUDA-core FP32",
            "h_fp32": {None: "autotuned (autotune.h_kernel)", 0: "three kernels", 1: "fused kernel"}[
                getattr(args, "fused_h", None)],
            "cg_launch": {None: "device-driven loop (conditional graph node)", 2: "device-driven loop (conditional graph node)",
                          1: "one graph per window", 0: "direct launches"}[getattr(args, "cuda_graphs", None)],
            "l2": "256 MB buffer written between steps, outside the timed interval",
            "parallelism": f"perturbation shards x{world}" if world > 1 else "1 GPU"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        # The raw samples go to $WGW_BENCH_OUT (default: the temporary directory); the line carries
        # their summary.
        out_dir = os.environ.get("WGW_BENCH_OUT") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_bench_{index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        cmd = ["nvidia-smi", "-i", str(self.index),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
               "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
               "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 7:
                    continue
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                for n, v in zip(names, parts[3:7]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


_CPU_STATE = {}


def _cpu_init(config, n_pert, pert_seed, cg_tol):
    """Worker set-up: the model and perturbations of the workload (host only; the ground state
    comes from the generator's cache when it has one)."""
    import synth
    from oracle.model import Model
    s = synth.make_system(config)
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, s.beta_G, s.d_proj)
    phi = synth.perturbations(s.miller_rho, s.L, n_pert, pert_seed)
    _CPU_STATE.update(m=m, dV=m.vsqrt[:, None] * phi, tol=cg_tol)


def _cpu_solve(job):
    """Solves the (v, p) systems of one job until its deadline; returns how many it finished."""
    from oracle import chi0
    systems, deadline = job
    done = 0
    for v, p in systems:
        if time.time() > deadline:
            break
        chi0.sternheimer_cg_drho(_CPU_STATE["m"], _CPU_STATE["dV"][:, [p]], tol=_CPU_STATE["tol"],
                                 systems=[(v, 0)])
        done += 1
    return done


def cpu_baseline(wl, sys_, budget_s=20.0, one_core=True):
    """The FP64 oracle's Sternheimer CG (plain numpy, one thread per process) on a bounded random
    sample of the same systems, one process per host core, each solving its own systems; with
    one_core also a single process.  Processes are spawned (never forked) before any GPU call."""
    import multiprocessing as mp
    import numpy as np
    nv = sys_.n_v
    order = [(v, p) for p in range(wl["n_pert"]) for v in range(nv)]
    pick = [order[i] for i in np.random.default_rng(0).permutation(len(order))]
    cores = os.cpu_count() or 1
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    init = (wl["config"], wl["n_pert"], wl["pert_seed"], wl["cg_tol"])
    desc = "FP64 numpy CG with FFT-applied H to the same cg_tol"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores, initializer=_cpu_init, initargs=init) as pool:
            pool.map(_cpu_solve, [([], 0.0)] * cores)                # set-up outside the timing
            t0 = time.time()
            done = sum(pool.map(_cpu_solve, [(pick[k::cores], t0 + budget_s) for k in range(cores)]))
            dt = time.time() - t0
        res = {"value": done / dt, "unit": "Sternheimer solves/s", "cores": cores, "kind": "oracle",
               "sample": f"{done} of {len(order)} (v, p) systems of the same workload, {desc}, "
                         f"{cores} single-threaded processes, {dt:.1f} s"}
        if one_core:
            with ctx.Pool(1, initializer=_cpu_init, initargs=init) as pool:
                pool.apply(_cpu_solve, (([], 0.0),))
                t0 = time.time()
                one = pool.apply(_cpu_solve, ((pick, t0 + budget_s),))
                dt1 = time.time() - t0
            res["one_core"] = {"value": one / dt1, "sample": f"{one} systems, one process, {dt1:.1f} s"}
        return res
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def run_reference(args, wl):
    import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    s = synth.make_system(wl["config"])
    lat = []
    for _ in range(args.warmup):
        cpu_baseline(wl, s, budget_s=2.0, one_core=False)
    vals = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(wl, s, budget_s=8.0, one_core=False)
        lat.append(time.perf_counter() - t0)
        vals.append(cb["value"])
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC,
            "value": v, "unit": "Sternheimer solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(lat), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": line_config(args, wl, 1, 1),
            "cpu_baseline": {"value": v, "unit": "Sternheimer solves/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "Sternheimer solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_dyson(args, wl):
    """The Dyson step of the next stage (wgw_dyson), host buffers, copies included."""
    import numpy as np
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    torch.cuda.set_device(local)
    from paper_2203_05623_gb300 import build
    build.build()
    import paper_2203_05623_gb300 as W
    n, nw = wl["n_pert"], wl["pert_seed"]
    rng = np.random.default_rng(7)
    A = np.zeros((nw, n, n))
    for k in range(nw):
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        A[k] = (Q * -rng.uniform(0.0, 8.0, n)) @ Q.T
    for _ in range(max(args.warmup, 1)):
        W.wgw_dyson(A)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        W.wgw_dyson(A)
        ts.append(time.perf_counter() - t0)
    total = sum(ts)
    print(json.dumps({"metric": "Dyson solves per second (one n x n matrix per imaginary frequency)",
                      "value": nw * args.steps / total, "unit": "matrices/s", "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": args.workload, "desc": wl["desc"],
                                 "timed": "host call including the host <-> device copies"}}), flush=True)


def run_g0(args, wl):
    """G0 Lanczos chains for I^SR (wgw_g0_lanczos), host buffers, copies included."""
    import numpy as np
    import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    s = synth.make_system(wl["config"])
    phi = synth.perturbations(s.miller_rho, s.L, wl["n_pert"], wl["pert_seed"])
    states = list(range(s.n_v - 4, s.n_v))
    n_steps = 32
    z = np.linspace(-1.0, 1.0, 4)[:, None] + 1j * np.array([0.05, 0.5, 2.0, 8.0])[None, :]
    cpu = None
    if not args.no_cpu_baseline:
        # The oracle's chains on a bounded sample (one state, 32 basis vectors, ~10 s), host cores
        # only, before the first GPU call.
        from oracle import g0 as g0_oracle
        from oracle.model import Model
        m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)
        t0 = time.perf_counter()
        g0_oracle.g0_lanczos(m, phi[:, :32], states[-1:], n_steps, z)
        dt = time.perf_counter() - t0
        cpu = {"value": 32 * n_steps / dt, "unit": "chain steps/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"32 chains (1 state x 32 basis vectors) of {n_steps} steps of the same workload, "
                         f"oracle.g0.g0_lanczos, {dt:.1f} s"}
    import torch
    torch.cuda.set_device(local)
    from paper_2203_05623_gb300 import build
    build.build()
    import paper_2203_05623_gb300 as W
    prec = W.WGW_MIXED if args.precision == "mixed" else W.WGW_FP64
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v,
                      W.wgw_default_options(precision=prec, fp64_emulation=args.fp64_emulation))
    for _ in range(max(args.warmup, 1)):
        W.wgw_g0_lanczos(ctx, phi, states, n_steps, z)
    # One untimed call with every launch bracketed by CUDA events: class shares and the roofline.
    W.wgw_profile_enable(ctx, True)
    W.wgw_g0_lanczos(ctx, phi, states, n_steps, z)
    prof = W.wgw_profile_read(ctx)
    W.wgw_profile_enable(ctx, False)
    ts = []
    with Clocks(local) as clk:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            W.wgw_g0_lanczos(ctx, phi, states, n_steps, z)
            ts.append(time.perf_counter() - t0)
    total = sum(ts)
    units = len(states) * wl["n_pert"] * n_steps
    tot_ms = max(sum(v["ms"] for v in prof.values()), 1e-9)
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    hbm, peak_kind = peaks()
    achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9 if d["ms"] > 0 else 0.0
    line = {"metric": "G0 Lanczos chain steps per second (one application of H per chain and step)",
            "value": units * args.steps / total, "unit": "chain steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "precision": args.precision,
                       "fp64_passes": ("float-float" if args.fp64_emulation else "native FP64")
                       if args.precision == "mixed" else "native FP64",
                       "timed": "host call including the host <-> device copies (35 MB in, 4 MB out)"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None, "peak_source": peak_kind,
                         "launches": d["launches"],
                         "timed_from": "CUDA events around every launch of one untimed call"},
            "kernel_share": {k: round(v["ms"] / tot_ms, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])
                             if v["launches"]},
            "kernel_gbs": {k: round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1)
                           for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"]) if v["ms"] > 0},
            "gpu_launches": int(sum(v["launches"] for v in prof.values())) * args.steps,
            "clocks": clk.summary()}
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


def run_freq(args, wl):
    """Full-frequency chi0(i w): complex-shifted solves batched over 32 imaginary frequencies through
    wgw_apply_chibar0 and Lanczos chains in the basis through wgw_lanczos (host buffers, copies
    included in both timings)."""
    import numpy as np
    import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    s = synth.make_system(wl["config"])
    phi = synth.perturbations(s.miller_rho, s.L, wl["n_pert"], wl["pert_seed"])
    oms, _ = synth.gauss_legendre_omega(32, 50.0)
    n_steps = 64
    cpu = None
    if not args.no_cpu_baseline:
        # The oracle's chains on a bounded sample (8 basis vectors x every state, 64 steps), host
        # cores only, before the first GPU call.
        from oracle import lanczos as lz_oracle
        from oracle.model import Model
        m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)
        t0 = time.perf_counter()
        lz_oracle.chi0_pdep(m, phi[:, :8], oms, n_steps)
        dt = time.perf_counter() - t0
        cpu = {"value": 8 * s.n_v * n_steps / dt, "unit": "chain steps/s", "cores": os.cpu_count(),
               "kind": "oracle", "sample": f"{8 * s.n_v} chains (8 basis vectors x {s.n_v} states) of {n_steps} "
                                           f"steps of the same workload, oracle.lanczos.chi0_pdep, {dt:.1f} s"}
    import torch
    torch.cuda.set_device(local)
    from paper_2203_05623_gb300 import build
    build.build()
    import paper_2203_05623_gb300 as W
    prec = W.WGW_MIXED if args.precision == "mixed" else W.WGW_FP64
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v,
                      W.wgw_default_options(precision=prec, cg_tol=wl["cg_tol"], max_cg_iter=400,
                                            fp64_emulation=args.fp64_emulation))
    for _ in range(max(args.warmup, 1)):
        W.wgw_apply_chibar0(ctx, phi, oms)
        W.wgw_lanczos(ctx, phi, n_steps, oms)
    ts, tl, st = [], [], None
    with Clocks(local) as clk:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            _, st, _ = W.wgw_apply_chibar0(ctx, phi, oms)
            ts.append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            _, _, _, lst = W.wgw_lanczos(ctx, phi, n_steps, oms)
            tl.append(time.perf_counter() - t0)
    n_sys = st["n_systems"]
    line = {"metric": "complex-shifted Sternheimer solves/s at 1e-8 rel err vs FP64 oracle (32 imaginary frequencies)",
            "value": n_sys * args.steps / sum(ts), "unit": "Sternheimer solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(ts) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "cg_tol": wl["cg_tol"],
                       "precision": args.precision,
                       "timed": "host calls including the host <-> device copies"},
            "solve": {"n_systems": n_sys, "max_iters": st["max_iters"], "refinements": st["refinements"],
                      "max_rel_residual": st["max_rel_residual"]},
            "lanczos": {"chains": lst["n_systems"], "steps": n_steps,
                        "value": lst["n_systems"] * n_steps * args.steps / sum(tl), "unit": "chain steps/s",
                        "ms_per_call": 1e3 * sum(tl) / args.steps},
            "clocks": clk.summary()}
    if cpu:
        line["lanczos"]["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


def run_qp(args, wl):
    """Quasiparticle energies through wgw_qp (chains, Sigma_X, I^SR, the residue term and the secant
    iterations all inside one call; host buffers, copies included)."""
    import numpy as np
    import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    s = synth.make_system(wl["config"])
    phi = 2.0 * synth.perturbations(s.miller_rho, s.L, wl["n_pert"], wl["pert_seed"])
    x, wts = np.polynomial.legendre.leggauss(16)
    nodes, weights = 10.0 * (x + 1.0), 10.0 * wts
    n_steps = 16
    cpu = None
    from oracle.model import Model
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)
    e = np.linalg.eigvalsh(m.h_dense())
    e_fermi = 0.5 * (e[s.n_v - 1] + e[s.n_v])
    states = list(range(s.n_v))
    prm = dict(n_steps_chi=n_steps, n_steps_g0=n_steps, nodes=nodes, weights=weights, e_fermi=e_fermi, eta=0.1)
    if not args.no_cpu_baseline:
        # The oracle's Sigma(w) of the highest state at one frequency (its chains, Lambda at the nodes
        # and at the residue frequencies), host cores only, before the first GPU call.
        from oracle import lanczos as lz_oracle, sigma as sg_oracle
        t0 = time.perf_counter()
        chi = lz_oracle.chi0_pdep(m, phi, nodes, n_steps)[0]
        lam = np.array([np.linalg.solve(np.eye(phi.shape[1]) - chi[:, :, k], chi[:, :, k]).real
                        for k in range(nodes.size)])
        i, w = s.n_v - 1, s.e_v[s.n_v - 1] - 0.05

        def lam_fn(z):
            c = lz_oracle.chi0_pdep_z(m, phi, [z], n_steps)[:, :, 0]
            return np.linalg.solve(np.eye(c.shape[0]) - c, c)
        sg_oracle.sigma_x(m, [i])
        sg_oracle.isr(m, phi, [i], n_steps, [w], lam, nodes, weights)
        sg_oracle.residue_term(m, phi, i, [w], e_fermi, 0.1, lam_fn)
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / dt, "unit": "Sigma evaluations/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"Sigma_X + I^SR + R of one state at one frequency with the same basis, chains and "
                         f"nodes (oracle.sigma, oracle.lanczos), {dt:.1f} s"}
    import torch
    torch.cuda.set_device(local)
    from paper_2203_05623_gb300 import build
    build.build()
    import paper_2203_05623_gb300 as W
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options(precision=W.WGW_FP64))
    for _ in range(max(args.warmup, 1)):
        W.wgw_qp(ctx, phi, states, **prm)
    ts, eq, it = [], None, None
    with Clocks(local) as clk:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            eq, sg, it = W.wgw_qp(ctx, phi, states, **prm)
            ts.append(time.perf_counter() - t0)
    line = {"metric": "quasiparticle energies per second (Eq. e_qp, secant on the GPU-evaluated Sigma)",
            "value": len(states) * args.steps / sum(ts), "unit": "QP energies/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(ts) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"],
                       "timed": "host call including the host <-> device copies"},
            "e_qp": [float(v) for v in eq], "e_ks": [float(v) for v in s.e_v], "secant_steps": [int(v) for v in it],
            "clocks": clk.summary()}
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


def run_spin(args, wl):
    """Spin-polarised block apply through wgw_apply_channels (host arrays, copies included)."""
    import numpy as np
    import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    up, dn = synth.make_spin_system(wl["config"])
    phi = synth.perturbations(up.miller_rho, up.L, wl["n_pert"], wl["pert_seed"])
    import torch
    torch.cuda.set_device(local)
    from paper_2203_05623_gb300 import build
    build.build()
    import paper_2203_05623_gb300 as W
    prec = W.WGW_MIXED if args.precision == "mixed" else W.WGW_FP64
    ctxs = [W.wgw_setup(c.L, c.ecut, c.grid, c.vloc_G, c.psi_v, c.e_v,
                        W.wgw_default_options(precision=prec, cg_tol=wl["cg_tol"], f_s=1.0,
                                              fp64_emulation=args.fp64_emulation)) for c in (up, dn)]
    for _ in range(max(args.warmup, 1)):
        W.wgw_apply_channels(ctxs, phi, [0.0], symmetrized=True)
    ts, st = [], None
    with Clocks(local) as clk:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            _, st, _ = W.wgw_apply_channels(ctxs, phi, [0.0], symmetrized=True)
            ts.append(time.perf_counter() - t0)
    total = sum(ts)
    n_sys = st["n_systems"]
    io = wl["n_pert"] * up.n_rho * 16
    print(json.dumps({"metric": "Sternheimer solves/s, spin-polarised (both channels)", "value": n_sys * args.steps / total,
                      "unit": "Sternheimer solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f32/f64" if args.precision == "mixed" else "f64",
                      "data": "synthetic",
                      "config": {"workload": args.workload, "desc": wl["desc"], "precision": args.precision,
                                 "timed": "host call including the host <-> device copies"},
                      "solve": st, "e2e": {"value": n_sys * args.steps / total, "unit": "Sternheimer solves/s",
                                           "h2d_bytes_per_step": 2 * io, "d2h_bytes_per_step": 2 * io},
                      "clocks": clk.summary()}), flush=True)


def run_serve(args, wl):
    """Served stream: requests submitted at Poisson arrival times through wgw_submit/wgw_wait."""
    import numpy as np
    import synth
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    torch.cuda.set_device(local)
    from paper_2203_05623_gb300 import build
    build.build()
    import paper_2203_05623_gb300 as W
    s = synth.make_system(wl["config"])
    pool = synth.perturbations(s.miller_rho, s.L, wl["n_pert"], wl["pert_seed"])
    opt = W.wgw_default_options(precision=W.WGW_MIXED, cg_tol=wl["cg_tol"], max_cg_iter=200)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, opt)
    for _ in range(max(args.warmup, 1)):
        W.wgw_apply_chibar0(ctx, pool)
    t0 = time.perf_counter()
    _, st, _ = W.wgw_apply_chibar0(ctx, pool)
    capacity = st["n_systems"] / (time.perf_counter() - t0)      # closed-loop systems/s
    rng = np.random.default_rng(6)
    results = []
    with Clocks(local) as clk:
        for load in (0.3, 0.6, 0.9):
            sizes = rng.integers(4, wl["n_pert"] + 1, size=100000)
            mean_sys = float(np.mean(sizes)) * s.n_v
            rate = load * capacity / mean_sys                       # requests/s
            duration = max(2.0, 4.0 * args.steps)
            gaps = rng.exponential(1.0 / rate, size=100000)
            arrivals = np.cumsum(gaps)
            n_req = int(np.searchsorted(arrivals, duration))
            tickets, t_start = [], time.perf_counter()
            for k in range(n_req):
                dt = arrivals[k] - (time.perf_counter() - t_start)
                if dt > 0:
                    time.sleep(dt)
                cols = rng.choice(wl["n_pert"], size=int(sizes[k]), replace=False)
                tickets.append((W.wgw_submit(ctx, pool[:, cols]), int(sizes[k]) * s.n_v))
            lat, systems, merged = [], 0, []
            for t, nsys in tickets:
                _, res = W.wgw_wait(t)
                if res["status"] != W.WGW_OK:
                    raise RuntimeError(f"request failed with status {res['status']}")
                lat.append(res["latency_s"])
                merged.append(res["batch_requests"])
                systems += nsys
            span = time.perf_counter() - t_start
            lat = np.sort(np.array(lat))
            results.append({"load": load, "requests": n_req, "offered_systems_per_s": load * capacity,
                            "served_systems_per_s": systems / span,
                            "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                                           "p99": 1e3 * float(np.percentile(lat, 99))},
                            "mean_requests_per_batch": float(np.mean(merged))})
    if rank == 0:
        mid = results[1]
        print(json.dumps({
            "metric": "served Sternheimer solves/s and request latency (arrival -> result on the host)",
            "value": mid["served_systems_per_s"], "unit": "Sternheimer solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "cg_tol": wl["cg_tol"],
                       "closed_loop_capacity_systems_per_s": capacity},
            "latency_ms": mid["latency_ms"], "loads": results, "clocks": clk.summary()}), flush=True)
    W.wgw_destroy(ctx)


def run_serve_mixed(args, wl):
    """Served mixed stream over contexts of different grids: chibar0 and PDEP requests submitted at
    Poisson arrival times through wgw_submit / wgw_submit_pdep, collected with wgw_wait."""
    import numpy as np
    import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    torch.cuda.set_device(local)
    from paper_2203_05623_gb300 import build
    build.build()
    import paper_2203_05623_gb300 as W
    t_gs = time.perf_counter()
    systems = [synth.make_system(c) for c in synth.serve_stream_configs()]
    t_gs = time.perf_counter() - t_gs
    ctxs, pools, caps = [], [], []
    for s in systems:
        kb = s.beta_G.shape[1] > 0
        opt = W.wgw_default_options(precision=W.WGW_MIXED, cg_tol=wl["cg_tol"], max_cg_iter=300, dav_tol=1e-8)
        ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, opt,
                          beta_G=s.beta_G if kb else None, d_proj=s.d_proj if kb else None)
        pool = synth.perturbations(s.miller_rho, s.L, wl["n_pert"], s.cfg.pert_seed)
        for _ in range(max(args.warmup, 1)):
            W.wgw_apply_chibar0(ctx, pool[:, :16])
        t0 = time.perf_counter()
        _, st, _ = W.wgw_apply_chibar0(ctx, pool[:, :32])
        caps.append(st["n_systems"] / (time.perf_counter() - t0))     # closed-loop systems/s
        ctxs.append(ctx)
        pools.append(pool)
    rng = np.random.default_rng(7)
    n_sys = len(systems)
    # Mean GPU time of a request (a PDEP request costs about 6 block applications of its size).
    mean_t = np.mean([(0.8 * 72 + 0.2 * 6 * 40) * s.n_v / caps[k] for k, s in enumerate(systems)])
    load = 0.7
    rate = load / mean_t
    duration = float(max(20.0, 12.0 * args.steps))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=100000))
    n_req = max(1, int(np.searchsorted(arrivals, duration)))
    plan = []
    for k in range(n_req):
        sys_k = int(rng.integers(n_sys))
        if rng.random() < 0.2:
            plan.append(("pdep", sys_k, int(rng.integers(16, 65)), None))
        else:
            n = int(rng.integers(16, 129))
            plan.append(("chibar0", sys_k, n, np.sort(rng.choice(wl["n_pert"], size=n, replace=False))))
    tickets = []
    with Clocks(local) as clk:
        t_start = time.perf_counter()
        for k, (kind, sys_k, n, cols) in enumerate(plan):
            dt = arrivals[k] - (time.perf_counter() - t_start)
            if dt > 0:
                time.sleep(dt)
            if kind == "pdep":
                tickets.append(W.wgw_submit_pdep(ctxs[sys_k], n))
            else:
                tickets.append(W.wgw_submit(ctxs[sys_k], pools[sys_k][:, cols], [0.0], kind=W.WGW_REQ_CHIBAR0))
        lat, solved, per_kind = [], 0, {"chibar0": [], "pdep": []}
        outs = []
        for (kind, sys_k, n, cols), t in zip(plan, tickets):
            out, res = W.wgw_wait(t)
            if res["status"] != W.WGW_OK:
                raise RuntimeError(f"{kind} request on system {sys_k} failed with status {res['status']}")
            lat.append(res["latency_s"])
            per_kind[kind].append(res["latency_s"])
            solved += res["batch_systems"] if kind == "pdep" else n * systems[sys_k].n_v
            outs.append(out)
        span = time.perf_counter() - t_start
    # Served results against the same request alone (first chibar0 request of every system).
    diff = 0.0
    for sys_k in range(n_sys):
        for (kind, sk, n, cols), out in zip(plan, outs):
            if kind == "chibar0" and sk == sys_k:
                alone, _, _ = W.wgw_apply_chibar0(ctxs[sys_k], pools[sys_k][:, cols])
                num = np.linalg.norm((out - alone).reshape(out.shape[0], -1), axis=0)
                den = np.linalg.norm(alone.reshape(alone.shape[0], -1), axis=0)
                diff = max(diff, float(np.max(num / den)))
                break

    def pct(v, q):
        return 1e3 * float(np.percentile(np.asarray(v), q)) if len(v) else None

    print(json.dumps({
        "metric": "served Sternheimer solves/s and request latency (arrival -> result on the host)",
        "value": solved / span, "unit": "Sternheimer solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "cg_tol": wl["cg_tol"],
                   "systems": [{"grid": s.grid, "n_pw": s.n_pw, "n_v": s.n_v, "kb_atoms": int(len(np.unique(s.proj_atom))),
                                "closed_loop_systems_per_s": caps[k]} for k, s in enumerate(systems)],
                   "offered_load": load, "arrival_window_s": duration, "ground_states_s": t_gs},
        "requests": n_req, "span_s": span,
        "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99)},
        "latency_ms_chibar0": {"p50": pct(per_kind["chibar0"], 50), "p99": pct(per_kind["chibar0"], 99)},
        "latency_ms_pdep": {"p50": pct(per_kind["pdep"], 50), "p99": pct(per_kind["pdep"], 99)},
        "served_vs_alone_rel_diff": diff, "clocks": clk.summary()}), flush=True)
    for c in ctxs:
        W.wgw_destroy(c)


def served_stream(W, ctx, s, phi, capacity, window_s=8.0, load=0.7, seed=11):
    """Served chibar0 requests on the context of the main line: Poisson arrivals (seed) at `load`
    of the closed-loop capacity (systems/s) for window_s seconds, each request 4-64 perturbations
    drawn from phi's columns, submitted through wgw_submit and collected with wgw_wait; latency =
    submission -> result in host memory (measured by the library).  The first request is solved
    again alone and compared with its served result."""
    import numpy as np
    rng = np.random.default_rng(seed)
    n_pool = phi.shape[1]
    sizes = rng.integers(4, min(64, n_pool) + 1, size=100000)
    rate = load * capacity / (float(np.mean(sizes)) * s.n_v)          # requests/s
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=100000))
    n_req = max(2, int(np.searchsorted(arrivals, window_s)))
    cols = [np.sort(rng.choice(n_pool, size=int(sizes[k]), replace=False)) for k in range(n_req)]
    tickets, t_start = [], time.perf_counter()
    for k in range(n_req):
        dt = arrivals[k] - (time.perf_counter() - t_start)
        if dt > 0:
            time.sleep(dt)
        tickets.append(W.wgw_submit(ctx, phi[:, cols[k]], [0.0], kind=W.WGW_REQ_CHIBAR0))
    lat, solved, merged, first = [], 0, [], None
    for k, t in enumerate(tickets):
        out, res = W.wgw_wait(t)
        if res["status"] != W.WGW_OK:
            raise RuntimeError(f"served request failed with status {res['status']}: {res.get('error')}")
        lat.append(res["latency_s"])
        merged.append(res["batch_requests"])
        solved += len(cols[k]) * s.n_v
        if k == 0:
            first = out
    span = time.perf_counter() - t_start
    alone, _, _ = W.wgw_apply_chibar0(ctx, phi[:, cols[0]])
    num = np.linalg.norm((first - alone).reshape(first.shape[0], -1), axis=0)
    den = np.linalg.norm(alone.reshape(alone.shape[0], -1), axis=0)
    lat = np.asarray(lat)
    return {"requests": n_req, "offered_load": load, "offered_systems_per_s": load * capacity,
            "served_systems_per_s": solved / span, "arrival_window_s": window_s, "span_s": span,
            "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99))},
            "mean_requests_per_batch": float(np.mean(merged)),
            "served_vs_alone_rel_diff": float(np.max(num / den)),
            "what": "chibar0 requests of 4-64 perturbations of the same model, Poisson arrivals at the offered "
                    "load through wgw_submit / wgw_wait, continuously batched; latency = submission -> result "
                    "in host memory"}


def library_baselines(W, ctx, s, prof_all):
    """The library's FP32 kernels against cuFFT and cuBLAS on the same shapes (untimed by the
    bench line; CUDA events around each variant, after warm-up).

    H psi for 1024 real-in-r wavefunctions (512 packed pairs) of the 48^3 model: the library's
    pruned FFT pipeline (wgw_apply_h_dev, FP32, including its sphere <-> real-basis conversions)
    against scatter + torch.fft.ifftn + V(r) + torch.fft.fftn + gather + kinetic term on the full
    complex64 grid (cuFFT).  P_c of 4096 FP32 systems against the 64 occupied states: the
    library's per-system time from the untimed profiled step against torch.matmul (cuBLAS) for
    C = Psi^T X, X -= Psi C in FP32 and in TF32."""
    import numpy as np
    import torch
    import synth

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    n_psi, N = 1024, s.grid
    x = synth.perturbations(s.miller_wfc, s.L, n_psi, 73)
    xd = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()
    outd = torch.empty_like(xd)
    ours_h = timed(lambda: W.wgw_apply_h_dev(ctx, xd, outd, fp32=True))
    mw = np.asarray(s.miller_wfc) % N
    idx = torch.from_numpy((mw[:, 0] * N + mw[:, 1]) * N + mw[:, 2]).cuda()
    b = 2.0 * np.pi / s.L
    kin = torch.from_numpy(0.5 * b * b * np.sum(np.asarray(s.miller_wfc, np.float64) ** 2, axis=1)).float().cuda()
    Xp = (xd[0::2] + 1j * xd[1::2]).to(torch.complex64)          # packed pairs: psi_a + i psi_b
    grid = torch.zeros((n_psi // 2, N ** 3), dtype=torch.complex64, device="cuda")
    vr = torch.rand((N, N, N), device="cuda")

    def cufft_h():
        grid.zero_()
        grid[:, idx] = Xp
        r = torch.fft.ifftn(grid.view(-1, N, N, N), dim=(1, 2, 3))
        r.mul_(vr)
        f = torch.fft.fftn(r, dim=(1, 2, 3)).view(n_psi // 2, -1)
        return f[:, idx] + kin * Xp

    def cufft_only():
        r = torch.fft.ifftn(grid.view(-1, N, N, N), dim=(1, 2, 3))
        return torch.fft.fftn(r, dim=(1, 2, 3))

    cu_h = timed(cufft_h)
    cu_fft = timed(cufft_only)
    del grid
    # P_c GEMMs.
    n, nv, n_sys = 2 * (s.miller_wfc.shape[0] // 2) + 1, s.psi_v.shape[1], 4096
    psi = torch.randn((n, nv), device="cuda")
    X = torch.randn((n, n_sys), device="cuda")

    def pc():
        C = psi.t() @ X
        return X - psi @ C

    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    cu_pc32 = timed(pc)
    torch.backends.cuda.matmul.allow_tf32 = True
    cu_pc_tf32 = timed(pc)
    torch.backends.cuda.matmul.allow_tf32 = old
    d = prof_all.get("pc_project", {"ms": 0.0, "launches": 0, "bytes": 0.0})
    # Algorithmic bytes per pc_project launch: 2 n_list n 4 + n nv 4.
    sys_done = (d["bytes"] - d["launches"] * n * nv * 4.0) / (8.0 * n)
    ours_pc = d["ms"] / sys_done * n_sys if sys_done > 0 else None
    return {"h_psi_1024_wavefunctions_ms": {"library_fp32": ours_h, "cufft_complex64": cu_h,
                                            "cufft_fft_pair_only": cu_fft},
            "pc_4096_systems_ms": {"library_tcgen05_3xtf32": ours_pc, "cublas_fp32": cu_pc32,
                                   "cublas_tf32": cu_pc_tf32},
            "what": "same shapes on the same GPU; library P_c per 4096 systems from the profiled step's "
                    "pc_project class (lists of varying length), cuBLAS as one call on 4096 systems"}


def largest_config(W, stream, hbm, peak_kind, steps=2):
    """The largest single-GPU configuration (96^3 grid, 256 KB projectors, 256 occupied states,
    256 perturbations = 65536 Sternheimer systems, mixed path) measured beside the main line: one
    warm-up apply, `steps` timed applies (CUDA events), one end-to-end apply through the host
    entry point, and the per-class kernel shares of one profiled apply."""
    import numpy as np
    import torch
    import synth
    wl = WORKLOADS["kb_L24_96"]
    t0 = time.perf_counter()
    s = synth.make_system(wl["config"])             # iterative ground state (cached on disk)
    t_gs = time.perf_counter() - t0
    phi = synth.perturbations(s.miller_rho, s.L, wl["n_pert"], wl["pert_seed"])
    opt = W.wgw_default_options(precision=W.WGW_MIXED, cg_tol=wl["cg_tol"], max_cg_iter=200)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, opt, beta_G=s.beta_G, d_proj=s.d_proj)
    x = torch.from_numpy(np.ascontiguousarray(phi.T)).cuda()
    out = torch.zeros((1, wl["n_pert"], s.n_rho), dtype=torch.complex128, device="cuda")
    st, _ = W.wgw_apply_chibar0_dev(ctx, x, [0.0], out, stream=stream.cuda_stream)     # warm-up
    times = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st, _ = W.wgw_apply_chibar0_dev(ctx, x, [0.0], out, stream=stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b) / 1e3)
    W.wgw_profile_enable(ctx, True)
    W.wgw_apply_chibar0_dev(ctx, x, [0.0], out, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    prof = W.wgw_profile_read(ctx)
    W.wgw_profile_enable(ctx, False)
    del x
    ph = np.ascontiguousarray(phi.T)
    oh = np.zeros((1, wl["n_pert"], s.n_rho), np.complex128)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    W.wgw_apply_chibar0(ctx, ph.T, [0.0], out=oh)
    e2e = time.perf_counter() - t1
    W.wgw_destroy(ctx)
    n = st["n_systems"]
    tot = max(sum(v["ms"] for v in prof.values()), 1e-9)
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    if dom == "pc_project_f64":
        # The float-float projector is bound by FP32 issue: one float-float multiply-add (2 flops at
        # FP64 accuracy) takes 12 FP32 instructions, so its peak is the FP32 lane rate / 6.
        roof = {"bound": "alu", "kernel": dom, "unit": "TFLOP/s",
                "achieved": d["flops"] / (d["ms"] / 1e3) / 1e12 if d["ms"] > 0 else 0.0,
                "peak": 152 * 128 * 2.07e9 * 2 / 12 / 1e12,
                "peak_source": "152 SMs x 128 FP32 lanes x 2.07 GHz / 12 instructions per float-float multiply-add (2 flops)"}
    else:
        roof = {"bound": "hbm", "kernel": dom, "unit": "GB/s",
                "achieved": d["bytes"] / (d["ms"] / 1e3) / 1e9 if d["ms"] > 0 else 0.0, "peak": hbm,
                "peak_source": peak_kind}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["timed_from"] = "one profiled apply, every launch bracketed by CUDA events"
    return {"workload": "kb_L24_96", "desc": wl["desc"], "value": n * steps / sum(times),
            "unit": "Sternheimer solves/s", "ms_per_step": 1e3 * sum(times) / steps, "steps": steps, "warmup": 1,
            "solve": {"n_systems": n, "max_iters": st["max_iters"], "refinements": st["refinements"],
                      "max_rel_residual": st["max_rel_residual"]},
            "e2e": {"value": n / e2e, "unit": "Sternheimer solves/s", "h2d_bytes_per_step": int(ph.nbytes),
                    "d2h_bytes_per_step": int(oh.nbytes)},
            "kernel_share": {k: round(v["ms"] / tot, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])
                             if v["launches"]},
            "kernel_gbs": {k: round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1)
                           for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"]) if v["ms"] > 0},
            "roofline": roof,
            "ground_state_s": t_gs}


def fp64_path(W, s, wl, x, out_mixed, stream, ph, oh, steps):
    """The same workload on the all-FP64 GPU path (FP64 CG to the same cg_tol, native FP64 FFT
    passes), measured in the same process: device time, end to end through the host-pointer
    entry point, and the relative difference of the mixed path's result from it."""
    import numpy as np
    import torch
    kb = s.beta_G.shape[1] > 0
    opt = W.wgw_default_options(precision=W.WGW_FP64, cg_tol=wl["cg_tol"], max_cg_iter=2000)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, opt,
                      beta_G=s.beta_G if kb else None, d_proj=s.d_proj if kb else None)
    out = torch.zeros_like(out_mixed)
    st, _ = W.wgw_apply_chibar0_dev(ctx, x, [0.0], out, stream=stream.cuda_stream)   # warm-up
    times = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st, _ = W.wgw_apply_chibar0_dev(ctx, x, [0.0], out, stream=stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b) / 1e3)
    e2e = []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        W.wgw_apply_chibar0(ctx, ph.T, [0.0], out=oh)
        e2e.append(time.perf_counter() - t0)
    ref = out[0].cpu().numpy()
    mix = out_mixed[0].cpu().numpy()
    diff = float(np.max(np.linalg.norm(mix - ref, axis=1) / np.linalg.norm(ref, axis=1)))
    W.wgw_destroy(ctx)
    n = st["n_systems"]
    return {"value": n * steps / sum(times), "unit": "Sternheimer solves/s", "ms_per_step": 1e3 * sum(times) / steps,
            "e2e": {"value": n * steps / sum(e2e), "unit": "Sternheimer solves/s"},
            "max_rel_residual": st["max_rel_residual"], "max_iters": st["max_iters"],
            "mixed_vs_fp64_rel_diff": diff,
            "what": "same workload, all-FP64 GPU path (FP64 CG and FFT passes), same process; "
                    "mixed_vs_fp64_rel_diff = max over perturbations of ||mixed - fp64|| / ||fp64||"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="pdep_L16_48", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-largest", action="store_true",
                    help="skip the 96^3 / 65536-system configuration measured beside the default line")
    ap.add_argument("--no-fp64-path", action="store_true",
                    help="skip the all-FP64 GPU path measured beside the mixed one")
    ap.add_argument("--no-library-baselines", action="store_true",
                    help="skip the cuFFT / cuBLAS comparison on the same shapes")
    ap.add_argument("--no-served", action="store_true",
                    help="skip the served-request stream on the main line's model")
    ap.add_argument("--n-pert", type=int, default=0,
                    help="perturbations per rank (default: the workload's); smaller values serve profiling")
    ap.add_argument("--fp64-emulation", type=int, default=1, choices=[0, 1],
                    help="1: FP64-accuracy FFT passes in float-float (default); 0: native FP64")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="mixed (FP32 CG + FP64-accuracy refinement, default) or the all-FP64 path")
    ap.add_argument("--fused-h", type=int, default=None, choices=[0, 1],
                    help="FP32 H application as one fused kernel per pair (default: the library's)")
    ap.add_argument("--tensor-cores", type=int, default=None, choices=[0, 1],
                    help="P_c of the FP32 solves on the tcgen05 tensor cores (default: the library's)")
    ap.add_argument("--cuda-graphs", type=int, default=None, choices=[0, 1, 2],
                    help="CG launch mode: 2 device-driven loop, 1 a graph per window, 0 direct (default: 2)")
    ap.add_argument("--fft-kernels", default=None,
                    help="FP32 FFT stage kernels G->r,x-line,r->G as three of 0 register, 1 register packed, "
                         "2 shared memory (default: autotuned); fixed choices keep a profiler's replays from "
                         "steering the autotuner")
    ap.add_argument("--tc-split", type=int, default=None,
                    help="tensor-core projector K split (default: autotuned)")
    ap.add_argument("--h-chunk", type=int, default=None,
                    help="pairs per L2-resident chunk of the FP32 H pipeline, 0 = none (default: autotuned)")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.n_pert > 0:
        wl["n_pert"] = args.n_pert
        wl["desc"] += f" (reduced to {args.n_pert} perturbations)"
    if args.impl == "reference":
        return run_reference(args, wl)
    if args.workload == "serve_mixed":
        return run_serve_mixed(args, wl)
    if args.workload.startswith("serve"):
        return run_serve(args, wl)
    if args.workload.startswith("dyson"):
        return run_dyson(args, wl)
    if args.workload.startswith("g0"):
        return run_g0(args, wl)
    if args.workload.startswith("spin"):
        return run_spin(args, wl)
    if args.workload == "chi0w_L10_24":
        return run_freq(args, wl)
    if args.workload == "qp_L10_24":
        return run_qp(args, wl)

    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import synth
    s = synth.make_system(wl["config"])
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, s)            # host-only work before the first GPU call
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2203_05623_gb300 import build
    build.build()
    import paper_2203_05623_gb300 as W

    # Each rank owns one block of n_pert perturbations of a global seeded batch (no collective
    # on the data path: the (v, p) systems are independent).
    from paper_2203_05623_gb300.shard import owned_perturbations
    phi_all = synth.perturbations(s.miller_rho, s.L, wl["n_pert"] * world, wl["pert_seed"])
    phi = phi_all[:, owned_perturbations(wl["n_pert"] * world, rank, world, wl["n_pert"])]
    if args.precision == "fp64":
        opt = W.wgw_default_options(precision=W.WGW_FP64, cg_tol=wl["cg_tol"], max_cg_iter=2000)
    else:
        opt = W.wgw_default_options(precision=W.WGW_MIXED, cg_tol=wl["cg_tol"], max_cg_iter=200,
                                    fp64_emulation=args.fp64_emulation)
    if args.tensor_cores is not None:
        opt.tensor_cores = args.tensor_cores
    if args.fused_h is not None:
        opt.fused_h = args.fused_h
    if args.cuda_graphs is not None:
        opt.cuda_graphs = args.cuda_graphs
    if args.fft_kernels is not None:
        opt.fft_kernels = (ctypes.c_int * 3)(*[int(v) for v in args.fft_kernels.split(",")])
    if args.tc_split is not None:
        opt.tc_split = args.tc_split
    if args.h_chunk is not None:
        opt.h_chunk_pairs = args.h_chunk
    kb = s.beta_G.shape[1] > 0
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, opt,
                      beta_G=s.beta_G if kb else None, d_proj=s.d_proj if kb else None)
    stream = torch.cuda.current_stream()
    x = torch.from_numpy(np.ascontiguousarray(phi.T)).cuda()
    out = torch.zeros((1, wl["n_pert"], s.n_rho), dtype=torch.complex128, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        st, _ = W.wgw_apply_chibar0_dev(ctx, x, [0.0], out, stream=stream.cuda_stream)
        return st

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    # One more untimed step with every launch bracketed by events: per-class shares, launches
    # per step and the dominant class.  Bracketing every launch stretches a step by ~15 %, so the
    # timed steps below bracket only the launches of the dominant class.
    W.wgw_profile_enable(ctx, True)
    step()
    torch.cuda.synchronize()
    prof_all = W.wgw_profile_read(ctx)
    W.wgw_profile_enable(ctx, False)
    dom = max(prof_all, key=lambda k: prof_all[k]["ms"])
    launches_per_step = int(sum(v["launches"] for v in prof_all.values()))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    W.wgw_profile_classes(ctx, [dom])
    W.wgw_profile_enable(ctx, True)
    times, stats = [], None
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)                      # evict L2 between steps (outside the timed interval)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            stats = step()
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b) / 1e3)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    prof = W.wgw_profile_read(ctx)
    W.wgw_profile_enable(ctx, False)
    W.wgw_profile_classes(ctx, None)
    total = sum(times)
    if dist:
        t = torch.tensor([total], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    n_sys = stats["n_systems"]
    value = world * n_sys * args.steps / total

    # End to end through the host-pointer entry point (pinned buffers, copies timed).
    ph = torch.from_numpy(np.ascontiguousarray(phi.T)).pin_memory().numpy()
    oh = torch.zeros((1, wl["n_pert"], s.n_rho), dtype=torch.complex128).pin_memory().numpy()
    W.wgw_apply_chibar0(ctx, ph.T, [0.0], out=oh)
    e2e_t = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        W.wgw_apply_chibar0(ctx, ph.T, [0.0], out=oh)
        e2e_t.append(time.perf_counter() - t0)
    e2e_total = sum(e2e_t)
    if dist:
        t = torch.tensor([e2e_total], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())
    io_bytes = wl["n_pert"] * s.n_rho * 16

    hbm, peak_kind = peaks()
    d = prof[dom]
    per_launch = d["bytes"] / max(d["launches"], 1)
    if dom == "pc_project_f64":
        # Float-float projector: FP32-issue-bound, 12 FP32 instructions per float-float multiply-add.
        bound, unit, peak = "alu", "TFLOP/s", 152 * 128 * 2.07e9 * 2 / 12 / 1e12
        peak_src = "152 SMs x 128 FP32 lanes x 2.07 GHz / 12 instructions per float-float multiply-add (2 flops)"
        achieved = d["flops"] / (d["ms"] / 1e3) / 1e12 if d["ms"] > 0 else 0.0
    elif dom in ("pc_project", "hpsi_fused"):
        # CUDA-core FP32 GEMMs, or the fused H kernel whose FFT intermediate never leaves the SMs:
        # bound by the FP32 FMA rate (152 SMs x 128 lanes x 2 flop x 2.07 GHz).  The fused kernel's
        # flops are counted as 5 n log2 n per length-n line transform.
        bound, unit, peak, peak_src = "alu", "TFLOP/s", 152 * 128 * 2 * 2.07e9 / 1e12, "FP32 FMA unit count x max SM clock"
        achieved = d["flops"] / (d["ms"] / 1e3) / 1e12 if d["ms"] > 0 else 0.0
    else:
        bound, unit, peak, peak_src = "hbm", "GB/s", hbm, peak_kind
        achieved = per_launch / (d["ms"] / 1e3 / max(d["launches"], 1)) / 1e9 if d["ms"] > 0 else 0.0
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f).get(args.workload, {}).get(dom)
        if t:
            traffic = t["dram_over_algorithmic"] * per_launch
    except Exception:
        traffic = None
    line = {
        "metric": METRIC,
        "value": value, "unit": "Sternheimer solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": line_config(args, wl, opt.tensor_cores, world),
        "latency_ms": {"p50": 1e3 * statistics.median(times),
                       "p99": 1e3 * sorted(times)[min(len(times) - 1, int(0.99 * len(times)))],
                       "what": "one block-apply request, device time"},
        "solve": {"n_systems": n_sys, "max_iters": stats["max_iters"], "refinements": stats["refinements"],
                  "max_rel_residual": stats["max_rel_residual"]},
        "e2e": {"value": world * n_sys * args.steps / e2e_total, "unit": "Sternheimer solves/s",
                "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes},
        "roofline": {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak, "unit": unit,
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": per_launch,
                     "launches": d["launches"], "avg_launch_ms": d["ms"] / max(d["launches"], 1),
                     "timed_from": "CUDA events around each launch of this class inside the timed steps",
                     "traffic_from": "DRAM/algorithmic byte ratio of one ncu capture (profiles/traffic.json) "
                                     "x the algorithmic bytes of the average timed launch"},
        "kernel_share": {k: round(v["ms"] / max(sum(q["ms"] for q in prof_all.values()), 1e-9), 4)
                         for k, v in sorted(prof_all.items(), key=lambda kv: -kv[1]["ms"]) if v["launches"]},
        "kernel_share_from": "one untimed step after warm-up with every launch bracketed by CUDA events",
        "kernel_gbs": {k: round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1)
                       for k, v in sorted(prof_all.items(), key=lambda kv: -kv[1]["ms"]) if v["ms"] > 0},
        "kernel_gbs_what": "algorithmic bytes of each class (the kernels' own inputs and outputs) / its event time",
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
    }
    if cpu:
        line["cpu_baseline"] = cpu
    line["autotune"] = W.wgw_autotune_info(ctx)
    line["autotune"]["fft"] = W.wgw_autotune_fft(ctx)
    line["autotune"]["h_chunk"] = W.wgw_autotune_chunk(ctx)
    if world == 1 and args.precision == "mixed" and not args.no_fp64_path and args.workload == "pdep_L16_48":
        line["fp64_path"] = fp64_path(W, s, wl, x, out, stream, ph, oh, min(args.steps, 3))
    if world == 1 and args.precision == "mixed" and not args.no_library_baselines:
        line["library_baseline"] = library_baselines(W, ctx, s, prof_all)
    if world == 1 and args.precision == "mixed" and args.workload == "pdep_L16_48" and not args.no_served:
        served = served_stream(W, ctx, s, phi, value)
        line["served"] = served
        line["latency_ms"] = dict(served["latency_ms"], what="served chibar0 requests (the served object)")
        line["block_apply_ms"] = {"p50": 1e3 * statistics.median(times),
                                  "what": "one 64-perturbation block apply, device time"}
    W.wgw_destroy(ctx)
    if world == 1 and args.precision == "mixed" and args.workload == "pdep_L16_48" and not args.no_largest:
        line["largest_config"] = largest_config(W, stream, hbm, peak_kind)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
