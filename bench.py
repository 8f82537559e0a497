#!/usr/bin/env python
"""Benchmark of the Schur-complement solve on one GB300 (or N replicas).

A step is the whole hot path on the 8^4 workload: for each of the four site
permutations P_I, P_II, P_I^T, P_II^T (Type II along x0), solve D x = f
through S_bb = D_bb - D_br D_rr^-1 D_rb -- inner BiCGStab on D_rr to 1e-12,
outer GMRES(30) on S_bb to 1e-10, back-substitution, and the FP64 true
residual ||f - D x|| / ||f||.  The four solves run at once
(schur_solve_batched, one context and stream per permutation); the line also
gives the same four solves one after another.  Field: SU(3) plaquette action at beta = 5.4
(200 Cabibbo-Marinari sweeps from a cold start, seed 1), Wilson m0 = -0.4,
one complex Gaussian source (seed 100).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead on the same step: the four permutations' complete solves,
one single-threaded oracle process per permutation on four host cores
(warm-up steps: one S_bb apply per process).  Further sections of the line:
mixed-precision and learned (network + FGMRES) inner solves on the same
workload, the 16^3 x 32 Type II mixed-precision workload, Table 1 of the
paper on the GPU (plain and V-cycle-preconditioned BiCGStab on the three
stand-in fields), the low-precision stencil on 32^3 x 64, one source of the
32^3 x 64 learned-preconditioner workload, and the batched workload (20
sources on 24^3 x 48, 16^4 and 8^4 solved together, against one at a time).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("S_bb solve time to 1e-10 rel. residual (learned+mixed vs plain FP64); "
          "dslash GB/s vs HBM peak")
UNIT = "S_bb solves/s"
WORKLOAD = ("8^4 SU(3) plaquette action beta=5.4 (200 Cabibbo-Marinari sweeps, cold start, "
            "seed 1), Wilson m0=-0.4 r=1, FP64, P_I/P_II/P_I^T/P_II^T (Type II along x0), "
            "outer GMRES(30) to 1e-10, inner BiCGStab to 1e-12, back-substitution, "
            "one Gaussian source (seed 100)")
PERMS = [(1, 0, 0), (2, 0, 0), (1, 0, 1), (2, 0, 1)]
FIELD = "8^4 heatbath b5.4"
M0 = -0.4
# nominal FP64 rate: 152 SMs x 2.07 GHz x 4 FP64 flop/clk/SM (1.26 TFLOP/s); the
# roofline divides by the rate gs_fp64_peak measures on the GPU at hand
FP64_NOMINAL_TFLOPS = 152 * 2.07e9 * 4 / 1e12
# Table 1 (Section 4): kappa = 1/6, the coarsening steps of each coupling and the
# paper's printed values (condition number, R plain, R with the V-cycle)
TABLE1_LEVELS = {5.4: [(1, 0, 1), (1, 0, 1)], 5.7: [(1, 0, 1), (1, 0, 1)],
                 5.9: [(2, 0, 1), (2, 1, 1)]}
TABLE1_PAPER = {5.4: (57, 0.76, 0.05), 5.7: (480, 0.83, 0.16), 5.9: (905, 0.89, 0.48)}
PERM_NAMES = ["P_I", "P_II", "P_I^T", "P_II^T"]
# DRAM traffic per launch from one ncu capture, per profiled kernel family
# (3: the persistent FP64 BiCGStab, the step's dominant kernel), with the hash
# of the sources it was taken on; other families report no traffic
NCU_SUMMARY = {3: (os.path.join(ROOT, "profiles", "bicg_persistent_f64_8x4_traffic.txt"),
                   ("persistent.cu", "dslash_f64.cuh", "gridsync.cuh"))}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _kernel_source_hash(files):
    import hashlib
    h = hashlib.sha256()
    for name in files:
        with open(os.path.join(ROOT, "paper_0704_2341_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic_per_launch(family):
    """DRAM bytes per launch of a kernel family from its committed ncu
    summary, or None if absent or taken on a different kernel source."""
    try:
        path, files = NCU_SUMMARY[family]
        kv = {}
        for line in open(path):
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha") != _kernel_source_hash(files):
            return None
        return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        import tempfile
        self.path = os.path.join(os.environ.get("GSCHUR_CLOCK_LOG_DIR", tempfile.gettempdir()),
                                 "gschur_clocks_rank%s.csv" % index)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


_ORACLE = {}


def _oracle_init():
    """(spawn worker) the workload's D, f and permutations, built once."""
    import lattice_inputs as li
    from oracle import dirac
    dims, U = li.workload_gauge(FIELD)
    _ORACLE["D"] = dirac.wilson_matrix(U, dims, M0)
    _ORACLE["f"] = li.gaussian_source(dims, 100).ravel()
    _ORACLE["dims"] = dims


def _oracle_solve(which):
    """(spawn worker) one complete solve of the workload by the oracle as it
    stands (outer GMRES(30) to 1e-10, inner BiCGStab to 1e-12)."""
    from oracle import permute, schur
    t, mu, inv = PERMS[which]
    D, f = _ORACLE["D"], _ORACLE["f"]
    perm, nb = permute.permutation(_ORACLE["dims"], t, mu, bool(inv))
    t0 = time.time()
    x, info = schur.schur_solve(D, perm, nb, f, tol=1e-10, m=30, inner="bicgstab", inner_tol=1e-12)
    t1 = time.time()
    res = float(np.linalg.norm(f - D @ x) / np.linalg.norm(f))
    return {"perm": PERM_NAMES[which], "start": t0, "end": t1, "seconds": t1 - t0,
            "true_residual": res, "outer_iters": info["iters"]}


def _oracle_warm(which):
    """(spawn worker) one S_bb apply of the oracle (a warm-up step)."""
    from oracle import permute, schur
    t, mu, inv = PERMS[which]
    D, f = _ORACLE["D"], _ORACLE["f"]
    perm, nb = permute.permutation(_ORACLE["dims"], t, mu, bool(inv))
    S = schur.SchurOperator(D, perm, nb, inner="bicgstab", inner_tol=1e-12)
    S(f[permute.expand_sites(perm[:nb])])
    return True


def oracle_pool(n=len(PERMS)):
    """n single-threaded oracle worker processes (spawn: safe after CUDA)."""
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                             "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        pool = mp.get_context("spawn").Pool(n, initializer=_oracle_init)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return pool


def oracle_step(pool):
    """One step of the workload by the oracle: the four solves at once, one
    process each.  Returns (wall seconds of the step, per-solve records)."""
    t0 = time.perf_counter()
    outs = pool.map(_oracle_solve, range(len(PERMS)))
    return time.perf_counter() - t0, outs


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline():
    """The oracle timed on the host's cores: one step (the four permutations'
    solves, one single-threaded process each, in parallel), plus the
    single-thread rate of the same solves."""
    pool = oracle_pool()
    try:
        wall, outs = oracle_step(pool)
    finally:
        pool.close()
        pool.join()
    per = [o["seconds"] for o in outs]
    return {"value": len(PERMS) / wall, "unit": UNIT, "cores": len(PERMS), "kind": "oracle",
            "host_cores_available": host_cores(),
            "sample": "one step of the 8^4 workload: the P_I, P_II, P_I^T, P_II^T solves by the "
                      "numpy/scipy FP64 oracle as it stands, one single-threaded process per "
                      "permutation, all four at once; %.1f s wall, max true residual %.1e"
                      % (wall, max(o["true_residual"] for o in outs)),
            "single_thread": {"value": len(PERMS) / sum(per), "unit": UNIT, "cores": 1,
                              "seconds_per_solve": {o["perm"]: o["seconds"] for o in outs}}}


def replica_totals(dist, device, times_ms, steps, world):
    """Whole-job numbers of N replicas: each rank solves the workload's
    len(PERMS) * steps problems on its own GPU (no data exchange); the job
    takes the slowest rank's time, so every elapsed time is the max over ranks
    (one all-reduce), and the throughput is all ranks' solves over it.
    Returns (max times in ms, solves per second for each)."""
    times_ms = [float(t) for t in times_ms]
    if dist is not None:
        import torch
        tt = torch.tensor(times_ms, dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        times_ms = [float(v) for v in tt]
    solves = len(PERMS) * steps * world
    return times_ms, [solves / (t / 1e3) for t in times_ms]


def run_reference(args, rank, world):
    """The CPU oracle timed as the reference arm (rank 0 only), on the same
    step as the GPU arm (the four permutations' complete solves): the K steps'
    4 K solves are spread over one single-threaded oracle process per host
    core, and the timed region is all of them; warm-up: one S_bb apply per
    permutation per warm-up step."""
    if rank != 0:
        return
    import lattice_inputs as li
    li.workload_gauge(FIELD)          # cache the field before the workers load it
    cores = max(1, min(host_cores(), len(PERMS) * args.steps))
    pool = oracle_pool(cores)
    try:
        pool.map(_oracle_warm, [k % len(PERMS) for k in range(len(PERMS) * args.warmup)], chunksize=1)
        t0 = time.perf_counter()
        outs = pool.map(_oracle_solve, [k % len(PERMS) for k in range(len(PERMS) * args.steps)],
                        chunksize=1)
        tot = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    worst = max(o["true_residual"] for o in outs)
    value = len(PERMS) * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "solves_per_step": len(PERMS)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "host_cores_available": host_cores(),
                             "sample": "the %d steps' %d solves (P_I, P_II, P_I^T, P_II^T of the 8^4 "
                                       "workload, each step) by the numpy/scipy FP64 oracle as it stands, "
                                       "spread over %d single-threaded processes, %.1f s wall; warm-up = "
                                       "one S_bb apply per permutation per warm-up step; max true "
                                       "residual %.1e" % (args.steps, len(outs), cores, tot, worst),
                             "single_thread": {"value": len(outs) / sum(o["seconds"] for o in outs),
                                               "unit": UNIT, "cores": 1}},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def kernel_case(args):
    """One kernel on a large lattice: `reps` launches timed with CUDA events."""
    dims = tuple(int(v) for v in args.dims.split(","))
    if args.case == "net_tc":
        print(json.dumps(net_case(dims, args.reps)), flush=True)
        return
    if args.case == "lp_solve":
        print(json.dumps(lp_solve_case(dims, args.prec, args.reps)), flush=True)
        return
    out = stencil_roofline(args.case, dims, args.prec, args.variant, args.reps)
    print(json.dumps(out), flush=True)


def lp_solve_case(dims, prec_name="f32", reps=3):
    """One mixed-precision inner D_rr solve (Type I rest set; FP32 or BF16
    storage; persistent low-precision BiCGStab cycles with FP64 defect
    correction, to 1e-10) on a lattice larger than L2 (exp(i 0.2 H) field, seed
    3, m0 = -0.35): the achieved algorithmic bytes/s of k_bicg_persistent_lp,
    from the library's CUDA-event profiling of its launches, against the
    measured HBM copy bandwidth (the command of its profile)."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_0704_2341_gb300 as gs
    from lattice_inputs import torchgen
    import lattice_inputs as li
    V = li.volume(dims)
    stream = torch.cuda.current_stream()
    ctx = gs.Context(dims, -0.35, stream.cuda_stream)
    ctx.set_gauge(torchgen.random_gauge_t(dims, 0.2, 3, "cuda"))
    nr = V - ctx.get_permutation(1, 0, 0, torch.empty(V, dtype=torch.int32, device="cuda"))
    gen = torch.Generator(device="cuda").manual_seed(5)
    t = torch.randn(nr * 12, dtype=torch.complex128, device="cuda", generator=gen)
    z = torch.empty_like(t)
    prec = gs.GS_F32 if prec_name == "f32" else gs.GS_BF16
    o = gs.gs_default_opts(inner_prec=prec, inner_tol=1e-10)
    ctx.solve_rr(1, 0, 0, t, z, o)      # warm-up: plans, stencil tuning, workspaces
    torch.cuda.synchronize()
    ctx.profile(True)
    iters = 0
    for _ in range(reps):
        st = ctx.solve_rr(1, 0, 0, t, z, o)
        iters += st.inner_iters
    p = ctx.profile_read(gs.GS_PROF_SOLVER_LP)
    ctx.profile(False)
    peaks = _peaks()
    ms = p.ms / p.launches
    gbs = p.bytes / p.launches / (ms / 1e3) / 1e9
    out = {"case": "lp_solve", "dims": dims, "prec": prec_name, "rest_sites": nr, "solves": reps,
           "inner_iterations_per_solve": iters / reps, "launches": p.launches,
           "us_per_launch": 1e3 * ms, "algorithmic_bytes_per_launch": p.bytes / p.launches,
           "gbs": gbs, "frac_hbm": gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
           "inner_residual": st.inner_residual}
    ctx.close()
    return out


def stencil_roofline(case, dims, prec_name="f32", variant=0, reps=20):
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_0704_2341_gb300 as gs
    import lattice_inputs as li
    V = li.volume(dims)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = gs.Context(dims, M0, stream.cuda_stream)
    # unitary links from a cheap recipe (the timing does not depend on the values)
    U = torch.from_numpy(li.random_gauge((dims[0], dims[1], dims[2], 2), 0.2, 3)).to(dev)
    U = U.reshape(dims[0] * dims[1] * dims[2], 2, 4, 3, 3)
    U = U.repeat(1, dims[3] // 2, 1, 1, 1).permute(1, 0, 2, 3, 4).reshape(V, 4, 3, 3).contiguous()
    ctx.set_gauge(U)
    x = torch.randn(V, 4, 3, dtype=torch.complex128, device=dev)
    y = torch.empty_like(x)
    if case == "wilson_f64":
        prec = gs.GS_F64
        run = lambda: ctx.wilson_apply(x, y)   # noqa: E731
    else:
        prec = gs.GS_F32 if prec_name == "f32" else gs.GS_BF16
        ctx.set_option(gs.GS_OPT_STENCIL_VARIANT, variant)
        xl = torch.empty(gs.lowp_bytes(V, prec), dtype=torch.uint8, device=dev)
        yl = torch.empty_like(xl)
        ctx.lowp_pack(0, 0, 0, prec, x, xl)
        run = lambda: ctx.wilson_apply_lowp(0, 0, 0, prec, xl, yl)   # noqa: E731
    del U
    for _ in range(3):
        run()
    ctx.profile(True)
    for _ in range(reps):
        run()
    p = ctx.profile_read(prec)
    ctx.profile(False)
    ms = p.ms / p.launches
    fp64_peak = ctx.fp64_peak()
    peaks = _peaks()
    out = {"case": case, "prec": prec_name if case != "wilson_f64" else "f64",
           "variant": ctx.get_option(gs.GS_OPT_STENCIL_VARIANT) if case != "wilson_f64" else None,
           "dims": dims, "sites": V, "launches": p.launches,
           "us_per_launch": 1e3 * ms, "sites_per_s": V / (ms / 1e3),
           "tflops": p.flops / p.launches / (ms / 1e3) / 1e12,
           "fp64_peak_measured_tflops": fp64_peak,
           "frac_fp64_peak": p.flops / p.launches / (ms / 1e3) / 1e12 / fp64_peak,
           "gbs": p.bytes / p.launches / (ms / 1e3) / 1e9,
           "frac_hbm": (p.bytes / p.launches / (ms / 1e3) / 1e9 / peaks["hbm_gbs"])
           if peaks.get("hbm_gbs") else None,
           "algorithmic_bytes_per_launch": p.bytes / p.launches}
    ctx.close()
    del x, y
    torch.cuda.empty_cache()
    return out


def _rest_count(gs, torch, ctx, ptype, mu, inv):
    perm = torch.empty(ctx.volume, dtype=torch.int32, device="cuda")
    return ctx.volume - ctx.get_permutation(ptype, mu, inv, perm)


def train_learned(torch, gs, li, kind, m0, perms, stream, n_pairs=2000, seed=0):
    """A 24-channel network trained on n_pairs pairs (t = D_rr z, z Gaussian)
    spread over the 8 seeded 8^4 training fields of `kind` and the given
    permutations: 400 Adam steps at lr 1e-3, 200 at 2e-4, batch 4."""
    from paper_0704_2341_gb300 import learned
    t0 = time.time()
    li.prepare_training_gauges(kind, 8)
    data, ctxs = [], []
    per_field = n_pairs // 8
    for i in range(8):
        dims, U = li.training_gauge(kind, i)
        c = gs.Context(dims, m0, stream.cuda_stream)
        c.set_gauge(torch.from_numpy(U).to("cuda"))
        ctxs.append(c)
        for k, (pt, mu, inv) in enumerate(perms):
            n = per_field // len(perms) + (1 if k < per_field % len(perms) else 0)
            nr = _rest_count(gs, torch, c, pt, mu, inv)
            Z = li.gaussian_source(dims, 1000 + 10 * i + k, n_src=n).reshape(n, -1, 12)[:, :nr]
            T, Zd = learned.make_pairs_apply(torch, c, pt, mu, inv, Z)
            data.append((c, pt, mu, inv, T, Zd))
    net = gs.Net(24)
    for layer, w in enumerate(learned.identity_like_weights(24, m0, 4 + seed)):
        net.set_weights(layer, w)
    hist = learned.train(torch, net, data, steps=400, batch=4, lr=1e-3, seed=7 + seed)
    hist += learned.train(torch, net, data, steps=200, batch=4, lr=2e-4, seed=8 + seed)
    torch.cuda.synchronize()
    info = {"fields": "8 seeded 8^4 %s fields" % ("beta=5.4 heatbath" if kind == "heatbath"
                                                  else "exp(i 0.2 H) + 10 APE"),
            "pairs": sum(d[4].shape[0] for d in data), "adam_steps": len(hist), "batch": 4,
            "loss_first": float(sum(hist[:5]) / 5), "loss_last50": float(sum(hist[-50:]) / 50),
            "seconds": time.time() - t0}
    del data
    for c in ctxs:
        c.close()
    torch.cuda.empty_cache()
    return net, info


def learned_headline(args, torch, gs, li, ctxs, probs, stream, plain_value, plain_seq_value):
    """The headline workload with the inner D_rr solve as FGMRES(64) + the
    trained network inside FP32 defect correction (same 1e-10 outer target):
    the four permutations' solves at once, as the plain FP64 step runs them
    (schur_solve_batched; each permutation's context holds its own copy of the
    trained network), and one after another on one context."""
    from paper_0704_2341_gb300 import learned
    net, info = train_learned(torch, gs, li, "heatbath", M0, PERMS, stream)
    nets = [net]
    for _ in range(len(ctxs) - 1):
        copy = gs.Net(24)
        for layer in range(3):
            copy.set_weights(layer, net.get(0, layer))
        nets.append(copy)
    o = learned.fgmres_net_opts(inner_restart=64, lowp_tol=1e-2)
    for c, n in zip(ctxs, nets):
        c.set_net(n)
    for _ in range(2):
        status, _ = gs.schur_solve_batched(probs, o)
        if status != gs.GS_OK:
            raise gs.GschurError(status, "learned schur_solve_batched: " + gs.gs_last_error(ctxs[0].handle))
    torch.cuda.synchronize()
    worst, inner = 0.0, 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        status, sts = gs.schur_solve_batched(probs, o)
        if status != gs.GS_OK:
            raise gs.GschurError(status, "learned schur_solve_batched: " + gs.gs_last_error(ctxs[0].handle))
        worst = max([worst] + [st.true_residual for st in sts])
        inner += sum(st.inner_iters for st in sts)
    torch.cuda.synchronize()
    conc_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    value = len(PERMS) / (conc_ms / 1e3)
    # one after another on the first context
    ctx, f, x = ctxs[0], probs[0]["f"], probs[0]["x"]
    lms, seq_worst = 0.0, 0.0
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for (t, mu, inv) in PERMS:
            st = ctx.schur_solve(t, mu, inv, f, x, o)
            seq_worst = max(seq_worst, st.true_residual)
        b.record(stream)
        b.synchronize()
        lms += a.elapsed_time(b)
    for c in ctxs:
        c.set_net(None)
    for n in nets:
        n.close()
    seq_value = len(PERMS) * args.steps / (lms / 1e3)
    return {"value": value, "unit": UNIT, "ms_per_step": conc_ms,
            "max_true_residual": worst, "speedup_vs_plain_f64": value / plain_value,
            "form": "the four permutations' solves at once (schur_solve_batched), wall clock around each "
                    "synchronous call",
            "inner_fgmres_steps_per_step": inner / args.steps,
            "one_after_another": {"value": seq_value, "unit": UNIT, "ms_per_step": lms / args.steps,
                                  "max_true_residual": seq_worst,
                                  "speedup_vs_plain_f64_one_after_another": seq_value / plain_seq_value},
            "inner": "FGMRES(64) with the network as right preconditioner, FP32 defect "
                     "correction (per-cycle tolerance 1e-2), tensor-core 24->24 layer",
            "training": info}


def learned_large(torch, gs, li):
    """One source of the 32^3 x 64 learned-preconditioner workload: the inner
    solve D_rr z = t (Type I rest set) to 1e-10 with FGMRES(64) + the network
    trained on 8^4 fields of the same recipe, against the plain FP64 BiCGStab
    on the same system (bounded at 3000 iterations)."""
    from lattice_inputs import torchgen
    from paper_0704_2341_gb300 import learned
    stream = torch.cuda.current_stream()
    m0 = -0.38
    net, info = train_learned(torch, gs, li, "ape", m0, [(1, 0, 0)], stream, seed=1)
    t0 = time.time()
    dims, U = torchgen.workload_gauge_t("32^3x64 eps0.2 ape10", "cuda")
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    ctx = gs.Context(dims, m0, stream.cuda_stream)
    ctx.set_gauge(U)
    del U
    torch.cuda.empty_cache()
    nr = _rest_count(gs, torch, ctx, 1, 0, 0)
    t = torch.from_numpy(li.gaussian_source(dims, 901).reshape(-1, 12)[:nr].copy()).to("cuda")
    z = torch.empty_like(t)
    ctx.set_net(net)
    for _ in range(3):
        net.apply(ctx.handle, 1, 0, 0, t, z)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(5):
        net.apply(ctx.handle, 1, 0, 0, t, z)
    b.record(stream)
    b.synchronize()
    apply_ms = a.elapsed_time(b) / 5
    out = {"workload": "32^3x64, exp(i 0.2 H) seed 5 + 10 APE steps (alpha 0.5), Wilson m0=-0.38, "
                       "Type I; source: complex Gaussian (seed 901) on the rest set",
           "sample": "1 of the 12 sources, the inner D_rr solve alone (the complete S_bb solve at this "
                     "size does not finish in a bench run)",
           "rest_sites": nr, "field_generation_s": gen_s, "net_apply_ms": apply_ms, "training": info}
    runs = (("fgmres_net", learned.fgmres_net_opts(inner_tol=1e-10, inner_restart=64, lowp_tol=1e-2)),
            ("plain_f64_bicgstab", gs.gs_default_opts(inner_tol=1e-10, inner_max_iter=3000)))
    for name, o in runs:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = ctx.solve_rr(1, 0, 0, t, z, o, allow=(gs.GS_OK, gs.GS_MAXITER, gs.GS_BREAKDOWN))
        b.record(stream)
        b.synchronize()
        out[name] = {"status": gs.STATUS_NAMES.get(st.status, st.status), "steps": st.inner_iters,
                     "true_residual": st.true_residual, "ms": a.elapsed_time(b)}
        if name == "fgmres_net":
            ctx.set_net(None)
    net.close()
    ctx.close()
    torch.cuda.empty_cache()
    return out


def batched_section(torch, gs, li, reps=1):
    """The batched workload: 12 spin-colour point sources on 24^3 x 48
    (exp(i 0.2 H) seed 3, m0 = -0.35) plus 4 Gaussian sources on each of
    8^4 (seed 6) and 16^4 (seed 4), Type I, FP32 inner / FP64 outer, all in
    one schur_solve_batched call (the 20 solves largest lattice first on four
    concurrent lanes, each persistent kernel sized for its share of the GPU
    at launch); against the same 20 solves one at a time on one stream.
    Warm-up: one batched call to a loose tolerance (plans, stencil tuning,
    lane contexts, workspaces)."""
    from lattice_inputs import torchgen
    specs = [("24^3x48 eps0.2", "point", 12), ("8^4 eps0.2", "gauss", 4), ("16^4 eps0.2", "gauss", 4)]
    m0 = -0.35
    ctxs, probs, streams = [], [], []
    for name, kind, n in specs:
        dims, U = torchgen.workload_gauge_t(name, "cuda")
        s = torch.cuda.Stream()
        c = gs.Context(dims, m0, s.cuda_stream)
        c.set_gauge(U)
        del U
        src = li.point_sources(dims) if kind == "point" else li.gaussian_source(dims, 300, n_src=n)
        f = torch.from_numpy(np.ascontiguousarray(src)).to("cuda")
        probs.append(dict(ctx=c.handle, type=1, dir=0, inverse=0, nrhs=n, f=f, x=torch.zeros_like(f)))
        ctxs.append(c)
        streams.append(s)
    o = gs.gs_default_opts(inner_prec=gs.GS_F32)
    warm = gs.gs_default_opts(inner_prec=gs.GS_F32)
    warm.tol = 1e-3
    torch.cuda.synchronize()
    gs.schur_solve_batched(probs, warm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    worst, status = 0.0, gs.GS_OK
    for _ in range(reps):
        for pr in probs:
            pr["x"].zero_()
        torch.cuda.synchronize()
        status, stats = gs.schur_solve_batched(probs, o)
        worst = max([worst] + [st.true_residual for st in stats])
    torch.cuda.synchronize()
    batched_s = (time.perf_counter() - t0) / reps
    # the same solves one source at a time, each lattice's total
    seq_worst, per_lattice = 0.0, {}
    for (name, _, _), c, pr in zip(specs, ctxs, probs):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for j in range(pr["nrhs"]):
            st = gs.schur_solve(c.handle, 1, 0, 0, pr["f"][j], pr["x"][j], o)
            seq_worst = max(seq_worst, st.true_residual)
        torch.cuda.synchronize()
        per_lattice[name] = round(time.perf_counter() - t1, 3)
    seq_s = sum(per_lattice.values())
    nsol = sum(pr["nrhs"] for pr in probs)
    lanes = ctxs[0].get_option(gs.GS_OPT_BATCH_LANES) or 4
    for c in ctxs:
        c.close()
    del probs
    torch.cuda.empty_cache()
    return {"workload": "12 point sources on 24^3x48 (exp(i 0.2 H) seed 3) + 4 Gaussian sources on each of "
                        "8^4 (seed 6) and 16^4 (seed 4), Wilson m0=-0.35, Type I, outer GMRES(30) to 1e-10, "
                        "FP32 inner / FP64 outer",
            "status": gs.STATUS_NAMES.get(status, status), "solves": nsol, "lanes": lanes,
            "batched_s": batched_s, "value": nsol / batched_s, "unit": "solves/s",
            "max_true_residual": worst, "one_at_a_time_s": seq_s,
            "one_at_a_time_s_per_lattice": per_lattice,
            "one_at_a_time_max_true_residual": seq_worst, "speedup": seq_s / batched_s,
            "timing": "wall clock around the call (host threads per lane), %d repetition(s)" % reps}


def reusken_section(torch, gs, li, reps=20):
    """The Section 3 approximation on the 8^4 workload (m0 = -0.4, the four
    permutations): time of one S~_bb apply (no inner solve) against one exact
    S_bb apply (inner BiCGStab to 1e-12), CUDA events, and the distance
    ||S~ x - S x|| / ||S x|| on a Gaussian x_b."""
    dims, U = li.workload_gauge(FIELD)
    stream = torch.cuda.current_stream()
    ctx = gs.Context(dims, M0, stream.cuda_stream)
    ctx.set_gauge(torch.from_numpy(U).to("cuda"))
    out = {"workload": WORKLOAD.split(", FP64")[0] + ", one Gaussian x_b per permutation", "permutations": {}}
    opts = gs.gs_default_opts()
    for (t, mu, inv) in PERMS:
        perm = torch.empty(ctx.volume, dtype=torch.int32, device="cuda")
        nb = ctx.get_permutation(t, mu, inv, perm)
        rng = np.random.default_rng(5)
        xb = torch.from_numpy(rng.standard_normal(nb * 12) + 1j * rng.standard_normal(nb * 12)).to("cuda")
        ya, ys = torch.empty_like(xb), torch.empty_like(xb)
        ctx.schur_apply_reusken(t, mu, inv, xb, ya)
        ctx.schur_apply(t, mu, inv, xb, ys, opts)
        times = {}
        for name, call in (("reusken", lambda: ctx.schur_apply_reusken(t, mu, inv, xb, ya)),
                           ("exact", lambda: ctx.schur_apply(t, mu, inv, xb, ys, opts))):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                call()
            b.record(stream)
            b.synchronize()
            times[name] = a.elapsed_time(b) / reps
        key = ("P_%s%s" % ("I" if t == 1 else "II", "^T" if inv else ""))
        out["permutations"][key] = {
            "reusken_apply_ms": times["reusken"], "exact_apply_ms": times["exact"],
            "speedup": times["exact"] / times["reusken"],
            "rel_distance": float(torch.linalg.norm(ya - ys) / torch.linalg.norm(ys))}
    ctx.close()
    return out


def table1_section(torch, gs, li):
    """Table 1 of the paper on the GPU (Section 4): D x = f to 1e-8 at kappa =
    1/6 (m0 = -1) on the 8^4 stand-in field of each coupling, Gaussian source
    (seed 100), BiCGStab plain and right-preconditioned by the 3-level
    V-cycle on the Section 3 approximation (P_I^T at both steps for beta =
    5.4 and 5.7, P_II^T along x0 then x1 for 5.9; rest-set solves by BiCGStab
    to 1e-2; coarsest level inverted exactly).  Times by CUDA events; the
    V-cycle's set-up (probing the coarse operators, the coarsest inverse) is
    reported apart.  Also the table's second row on the GPU: the condition
    number of D and its eigenvalue of smallest real part."""
    li.prepare_gauges([("coupling", b, 0) for b in TABLE1_LEVELS])
    stream = torch.cuda.current_stream()
    out = {"workload": "8^4 plaquette-action stand-in fields (beta 5.4 / 5.7 / 5.9, 200 Cabibbo-Marinari "
                       "sweeps, cold start, seeds 21 / 51 / 71), Wilson kappa = 1/6 (m0 = -1), Gaussian "
                       "source, D x = f to 1e-8", "columns": {}}
    for beta, levels in TABLE1_LEVELS.items():
        dims, U = li.coupling_gauge(beta, 0)
        ctx = gs.Context(dims, -1.0, stream.cuda_stream)
        ctx.set_gauge(torch.from_numpy(U).to("cuda"))
        f = torch.from_numpy(li.gaussian_source(dims, 100)).to("cuda")
        x = torch.empty_like(f)
        col = {"paper": dict(zip(("condition", "R_plain", "R_preconditioned"), TABLE1_PAPER[beta])),
               "levels": [list(l) for l in levels]}
        # Table 1's second row: the 2-norm condition number of D (Lanczos on
        # D^H D to 1e-6), and the eigenvalue of D with the smallest real part
        # (800 Arnoldi steps); start vector: Gaussian, seed 14
        start = torch.from_numpy(li.gaussian_source(dims, 14)).to("cuda")
        t0 = time.perf_counter()
        kappa, smin, smax, lsteps = ctx.condition_number(start, max_steps=20000, tol=1e-6,
                                                         allow=(gs.GS_OK, gs.GS_MAXITER))
        cond_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        ev = ctx.leftmost_eigenvalues(start, m=800, k=2)
        col["condition"] = {"kappa": kappa, "sigma_min": smin, "sigma_max": smax, "lanczos_steps": lsteps,
                            "seconds": cond_s}
        col["leftmost_eigenvalue"] = {"re": ev[0].real, "im": abs(ev[0].imag), "arnoldi_steps": 800,
                                      "seconds": time.perf_counter() - t0}
        del start
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st, R, hist = ctx.solve_bicgstab(None, f, x, tol=1e-8, max_iter=3000,
                                         allow=(gs.GS_OK, gs.GS_MAXITER, gs.GS_BREAKDOWN))
        b.record(stream)
        b.synchronize()
        col["plain"] = {"status": gs.STATUS_NAMES.get(st.status, st.status), "steps": st.outer_iters,
                        "R": R, "true_residual": st.true_residual, "ms": a.elapsed_time(b)}
        t0 = time.perf_counter()
        vc = gs.VCycle(ctx, levels, order=2, rest_tol=1e-2)
        setup_s = time.perf_counter() - t0
        a.record(stream)
        st, R, hist = ctx.solve_bicgstab(vc, f, x, tol=1e-8, max_iter=300,
                                         allow=(gs.GS_OK, gs.GS_MAXITER, gs.GS_BREAKDOWN))
        b.record(stream)
        b.synchronize()
        col["preconditioned"] = {"status": gs.STATUS_NAMES.get(st.status, st.status),
                                 "steps": st.outer_iters, "R": R, "true_residual": st.true_residual,
                                 "ms": a.elapsed_time(b), "setup_s": setup_s,
                                 "rest_solves": st.inner_solves, "rest_steps": st.inner_iters,
                                 "rest_solves_at_limit": st.lowp_fallbacks,
                                 "levels_sites": [vc.level(l)["sites"] for l in range(vc.nlevels)],
                                 "probe_colours": [vc.level(l)["colours"] for l in range(vc.nlevels - 1)]}
        vc.close()
        ctx.close()
        out["columns"]["%.1f" % beta] = col
    return out


def mixed_large_section(torch, gs, li):
    """The 16^3 x 32 mixed-precision workload: exp(i 0.25 H) + 5 APE steps
    (alpha 0.5, seed 2; made on the GPU), Wilson m0 = -0.3, Type II along x0,
    one Gaussian source (seed 100), outer GMRES(30) to 1e-10: the complete
    schur_solve with the plain FP64 inner solve against the FP32 and BF16
    inner solves (FP64 defect correction), each after one untimed solve."""
    from lattice_inputs import torchgen
    stream = torch.cuda.current_stream()
    dims, U = torchgen.workload_gauge_t("16^3x32 eps0.25 ape5", "cuda")
    ctx = gs.Context(dims, -0.3, stream.cuda_stream)
    ctx.set_gauge(U)
    del U
    f = torch.from_numpy(li.gaussian_source(dims, 100)).to("cuda")
    x = torch.empty_like(f)
    out = {"workload": "16^3x32, exp(i 0.25 H) seed 2 + 5 APE steps (alpha 0.5), Wilson m0=-0.3, Type II "
                       "along x0, one Gaussian source (seed 100), outer GMRES(30) to 1e-10, back-substitution",
           "inner": {}}
    for name, prec in (("f64", gs.GS_F64), ("f32", gs.GS_F32), ("bf16", gs.GS_BF16)):
        o = gs.gs_default_opts(inner_prec=prec)
        ctx.schur_solve(2, 0, 0, f, x, o)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = ctx.schur_solve(2, 0, 0, f, x, o)
        b.record(stream)
        b.synchronize()
        out["inner"][name] = {"ms": a.elapsed_time(b), "true_residual": st.true_residual,
                              "outer_iters": st.outer_iters, "inner_iters": st.inner_iters,
                              "lowp_cycles": st.lowp_cycles}
    for name in ("f32", "bf16"):
        out["inner"][name]["speedup_vs_f64"] = out["inner"]["f64"]["ms"] / out["inner"][name]["ms"]
    ctx.close()
    torch.cuda.empty_cache()
    return out


def net_case(dims, reps=5):
    """The learned preconditioner's network (24 channels, identity-like
    weights, tensor-core kernels) applied `reps` times on one lattice: the
    command the network's ncu profiles are taken with."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_0704_2341_gb300 as gs
    from paper_0704_2341_gb300 import learned
    import lattice_inputs as li
    from lattice_inputs import torchgen
    V = li.volume(dims)
    stream = torch.cuda.current_stream()
    ctx = gs.Context(dims, -0.38, stream.cuda_stream)
    ctx.set_gauge(torchgen.random_gauge_t(dims, 0.2, 5, "cuda"))
    net = gs.Net(24)
    for layer, w in enumerate(learned.identity_like_weights(24, -0.38, 4)):
        net.set_weights(layer, w)
    nr = V - ctx.get_permutation(1, 0, 0, torch.empty(V, dtype=torch.int32, device="cuda"))
    t = torch.randn(nr, 12, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(t)
    net.apply(ctx.handle, 1, 0, 0, t, y)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        net.apply(ctx.handle, 1, 0, 0, t, y)
    b.record(stream)
    b.synchronize()
    out = {"case": "net_tc", "dims": dims, "rest_sites": nr, "apply_ms": a.elapsed_time(b) / reps}
    net.close()
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-lowp-dslash", action="store_true",
                    help="skip the 32^3x64 low-precision stencil roofline")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-preconditioner sections")
    ap.add_argument("--no-table1", action="store_true",
                    help="skip Table 1 on the GPU (plain / V-cycle BiCGStab on three 8^4 fields)")
    ap.add_argument("--no-mixed-large", action="store_true",
                    help="skip the 16^3x32 Type II mixed-precision solve")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched multi-lattice multi-source section (about 2.5 minutes)")
    ap.add_argument("--only", default=None,
                    choices=["batched", "learned_large", "reusken", "table1", "mixed_large"],
                    help="run one section alone and print it")
    ap.add_argument("--case", default=None, choices=["wilson_f64", "wilson_lp", "net_tc", "lp_solve"],
                    help="kernel micro-benchmark instead of the solve (for profiling)")
    ap.add_argument("--prec", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--variant", type=int, default=0, choices=[0, 1, 2, 3, 4, 5, 6],
                    help="low-precision stencil variant (0 = autotuned)")
    ap.add_argument("--dims", default="24,24,24,48")
    ap.add_argument("--reps", type=int, default=20)
    args = ap.parse_args()
    if args.case:
        kernel_case(args)
        return
    if args.only is not None:
        import torch
        import __graft_entry__ as g
        g.build()
        import paper_0704_2341_gb300 as gs
        import lattice_inputs as li
        out = {"batched": batched_section, "learned_large": learned_large,
               "reusken": reusken_section, "table1": table1_section,
               "mixed_large": mixed_large_section}[args.only](torch, gs, li)
        print(json.dumps(out), flush=True)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.warmup < 3:
        args.warmup = 3

    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_0704_2341_gb300 as gs
    import lattice_inputs as li

    # every seeded field the run needs, generated (in parallel, spawn workers)
    # before the first GPU call if the cache lacks it
    specs = [("workload", FIELD, None)]
    if not args.no_learned:
        specs += [("training", kind, i) for kind in ("heatbath", "ape") for i in range(8)]
    if not args.no_table1:
        specs += [("coupling", b, 0) for b in TABLE1_LEVELS]
    if local == 0:
        li.prepare_gauges(specs)

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    dims, U = li.workload_gauge(FIELD)
    f_np = li.gaussian_source(dims, 100)
    stream = torch.cuda.current_stream(dev)
    Ud = torch.from_numpy(U).to(dev)
    # one context and stream per permutation: a step solves the four systems
    # at once (schur_solve_batched; each solve's persistent kernels granted
    # one tile round by the call's block ledger)
    pstreams = [torch.cuda.Stream(device=dev) for _ in PERMS]
    ctxs = []
    for ps in pstreams:
        c = gs.Context(dims, M0, ps.cuda_stream)
        c.set_gauge(Ud)
        ctxs.append(c)
    ctx = ctxs[0]
    f = torch.from_numpy(f_np).to(dev)
    xs = [torch.empty_like(f) for _ in PERMS]
    x = xs[0]
    probs = [dict(ctx=c.handle, type=t, dir=mu, inverse=inv, nrhs=1, f=f, x=xx)
             for c, (t, mu, inv), xx in zip(ctxs, PERMS, xs)]
    opts = gs.gs_default_opts()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def step(o=opts):
        status, sts = gs.schur_solve_batched(probs, o)
        if status != gs.GS_OK:
            raise gs.GschurError(status, "schur_solve_batched: " + gs.gs_last_error(ctxs[0].handle))
        return sum(st.kernel_launches for st in sts), max(st.true_residual for st in sts)

    def bracket(fn):
        """Device time of fn() between two events on the main stream, with
        the permutation streams ordered after the first and the second after
        them."""
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for ps in pstreams:
            ps.wait_event(a)
        out = fn()
        for ps in pstreams:
            e = torch.cuda.Event()
            e.record(ps)
            stream.wait_event(e)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b), out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(K, profile=False, o=opts):
        if profile:
            for c in ctxs:
                c.profile(True)
        ms, launches, worst = 0.0, 0, 0.0
        barrier()
        for k in range(K):
            flush.zero_()
            t, (n, w) = bracket(lambda: step(o))
            ms += t
            launches += n
            worst = max(worst, w)
        barrier()
        prof = None
        if profile:
            prof = {}
            for fam in (gs.GS_PROF_STENCIL_F64, gs.GS_PROF_SOLVER_F64):
                reads = [c.profile_read(fam) for c in ctxs]
                iv = sorted(iv for c in ctxs for iv in c.profile_timeline(fam))
                union, cur = 0.0, None
                for a0, a1 in iv:            # length of the union of the launch intervals
                    if cur is None or a0 > cur[1]:
                        if cur is not None:
                            union += cur[1] - cur[0]
                        cur = [a0, a1]
                    else:
                        cur[1] = max(cur[1], a1)
                if cur is not None:
                    union += cur[1] - cur[0]
                prof[fam] = {"launches": sum(r.launches for r in reads),
                             "ms": sum(r.ms for r in reads), "union_ms": union,
                             "flops": sum(r.flops for r in reads), "bytes": sum(r.bytes for r in reads)}
            for c in ctxs:
                c.profile(False)
        return ms, launches, worst, prof

    smi_index = (os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local]
                 if os.environ.get("CUDA_VISIBLE_DEVICES") else str(local))
    clocks = ClockSampler(smi_index)
    clocks.start()
    ms, launches, worst, _ = timed(args.steps)
    clock_info = clocks.stop()
    # the same K steps again with the kernel launches bracketed by events
    ms_prof, _, _, prof = timed(args.steps, profile=True)

    fp64_peak = ctx.fp64_peak()

    # end to end: pinned host source in, four solutions out, every step
    f_host = torch.from_numpy(f_np).pin_memory()
    x_host = [torch.empty_like(f_host).pin_memory() for _ in PERMS]
    e2e_ms = 0.0
    barrier()
    for _ in range(args.steps):
        flush.zero_()

        def e2e_step():
            f.copy_(f_host, non_blocking=True)
            stream.synchronize()
            step()
            for k in range(len(PERMS)):
                x_host[k].copy_(xs[k], non_blocking=True)
        t, _ = bracket(e2e_step)
        e2e_ms += t
    barrier()

    # the four solves one after another on one context (no concurrency)
    seq_ms, seq_worst = 0.0, 0.0
    barrier()
    for _ in range(args.steps):
        flush.zero_()

        def seq_step():
            w = 0.0
            for (t, mu, inv) in PERMS:
                w = max(w, ctx.schur_solve(t, mu, inv, f, x, opts).true_residual)
            return w
        t, w = bracket(seq_step)
        seq_ms += t
        seq_worst = max(seq_worst, w)
    sequential = {"value": len(PERMS) * args.steps / (seq_ms / 1e3), "unit": UNIT,
                  "ms_per_step": seq_ms / args.steps, "max_true_residual": seq_worst,
                  "form": "the same four solves one after another on one context and stream"}

    # the same workload with the mixed-precision inner solve (same tolerances,
    # four at once)
    mixed = {}
    for name, prec in (("f32", gs.GS_F32), ("bf16", gs.GS_BF16)):
        o = gs.gs_default_opts(inner_prec=prec)
        for _ in range(2):
            step(o)
        mms, _, mworst, _ = timed(args.steps, o=o)
        mixed[name] = {"value": len(PERMS) * args.steps / (mms / 1e3), "unit": UNIT,
                       "ms_per_step": mms / args.steps, "max_true_residual": mworst}
    (ms, e2e_ms), (value, e2e_value) = replica_totals(dist, dev, (ms, e2e_ms), args.steps, world)
    if rank != 0:
        for c in ctxs:
            c.close()
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks = _peaks()
    fam_names = {gs.GS_PROF_STENCIL_F64: "k_dslash_f64 (Wilson stencil on label ranges, FP64)",
                 gs.GS_PROF_SOLVER_F64: "k_bicg_persistent_f64 (whole inner BiCGStab solve in one "
                                         "cooperative launch: two D_rr stencils + vector updates per "
                                         "iteration, FP64)"}
    dom = max(prof, key=lambda fam: prof[fam]["union_ms"])

    def fam_view(p):
        n = max(p["launches"], 1)
        avg_ms = p["ms"] / n
        ach = p["flops"] / (p["union_ms"] / 1e3) / 1e12 if p["union_ms"] > 0 else 0.0
        return avg_ms, p["flops"] / n, p["bytes"] / n, ach

    avg_ms, flops_per_launch, bytes_per_launch, achieved = fam_view(prof[dom])
    concurrency = prof[dom]["ms"] / prof[dom]["union_ms"] if prof[dom]["union_ms"] > 0 else 1.0
    traffic = _ncu_traffic_per_launch(dom)
    roofline = {
        "kernel": fam_names[dom],
        "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
        "frac": achieved / fp64_peak, "traffic": traffic,
        "peak_source": "FP64 ALU, measured in this run by gs_fp64_peak (8 independent FMA chains per "
                       "thread, 8 x 256 threads per SM, CUDA events; MEASURED_PEAKS.json has no FP64 "
                       "entry); nominal 152 SMs x 2.07 GHz x 4 flop/clk = %.3f TFLOP/s"
                       % FP64_NOMINAL_TFLOPS,
        "achieved_definition": "algorithmic flops of all the family's launches in the timed steps / the "
                               "union of their CUDA-event intervals (the four permutations' solver "
                               "launches run concurrently, %.2f at a time on average)" % concurrency,
        "launches": prof[dom]["launches"], "avg_launch_us": 1e3 * avg_ms,
        "per_launch_achieved_tflops": flops_per_launch / (avg_ms / 1e3) / 1e12 if avg_ms > 0 else 0.0,
        "algorithmic_flops_per_launch": flops_per_launch,
        "algorithmic_bytes_per_launch": bytes_per_launch,
        "hbm_view": {"achieved_gbs": prof[dom]["bytes"] / (prof[dom]["union_ms"] / 1e3) / 1e9,
                     "peak_gbs": peaks.get("hbm_gbs"),
                     "frac_of_measured": (prof[dom]["bytes"] / (prof[dom]["union_ms"] / 1e3) / 1e9 /
                                          peaks["hbm_gbs"]) if peaks.get("hbm_gbs") else None},
        "share_of_step": prof[dom]["union_ms"] / ms_prof if ms_prof > 0 else None,
        "step_ms_with_events": ms_prof / args.steps,
        "other_kernels": {},
    }
    for fam in prof:
        if fam == dom or prof[fam]["launches"] == 0:
            continue
        o_ms, o_fl, o_by, o_ach = fam_view(prof[fam])
        roofline["other_kernels"][fam_names[fam]] = {
            "launches": prof[fam]["launches"], "avg_launch_us": 1e3 * o_ms,
            "achieved_tflops": o_ach, "frac_fp64_alu": o_ach / fp64_peak,
            "share_of_step": prof[fam]["union_ms"] / ms_prof if ms_prof > 0 else None}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "solves_per_step": len(PERMS),
                   "form": "plain FP64; the four permutations' solves at once (schur_solve_batched: one "
                           "context and stream per permutation, each solve's persistent kernels granted "
                           "one round of 32-site tiles, 120 or 64 of the 456 co-resident blocks, by the "
                           "call's block ledger)",
                   "l2": "flushed between steps (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "max_true_residual": worst},
        "roofline": roofline,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": f_host.numel() * f_host.element_size(),
                "d2h_bytes_per_step": sum(t.numel() * t.element_size() for t in x_host)},
        "clocks": clock_info,
        "plain_f64_sequential": sequential,
    }
    for name in mixed:
        mixed[name]["speedup_vs_plain_f64"] = mixed[name]["value"] / value
    line["mixed_inner"] = mixed
    if not args.no_learned:
        line["learned_mixed"] = learned_headline(args, torch, gs, li, ctxs, probs, pstreams[0], value,
                                                 sequential["value"])
    if not args.no_mixed_large:
        line["mixed_16x16x16x32"] = mixed_large_section(torch, gs, li)
    if not args.no_table1:
        line["table1_gpu"] = table1_section(torch, gs, li)
    for c in ctxs:
        c.close()
    ctx = None
    del Ud
    torch.cuda.empty_cache()
    if not args.no_lowp_dslash:
        lowp = {}
        for pn in ("f32", "bf16"):
            r = stencil_roofline("wilson_lp", (32, 32, 32, 64), pn, 0, 20)
            lowp[pn] = {"gbs": r["gbs"], "frac_of_measured_hbm": r["frac_hbm"],
                        "us_per_launch": r["us_per_launch"], "variant": r["variant"],
                        "algorithmic_bytes_per_launch": r["algorithmic_bytes_per_launch"]}
        line["dslash_lowp_32x32x32x64"] = lowp
    if not args.no_batched:
        torch.cuda.empty_cache()
        line["batched"] = batched_section(torch, gs, li)
    if not args.no_learned:
        torch.cuda.empty_cache()
        line["learned_32x32x32x64"] = learned_large(torch, gs, li)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
