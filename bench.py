#!/usr/bin/env python
"""Throughput of the Cholesky J/K engine on one B300 (or N replicas).

One step = one full J/K build (panels, J metric dot, J back-contraction,
K rank update, final FP64 reduction) for the multi-state workload:
nbf = 400, naux = 2400, eight densities of width 40 (one symmetric ground
density, seven non-symmetric transition densities), seeded synthetic inputs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision split|fp64]
                  [--impl ours|reference]

Prints ONE JSON line on rank 0.  `value` is algorithmic TFLOP/s (FP64-
equivalent work, slice products of the split path are cost, not counted) with
all inputs resident in HBM; `e2e` is the same metric through the public API
with pinned host inputs copied in and J/K copied out inside the timed region.
Under torchrun every rank runs its own replica (the path has no exchange
step); value = all ranks' work / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Cholesky J/K TFLOP/s (% tensor peak), split-prec vs FP64 GPU at ≤1e-10 error"
WORKLOAD = "multi-state nbf=400 naux=2400 tau=400, 8 densities k=40 (1 symmetric ground + 7 non-symmetric transition), FP64 in/out"

# FP64 issue-rate peak of B300 for the plain engine's roofline: a dependent-
# free FP64 FMA stream measured 1.20 TFLOP/s on this machine's B300 (148 SMs at
# 2032 MHz, i.e. 2 FP64 FMA per clock per SM; nominal 1.25 TFLOP/s).
FP64_PEAK_TFLOPS = 1.20


def build_flops(n, naux, ks, sym):
    """Algorithmic flops of one build: panels 2n^2kA per half-transform, rank
    update 2n^2kA (n^2kA for a symmetric density), J back-contraction 2n^2A,
    gamma from the panel 2nkA, per density."""
    f = 0.0
    for k, s in zip(ks, sym):
        f += (3.0 if s else 6.0) * n * n * k * naux
        f += 2.0 * n * n * naux + 2.0 * n * k * naux
    return f


# DRAM bytes of the sliced GEMM measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) on the profile case (nbf=400, naux=600, 8 densities
# k=40; summary in profiles/ozgemm_tcgen05_profile_case.md) in the tuned
# configuration (one aux chunk, grouped schedule: one panel launch and one
# rank-update launch per build): the panel launch moved 2.268 GB and the
# grouped rank-update launch 2.040 GB for 600 aux indices.  Both grow in
# proportion to naux, which is how they are scaled to the full multi-state
# launches.
OZ_PANEL_BYTES_PER_P = 2.268e9 / 600
OZ_RANK_BYTES_PER_P = 2.040e9 / 600


def panel_rank_flops(n, naux, ks, sym):
    return sum((3.0 if s else 6.0) * n * n * k * naux for k, s in zip(ks, sym))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = max((num(r[2]) for r in rows if num(r[2]) is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) for r in rows if num(r[3]) is not None), default=None)}


def dist_init():
    """Replicas: one process per GPU (RANK / WORLD_SIZE / MASTER_* from the
    launcher).  NCCL between GPUs; gloo where no GPU is visible (CPU tests of
    the multi-process logic)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    """The slowest rank's time: the whole job finishes when it does."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    if dist.get_backend() == "gloo":
        device = "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_tflops(flops_per_rank, ms_max, world):
    """Whole-job throughput of `world` replicas that each did flops_per_rank
    in at most ms_max milliseconds (weak scaling)."""
    return world * flops_per_rank / (ms_max * 1e-3) / 1e12


_CPU_SAMPLE = {}


def cpu_baseline_sample(L=None):
    """The oracle as it stands on a bounded sample of the workload: three of
    the seven non-symmetric densities (k=40) over all 2400 aux indices."""
    import oracle
    from paper_2608_06536_b300 import inputs
    n, tau, na, nds = 400, 400.0, 2400, 3
    if "L" not in _CPU_SAMPLE:
        _CPU_SAMPLE["L"] = L if L is not None else inputs.factor(n, na, tau, 0)
        _CPU_SAMPLE["XY"] = [inputs.transition_density(n, 40, s, 0) for s in range(1, 1 + nds)]
    L = _CPU_SAMPLE["L"]
    X = [xy[0] for xy in _CPU_SAMPLE["XY"]]
    Y = [xy[1] for xy in _CPU_SAMPLE["XY"]]
    oracle.build(L[:2], X[:1], Y[:1])   # load + warm
    t0 = time.perf_counter()
    oracle.build(L, X, Y)
    dt = time.perf_counter() - t0
    flops = build_flops(n, na, [40] * nds, [False] * nds)
    cores = len(os.sched_getaffinity(0))
    omp = os.environ.get("OMP_NUM_THREADS")
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": int(omp) if omp else cores,
            "kind": "oracle",
            "sample": f"{nds} of the 7 non-symmetric densities (k=40) x all {na} aux indices, nbf=400; "
                      f"{flops:.3g} algorithmic flop in {dt:.2f} s",
            "seconds": dt}


def run_reference(args, rank, world):
    if rank != 0:
        return
    steps = []
    for _ in range(args.warmup):
        cpu_baseline_sample()
    for _ in range(args.steps):
        steps.append(cpu_baseline_sample())
    v = statistics.median(s["value"] for s in steps)
    sec = statistics.median(s["seconds"] for s in steps)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (long double accumulation)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": steps[0]["sample"]},
            "cpu_baseline": {k: steps[0][k] for k in ("unit", "cores", "kind", "sample")} | {"value": v},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    from paper_2608_06536_b300 import inputs, jk

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.case == "profile":
        # same structure, a quarter of the aux indices (L = 768 MB > L2): for ncu captures
        m = inputs.molecule(400, 600, 400.0, [(40, True)] + [(40, False)] * 7, 0)
    else:
        m = inputs.multi_state()
    n, naux, ks, sym = m.n, m.naux, m.ks, m.sym
    flops = build_flops(n, naux, ks, sym)
    # --packed-factor: the factor resident as packed upper triangles (half the memory)
    Ld = (jk.pack_factor(m.L) if args.packed_factor else torch.from_numpy(m.L)).to(dev)
    Xd = [torch.from_numpy(x).to(dev) for x in m.X]
    Yd = [torch.from_numpy(y).to(dev) for y in m.Y]
    eng = jk.Engine(dev)
    eng.set_option("slicer", args.slicer)
    eng.set_option("syrk", args.syrk)
    eng.set_option("packed_factor", 1 if args.packed_factor else 0)
    prec = args.precision
    st = torch.cuda.current_stream(dev)

    # autotune (untimed): the fastest run-time configuration for this shape is
    # cached and every build below uses it
    tuned = None
    if args.config:
        # a fixed configuration (for profiling runs): no tuning
        for name, v in zip(("aux_chunk", "schedule", "raster"), args.config.split(",")):
            eng.set_option(name, int(v))
        tuned = {"fixed": args.config}
    elif args.tune:
        cfg, tms = eng.autotune(Ld, Xd, Yd, sym, prec, reps=1 if prec == "fp64" else 2)
        tuned = dict(cfg, ms=tms)
    # warm-up (also sizes the arena)
    for _ in range(args.warmup):
        J, K = eng.build(Ld, Xd, Yd, sym, prec)
    eng.sync_status()
    torch.cuda.synchronize(dev)

    # ---- device-resident timed region --------------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    eng.profile(True)
    eng.profile_reset()
    l0 = eng.launch_count()
    tf0 = eng.issued_tensor_flops()
    barrier(world)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        J, K = eng.build(Ld, Xd, Yd, sym, prec, J=J, K=K)
    e1.record(st)
    torch.cuda.synchronize(dev)
    barrier(world)
    ms = e0.elapsed_time(e1) / args.steps
    launches = eng.launch_count() - l0
    issued = eng.issued_tensor_flops() - tf0
    prof = eng.profile_read()
    eng.profile(False)
    clk = clocks.stop()
    eng.sync_status()
    ms_max = max_over_ranks(ms, world, dev)
    value = job_tflops(flops, ms_max, world)

    if args.quick:
        if rank == 0:
            print(json.dumps({"case": args.case, "engine": prec, "ms_per_step": ms_max, "value": value,
                              "kernels_ms": {k: v[0] / args.steps for k, v in prof.items()},
                              "launches_per_step": launches / args.steps, "tuned": tuned, "slicer": args.slicer,
                              "syrk": args.syrk, "packed_factor": bool(args.packed_factor),
                              "issued_tensor_tflops": issued / args.steps / (ms_max * 1e-3) / 1e12}),
                  flush=True)
        return

    # ---- end to end through the public API, host buffers ---------------------
    # --e2e-packed: the factor kept on the host as packed upper triangles (its
    # layout as a symmetric matrix), half the bytes over the host link
    Lh = (jk.pack_factor(m.L) if args.e2e_packed else torch.from_numpy(m.L)).pin_memory()
    Xh = [torch.from_numpy(x).pin_memory() for x in m.X]
    Yh = [torch.from_numpy(y).pin_memory() for y in m.Y]
    Jh = torch.empty((len(ks), n, n), dtype=torch.float64).pin_memory()
    Kh = torch.empty((len(ks), n, n), dtype=torch.float64).pin_memory()
    h2d = Lh.numel() * 8 + sum(x.numel() * 8 for x in Xh) + sum(y.numel() * 8 for y, s in zip(Yh, sym) if not s)
    d2h = (Jh.numel() + Kh.numel()) * 8
    e2e_steps = max(1, min(args.steps, 3))
    eng.set_option("packed_factor", 0)      # the host builds take the factor from host memory
    # jk_build_host: the library streams the factor to the device in aux chunks
    # on its own copy stream, overlapped with the build of the previous chunk;
    # densities up and J, K down on the caller's stream.  One untimed call sizes
    # the arena.
    eng.build_host(Lh, Xh, Yh, sym, prec, J=Jh, K=Kh, stream=st, packed=args.e2e_packed)
    barrier(world)
    torch.cuda.synchronize(dev)
    e0.record(st)
    for _ in range(e2e_steps):
        eng.build_host(Lh, Xh, Yh, sym, prec, J=Jh, K=Kh, stream=st, sync=False, packed=args.e2e_packed)
    e1.record(st)
    torch.cuda.synchronize(dev)
    eng.sync_status(st)
    ms_e2e = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, world, dev)
    e2e = {"value": job_tflops(flops, ms_e2e, world), "unit": "TFLOP/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": ms_e2e,
           "packed_factor": bool(args.e2e_packed),
           "path": "jk_build_host: pinned host inputs and outputs, factor streamed in aux chunks "
                   "overlapped with the build"}

    # ---- roofline of the dominant kernel ------------------------------------
    peaks, peak_src = load_peaks()
    top = max(prof.items(), key=lambda kv: kv[1][0]) if prof else ("none", (0.0, 0))
    top_name, (top_ms, top_cnt) = top
    roofline = None
    if top_name == "dgemm_fp64" and top_cnt:
        alg = panel_rank_flops(n, naux, ks, sym) * args.steps
        achieved = alg / (top_ms * 1e-3) / 1e12
        roofline = {"kernel": top_name, "bound": "alu", "achieved": achieved,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                    "peak_source": "FP64 FMA stream probe, 1.20 TFLOP/s (148 SM x 2 FMA/clk x 2032 MHz)",
                    "traffic": None, "avg_launch_ms": top_ms / top_cnt,
                    "share_of_step": top_ms / (ms * args.steps)}
    elif top_name == "ozgemm_tcgen05" and top_cnt:
        pk = peaks.get("bf16_tflops_sustained")
        traffic = None
        if args.case == "multi_state":
            per_step = (OZ_PANEL_BYTES_PER_P + OZ_RANK_BYTES_PER_P) * naux
            traffic = per_step * args.steps / top_cnt
        achieved = issued / (top_ms * 1e-3) / 1e12 if issued else None
        alg = panel_rank_flops(n, naux, ks, sym) * args.steps
        roofline = {"kernel": top_name, "bound": "tensor", "achieved": achieved, "peak": pk,
                    "unit": "TFLOP/s", "frac": (achieved / pk) if achieved else None,
                    "peak_source": f"bf16_tflops_sustained of {peak_src} (MEASURED_PEAKS)",
                    "achieved_counts": "dense BF16 MMA flops issued (21 slice pairs over padded tiles)",
                    "algorithmic_fp64_equiv_tflops": alg / (top_ms * 1e-3) / 1e12,
                    "traffic": traffic,
                    "traffic_note": "DRAM bytes per launch, ncu capture of the profile case scaled by naux",
                    "avg_launch_ms": top_ms / top_cnt,
                    "share_of_step": top_ms / (ms * args.steps)}

    if rank != 0:
        return
    cpu = cpu_baseline_sample(m.L)
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == "fp64" else "bf16-slices/fp32-tmem/int64 -> f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "engine": prec, "nbf": n, "naux": naux, "nd": len(ks),
                   "k": ks[0], "l2": "inputs larger than L2 (L = 3.07 GB FP64), no flush",
                   "parallelism": f"replicas x{world}", "tuned": tuned, "slicer": args.slicer,
                   "syrk": args.syrk, "packed_factor": bool(args.packed_factor)},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "launches_per_step": launches / args.steps,
        "kernels_ms": {k: v[0] / args.steps for k, v in prof.items()},
        "roofline": roofline,
        "cpu_baseline": {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def adjoint_flops(n, naux, ks, sym):
    """Algorithmic flops of the adjoint: 12 n^2 k naux (dX, dY with the panels
    recomputed) + 4 n^2 k naux (dL outer products) + 4 n^2 naux (J terms) per
    density."""
    return sum(12.0 * n * n * k * naux + 4.0 * n * n * k * naux + 4.0 * n * n * naux for k in ks)


def dense_flops(n, naux, nd):
    """Algorithmic flops of jk_build_dense (J and K) for nd dense densities:
    K 2n^3 naux for the panels L^P D and 2n^3 naux for the rank update, J
    2n^2 naux for the metric dot and 2n^2 naux for the back-contraction."""
    return nd * (4.0 * n ** 3 * naux + 4.0 * n * n * naux)


def pair_flops(n, naux, kl, syml, kr, symr):
    """Algorithmic flops of jk_pair with both pairings: the right densities'
    build plus, per map and right density, U_b = M_b Z_L (2 n^2 ctot_L) and the
    pair dots (2 n k_a per pair)."""
    ctot_l = sum(k if s else 2 * k for k, s in zip(kl, syml))
    contract = 2 * len(kr) * (2.0 * n * n * ctot_l + sum(2.0 * n * k for k in kl))
    return build_flops(n, naux, kr, symr) + contract


PAIR_WORKLOAD = ("bra-ket pairings: nbf=400 naux=2400 tau=400, 8 left x 8 right non-symmetric densities k=40; "
                 "jk_pair Jp and Kp")
LAPLACE_WORKLOAD = ("Laplace (LT-AO) builds: nbf=400 naux=2400 tau=400, 8 Gauss-Laguerre points, m=40 occupied "
                    "against virtual coefficient columns; jk_build_laplace weighted J and K")

DENSE_WORKLOAD = ("dense densities: nbf=400 naux=2400 tau=400, 8 general non-symmetric D_s "
                  "(N(0, 1/nbf^2) entries); jk_build_dense J and K, and jk_density_grad K(W) + J(V)")


def run_extra_case(args, rank, local):
    """Reported beside the headline workload (not the bench contract's line):
    the adjoint case, the uneven batch replayed as a CUDA graph, and the dense
    densities."""
    import numpy as np
    import torch
    from paper_2608_06536_b300 import inputs, jk

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    eng = jk.Engine(dev)
    st = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"case": args.case, "engine": args.precision}
    if args.case == "adjoint":
        m, W, V = inputs.adjoint_case(with_factor=False)
        L = inputs.factor_device(m.n, m.naux, m.tau, m.seed, device=dev)
        X = [torch.from_numpy(x).to(dev) for x in m.X]
        Y = [torch.from_numpy(y).to(dev) for y in m.Y]
        Wd = torch.tensor(np.array(W), device=dev)
        Vd = torch.tensor(np.array(V), device=dev)
        for _ in range(args.warmup):
            eng.adjoint(L, X, Y, m.sym, Wd, Vd, precision=args.precision)
        torch.cuda.synchronize(dev)
        e0.record(st)
        for _ in range(args.steps):
            eng.adjoint(L, X, Y, m.sym, Wd, Vd, precision=args.precision)
        e1.record(st)
        torch.cuda.synchronize(dev)
        eng.sync_status()
        ms = e0.elapsed_time(e1) / args.steps
        out.update({"workload": "adjoint nbf=600 naux=3600, 8 non-symmetric densities k=60, W,V N(0,1); "
                                "dX, dY and the symmetrized dL",
                    "ms_per_step": ms, "value": adjoint_flops(m.n, m.naux, m.ks, m.sym) / (ms * 1e-3) / 1e12,
                    "unit": "TFLOP/s (algorithmic)"})
    elif args.case == "dense":
        n, naux, nd = 400, 2400, 8
        L = inputs.factor_device(n, naux, 400.0, 0, device=dev)
        D = torch.from_numpy(inputs.dense_densities(n, nd, seed=0)).to(dev)
        W = torch.from_numpy(inputs.dense_densities(n, nd, seed=1)).to(dev)
        res = {}
        for name, call in (("build_dense", lambda: eng.build_dense(L, D, args.precision)),
                           ("density_grad", lambda: eng.density_grad(L, W, D, args.precision))):
            for _ in range(args.warmup):
                call()
            torch.cuda.synchronize(dev)
            e0.record(st)
            for _ in range(args.steps):
                call()
            e1.record(st)
            torch.cuda.synchronize(dev)
            eng.sync_status()
            ms = e0.elapsed_time(e1) / args.steps
            res[name] = {"ms_per_step": ms, "value": dense_flops(n, naux, nd) / (ms * 1e-3) / 1e12}
        out.update({"workload": DENSE_WORKLOAD, "unit": "TFLOP/s (algorithmic)", **res})
    elif args.case in ("pairs", "laplace"):
        n, naux, k, nq = 400, 2400, 40, 8
        L = inputs.factor_device(n, naux, 400.0, 0, device=dev)
        left = inputs.custom_densities(n, [k] * 8, seed=1)
        right = inputs.custom_densities(n, [k] * 8, seed=2)
        XL, YL = ([torch.from_numpy(x).to(dev) for x in side] for side in left)
        XR, YR = ([torch.from_numpy(x).to(dev) for x in side] for side in right)
        if args.case == "pairs":
            call = lambda: eng.pairs(L, XL, YL, None, XR, YR, None, args.precision)
            flops, workload = pair_flops(n, naux, [k] * 8, [False] * 8, [k] * 8, [False] * 8), PAIR_WORKLOAD
        else:
            t, u = np.polynomial.laguerre.laggauss(nq)
            alpha, w = t, u * np.exp(t)
            rng = np.random.default_rng([0, 5])
            ei = torch.from_numpy(-np.sort(rng.uniform(0.3, 1.5, k))).to(dev)
            ea = torch.from_numpy(np.sort(rng.uniform(0.2, 2.0, k))).to(dev)
            call = lambda: eng.build_laplace(L, XL[0], ei, +1, alpha, w, YL[0], ea, -1, args.precision)
            flops, workload = build_flops(n, naux, [k] * nq, [False] * nq), LAPLACE_WORKLOAD
        for _ in range(args.warmup):
            call()
        torch.cuda.synchronize(dev)
        e0.record(st)
        for _ in range(args.steps):
            call()
        e1.record(st)
        torch.cuda.synchronize(dev)
        eng.sync_status()
        ms = e0.elapsed_time(e1) / args.steps
        out.update({"workload": workload, "ms_per_step": ms, "value": flops / (ms * 1e-3) / 1e12,
                    "unit": "TFLOP/s (algorithmic)"})
    else:
        mols = inputs.uneven_batch(with_factor=False)

        def factor(mm):
            Lf = inputs.factor_device(mm.n, mm.naux, mm.tau, mm.seed, device=dev)
            return jk.pack_factor(Lf) if args.packed_factor else Lf      # packed: 104 GB instead of 208 GB

        eng.set_option("packed_factor", 1 if args.packed_factor else 0)
        eng.set_option("syrk", args.syrk)
        args_b = [(factor(mm), [torch.from_numpy(x).to(dev) for x in mm.X], [torch.from_numpy(y).to(dev) for y in mm.Y],
                   mm.sym) for mm in mols]
        flops = sum(build_flops(mm.n, mm.naux, mm.ks, mm.sym) for mm in mols)
        eng.build_batched(args_b, args.precision)
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream(dev)
        cs.wait_stream(st)
        with torch.cuda.stream(cs):
            with torch.cuda.graph(g, stream=cs):
                eng.build_batched(args_b, args.precision, stream=cs)
        st.wait_stream(cs)
        for _ in range(args.warmup):
            g.replay()
        torch.cuda.synchronize(dev)
        e0.record(st)
        for _ in range(args.steps):
            g.replay()
        e1.record(st)
        torch.cuda.synchronize(dev)
        eng.sync_status()
        ms = e0.elapsed_time(e1) / args.steps
        out.update({"workload": "uneven batch: 64 molecules nbf U{100..600}, naux 6 nbf, 560 non-symmetric "
                                "densities k = nbf/10 (208 GB of factors), one batched build replayed as a CUDA graph",
                    "ms_per_step": ms, "value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s (algorithmic)",
                    "packed_factor": bool(args.packed_factor)})
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["split", "fp64"], default="split")
    ap.add_argument("--case", choices=["multi_state", "profile", "adjoint", "batched", "dense", "pairs", "laplace"],
                    default="multi_state",
                    help="profile: nbf=400, naux=600 variant for ncu captures; adjoint, batched, dense, pairs, "
                         "laplace: extra reported cases")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="skip the autotuner (default configuration)")
    ap.add_argument("--config", default="",
                    help="fixed run-time configuration aux_chunk,schedule,raster (skips the autotuner)")
    ap.add_argument("--slicer", type=int, choices=[0, 1], default=0,
                    help="digit extraction of the vector slicer: 0 integer (default), 1 FP32 additions")
    ap.add_argument("--syrk", type=int, choices=[0, 1], default=0,
                    help="symmetric densities (split engine): 0 full rank update (default), "
                         "1 blocked symmetric rank update, the rest mirrored")
    ap.add_argument("--packed-factor", dest="packed_factor", action="store_true",
                    help="device factor stored as packed upper triangles (half the memory; chunks expanded "
                         "in the workspace)")
    ap.add_argument("--e2e-packed", dest="e2e_packed", action="store_true",
                    help="end-to-end leg with the factor on the host as packed upper triangles "
                         "(jk_build_host_packed: half the bytes over the host link)")
    ap.add_argument("--quick", action="store_true",
                    help="device-resident timing only (no e2e, no CPU baseline)")
    args = ap.parse_args()
    rank, world, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.case in ("adjoint", "batched", "dense", "pairs", "laplace"):
        run_extra_case(args, rank, local)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
