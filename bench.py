#!/usr/bin/env python
"""Throughput of the Cholesky J/K engine on one B300 (or N replicas).

One step = one full split-precision J/K build (panels L^P X, L^P Y on the
tensor cores, J metric dot, FP64 J back-contraction, K rank update, FP64
final reduction) for the large single molecule: nbf = 1000, naux = 5000,
sixteen non-symmetric transition densities of width 100, the 40 GB FP64
factor drawn on the device (seeded synthetic inputs).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--case large_single|multi_state|...] [--headline-only]

Prints ONE JSON line on rank 0.  `value` is algorithmic TFLOP/s (the
FP64-equivalent work of the build; the split path's slice products are cost,
not counted) with every input resident in HBM.  In the same line:
  e2e            the same metric through jk_build_host(_packed) with pinned
                 host inputs uploaded and J, K read back inside the timed region;
  fp64_gpu       the plain FP64 engine on the same inputs: time, TFLOP/s, the
                 split engine's speed-up over it;
  error          max |split - FP64 engine| per output, and both engines
                 against the CPU oracle on sampled entries;
  roofline       the dominant kernel (the tcgen05 sliced GEMM): algorithmic
                 TFLOP/s against the measured BF16 peak, beside the issued
                 BF16 MMA rate;
  j_stream       the J back-contraction: on the tensor cores its own
                 kernels (the transposed factor slicing and the scatter onto
                 J; its sliced GEMM runs inside the GEMM kind): time, HBM GB/s
                 of their algorithmic bytes against the measured HBM peak;
                 the FP64 form (dense-density builds) as HBM GB/s and FP64
                 TFLOP/s against the FP64 FMA rate this run measures with
                 the library's probe kernel;
  cpu_baseline   the oracle on a bounded, named sample of the same workload;
  configs        the other workloads (one molecule small, multi-state,
                 adjoint, uneven batch replayed as a CUDA graph), unless
                 --headline-only.
Under torchrun every rank runs its own replica (the path has no exchange
step); value = all ranks' work / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
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
WORKLOADS = {
    "large_single": "large single molecule: nbf=1000 naux=5000 tau=1000 (L = 40 GB FP64, drawn on the device), "
                    "16 non-symmetric transition densities k=100, split precision vs the FP64 engine",
    "multi_state": "multi-state nbf=400 naux=2400 tau=400, 8 densities k=40 (1 symmetric ground + 7 "
                   "non-symmetric transition), FP64 in/out",
    "small": "one molecule small: nbf=48 naux=300 tau=60, one non-symmetric density k=6",
    "profile": "the large single molecule's structure with naux=400 (L = 3.2 GB FP64, larger than L2), for ncu",
}
SPLIT_GATE = 1e-10       # absolute, output units (split engine)
FP64_GATE = 1e-12        # relative to max |output| (FP64 engine)

# ncu figures of the sliced GEMM (one capture of the profile case), valid only
# for the kernel sources they were taken on: keyed by kernel_source_hash().
# Each entry: per-launch DRAM bytes of a full-size launch (dram__bytes_read.sum
# + dram__bytes_write.sum of the capture, scaled by aux indices),
# sm__pipe_tensor_cycles_active (% of peak, elapsed) and the capture's command.
NCU_GEMM = {
    "5c4421038faf8689": {
        # profile case (naux=400, one aux chunk): panel launch 14.49 + 10.26 GB,
        # rank-update launch 52.66 + 2.65 GB; scaled to the headline's 338-index
        # chunks (x 338/400) and averaged over its two launches per chunk
        "traffic": 0.5 * (24.75 + 55.31) * 338 / 400 * 1e9,
        # sm__pipe_tensor_cycles_active: panel 56.8 %, rank update 56.3 %, time-weighted
        "tensor_pipe_active": 0.566,
        "capture": "ncu --set full --clock-control none -k regex:ozgemm -c 1 (panel) and -s 1 -c 1 (rank update) "
                   "python bench.py --case profile --quick --steps 1 --warmup 1 --config 400,1,0,0",
    },
}
KERNEL_SOURCES = ("ozgemm.cuh", "ozcfg.cuh", "tc.cuh", "fixed.cuh")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2608_06536_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def build_flops(n, naux, ks, sym):
    """Algorithmic flops of one build: panels 2n^2kA per half-transform, rank
    update 2n^2kA (n^2kA for a symmetric density), J back-contraction 2n^2A,
    gamma from the panel 2nkA, per density."""
    f = 0.0
    for k, s in zip(ks, sym):
        f += (3.0 if s else 6.0) * n * n * k * naux
        f += 2.0 * n * n * naux + 2.0 * n * k * naux
    return f


def panel_rank_flops(n, naux, ks, sym):
    """The part of build_flops the sliced GEMM carries (panels and rank updates)."""
    return sum((3.0 if s else 6.0) * n * n * k * naux for k, s in zip(ks, sym))


def jstream_bytes_flops(n, naux, nd):
    """Algorithmic HBM bytes and FP64 flops of the J back-contraction: the
    upper triangle of every L^P read once for all densities, J written once;
    one FMA per upper-triangle entry, aux index and density."""
    tri = n * (n + 1) // 2
    return 8.0 * tri * naux + 8.0 * nd * n * n, 2.0 * tri * naux * nd


def jtri_bytes(n, naux, nd, nchunks):
    """Algorithmic HBM bytes of the tensor-core J back-contraction's own
    kernels: the upper triangle of every L^P read twice (exponents, then
    digits) and written as six BF16 planes; per aux chunk the FP64 product
    C [n(n+1)/2][nd] read and J written over both triangles (read too after
    the first chunk)."""
    tri = n * (n + 1) // 2
    return (8.0 + 8.0 + 12.0) * tri * naux + nchunks * 8.0 * (tri * nd + 2.0 * nd * n * n) - 8.0 * nd * n * n


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


# ---------------------------------------------------------------------------
# The oracle on bounded samples (CPU baseline and reference arm)
# ---------------------------------------------------------------------------
# (densities, aux indices) of the oracle's sample per workload: about 10-30 s
# of CPU work on the machine's host cores.
CPU_SAMPLE = {"large_single": (2, 160), "profile": (2, 160), "multi_state": (3, 2400), "small": (1, 300)}


def cpu_sample_molecule(case):
    from paper_2608_06536_b300 import inputs
    if case in ("large_single", "profile"):
        return inputs.large_single()
    if case == "small":
        return inputs.one_molecule_small(with_factor=False)
    return inputs.multi_state(with_factor=False)


def cpu_baseline_sample(case, L=None, _cache={}):
    """The oracle as it stands on a bounded sample of the workload: the first
    `nds` non-symmetric densities over the first `na` aux indices (exact
    subsets of the same inputs, never extrapolated).  L: the workload's host
    factor, if the caller has it (else the needed slices are drawn)."""
    import numpy as np
    import oracle
    from paper_2608_06536_b300 import inputs
    m = cpu_sample_molecule(case)
    nds, na = CPU_SAMPLE.get(case, (2, 160))
    na = min(na, m.naux)
    sel = [s for s in range(m.nd) if not m.sym[s]][:nds]
    key = (case, na)
    if key not in _cache:
        _cache[key] = np.ascontiguousarray(L[:na]) if L is not None else inputs.factor(m.n, na, m.tau, m.seed)
    Ls = _cache[key]
    X = [m.X[s] for s in sel]
    Y = [m.Y[s] for s in sel]
    oracle.build(Ls[:2], X[:1], Y[:1])   # load + warm
    t0 = time.perf_counter()
    oracle.build(Ls, X, Y)
    dt = time.perf_counter() - t0
    flops = build_flops(m.n, na, [m.ks[s] for s in sel], [False] * len(sel))
    cores = len(os.sched_getaffinity(0))
    omp = os.environ.get("OMP_NUM_THREADS")
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": int(omp) if omp else cores,
            "kind": "oracle",
            "sample": f"{len(sel)} of the {m.nd} densities (k={m.ks[sel[0]]}) x the first {na} of {m.naux} aux "
                      f"indices, nbf={m.n}; {flops:.3g} algorithmic flop in {dt:.2f} s",
            "seconds": dt}


def run_reference(args, rank, world):
    if rank != 0:
        return
    case = args.case if args.case in CPU_SAMPLE else "large_single"
    steps = []
    for _ in range(args.warmup):
        cpu_baseline_sample(case)
    for _ in range(args.steps):
        steps.append(cpu_baseline_sample(case))
    v = statistics.median(s["value"] for s in steps)
    sec = statistics.median(s["seconds"] for s in steps)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (long double accumulation)", "data": "synthetic",
            "config": {"workload": WORKLOADS[case], "sample": steps[0]["sample"]},
            "cpu_baseline": {k: steps[0][k] for k in ("unit", "cores", "kind", "sample")} | {"value": v},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Measurement helpers
# ---------------------------------------------------------------------------
_T0 = time.perf_counter()


def phase(name):
    """Wall-clock progress on stderr (the JSON line stays alone on stdout)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {name}", file=sys.stderr, flush=True)


def timed(fn, steps, warmup, stream):
    """ms per call of fn() on `stream`: warmup untimed calls, then `steps`
    calls bracketed by CUDA events, synchronized on both sides."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def fp64_peak(eng, stream):
    """FP64 TFLOP/s of the library's FMA-stream probe (best of five launches)."""
    import torch
    eng.fp64_fma_probe(stream=stream)
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fl = eng.fp64_fma_probe(blocks_per_sm=4, iters=1 << 15, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        best = max(best, fl / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


def sample_entries(rng, nd, n, count):
    s = rng.integers(0, nd, count)
    mu = rng.integers(0, n, count)
    nu = rng.integers(0, n, count)
    s[:2] = [0, nd - 1]
    mu[:2] = [0, n - 1]
    nu[:2] = [n - 1, 0]
    return s, mu, nu


def gemm_roofline(prof, flops_alg_per_step, issued, steps, peaks, peak_src):
    ms, cnt = prof.get("ozgemm_tcgen05", (0.0, 0))
    if not cnt:
        return None
    pk = peaks.get("bf16_tflops_sustained")
    achieved = flops_alg_per_step * steps / (ms * 1e-3) / 1e12
    issued_tf = issued / (ms * 1e-3) / 1e12 if issued else None
    h = kernel_source_hash()
    ncu = NCU_GEMM.get(h)
    return {"kernel": "ozgemm_kernel (tcgen05 sliced GEMM: panels and rank updates)", "bound": "tensor",
            "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
            "achieved_counts": "algorithmic (FP64-equivalent) flops of the panels and rank updates, 6 n^2 k naux "
                               "per non-symmetric density; slice products are cost, not counted",
            "peak_source": f"bf16_tflops_sustained of the {peak_src} peaks (MEASURED_PEAKS.json)",
            "issued_tflops": issued_tf, "issued_frac": (issued_tf / pk) if issued_tf else None,
            "issued_counts": "dense BF16 MMA flops issued (21 slice pairs over the padded tiles)",
            "traffic": ncu["traffic"] if ncu else None,
            "tensor_pipe_active": ncu["tensor_pipe_active"] if ncu else None,
            "ncu_capture": ncu["capture"] if ncu else "none for the current kernel sources",
            "kernel_sources": h, "avg_launch_ms": ms / cnt, "launches": cnt}


def jstream_roofline(prof, n, naux, nd, steps, peaks, fp64_tflops, nchunks=1):
    ms, cnt = prof.get("jstream_fp64", (0.0, 0))
    if not cnt:
        ms, cnt = prof.get("j_tri", (0.0, 0))
        if not cnt:
            return None
        by = jtri_bytes(n, naux, nd, nchunks)
        per = ms / steps
        gbs = by / (per * 1e-3) / 1e9
        hbm = peaks.get("hbm_gbs")
        return {"kernel": "expo_tri_kernel, slice_tri_kernel, j_tri_add_kernel (J on the tensor cores: the "
                          "transposed factor slicing and the scatter; its sliced GEMM is in the GEMM kind)",
                "ms_per_step": per, "launches": cnt, "aux_chunks": nchunks, "algorithmic_bytes": by,
                "achieved_gbs": gbs, "hbm_peak_gbs": hbm, "hbm_frac": gbs / hbm, "bound": "hbm"}
    by, fl = jstream_bytes_flops(n, naux, nd)
    per = ms / steps
    gbs = by / (per * 1e-3) / 1e9
    tf = fl / (per * 1e-3) / 1e12
    hbm = peaks.get("hbm_gbs")
    return {"kernel": "jstream_sym_kernel (FP64 J back-contraction, second stream)", "ms_per_step": per,
            "launches": cnt, "algorithmic_bytes": by, "achieved_gbs": gbs, "hbm_peak_gbs": hbm,
            "hbm_frac": gbs / hbm, "fp64_tflops": tf, "fp64_peak_tflops": fp64_tflops,
            "fp64_frac": tf / fp64_tflops if fp64_tflops else None,
            "fp64_peak_source": "the library's FP64 FMA-stream probe (jk_debug_fp64_fma), measured in this run",
            "bound": "fp64" if (fp64_tflops and tf / fp64_tflops > gbs / hbm) else "hbm"}


# ---------------------------------------------------------------------------
# Headline: one molecule, split engine, beside the FP64 engine
# ---------------------------------------------------------------------------
def headline_molecule(case, dev):
    """(molecule, device factor, host factor or None)."""
    import torch
    from paper_2608_06536_b300 import inputs
    if case == "large_single":
        m = inputs.large_single()
        return m, inputs.factor_device(m.n, m.naux, m.tau, m.seed, device=dev), None
    if case == "profile":
        m = inputs.molecule(1000, 400, 1000.0, [(100, False)] * 16, 0, with_factor=False)
        return m, inputs.factor_device(m.n, m.naux, m.tau, m.seed, device=dev), None
    m = inputs.one_molecule_small() if case == "small" else inputs.multi_state()
    return m, torch.from_numpy(m.L).to(dev), m.L


def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    from paper_2608_06536_b300 import jk

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    st = torch.cuda.current_stream(dev)
    case = args.case
    m, Ld, Lhost = headline_molecule(case, dev)
    phase(f"inputs of {case} ready")
    n, naux, ks, sym = m.n, m.naux, m.ks, m.sym
    flops = build_flops(n, naux, ks, sym)
    Lfac = jk.pack_factor(Ld) if args.packed_factor else Ld     # packed: half the device memory
    Xd = [torch.from_numpy(x).to(dev) for x in m.X]
    Yd = [torch.from_numpy(y).to(dev) for y in m.Y]
    eng = jk.Engine(dev)
    eng.set_option("slicer", args.slicer)
    eng.set_option("syrk", args.syrk)
    eng.set_option("packed_factor", 1 if args.packed_factor else 0)
    eng.set_option("j_path", args.j_path)

    # run-time configuration: fixed (--config), or the autotuner's pick for
    # this shape (untimed; the cached pick is used by every build below)
    tuned = None
    if args.config:
        for name, v in zip(("aux_chunk", "schedule", "raster", "tile"), args.config.split(",")):
            eng.set_option(name, int(v))
        tuned = {"fixed": args.config}
    elif args.tune:
        cfg, tms = eng.autotune(Lfac, Xd, Yd, sym, "split", reps=1)
        tuned = dict(cfg, ms=tms)
    phase(f"configuration {tuned}")
    J, K = eng.build(Lfac, Xd, Yd, sym, "split")
    eng.sync_status()

    # ---- device-resident timed region (split engine) -----------------------
    for _ in range(args.warmup):
        eng.build(Lfac, Xd, Yd, sym, "split", J=J, K=K)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    eng.profile(True)
    eng.profile_reset()
    l0 = eng.launch_count()
    tf0 = eng.issued_tensor_flops()
    barrier(world)
    ms = timed(lambda: eng.build(Lfac, Xd, Yd, sym, "split", J=J, K=K), args.steps, 0, st)
    barrier(world)
    prof = eng.profile_read()
    launches = eng.launch_count() - l0
    issued = eng.issued_tensor_flops() - tf0
    eng.profile(False)
    clk = clocks.stop()
    eng.sync_status()
    ms_max = max_over_ranks(ms, world, dev)
    value = job_tflops(flops, ms_max, world)
    kernels_ms = {k: v[0] / args.steps for k, v in prof.items()}
    phase(f"split engine: {ms:.2f} ms per build")

    if args.quick:
        if rank == 0:
            print(json.dumps({"case": case, "ms_per_step": ms_max, "value": value, "kernels_ms": kernels_ms,
                              "launches_per_step": launches / args.steps, "tuned": tuned, "slicer": args.slicer,
                              "syrk": args.syrk, "packed_factor": bool(args.packed_factor), "j_path": args.j_path,
                              "issued_tensor_tflops": issued / args.steps / (ms_max * 1e-3) / 1e12,
                              "clocks": clk}), flush=True)
        return

    # ---- the FP64 engine on the same inputs --------------------------------
    fp64 = None
    Jf = Kf = None
    if not args.no_fp64:
        nwarm = max(1, naux // 10)
        eng.build(Lfac[:nwarm], Xd, Yd, sym, "fp64")        # warm-up on the first tenth of the aux indices
        torch.cuda.synchronize(dev)
        Jf, Kf = torch.empty_like(J), torch.empty_like(K)
        ms64 = timed(lambda: eng.build(Lfac, Xd, Yd, sym, "fp64", J=Jf, K=Kf), 1, 0, st)
        eng.sync_status()
        phase(f"FP64 engine: {ms64:.1f} ms per build")
        fp64 = {"ms_per_step": ms64, "value": flops / (ms64 * 1e-3) / 1e12, "unit": "TFLOP/s",
                "speedup_split_over_fp64": ms64 / ms_max, "steps": 1,
                "how": "the plain FP64 engine (FP64 SIMT GEMMs, FP64 J kernels) on the same inputs: one timed "
                       "build after a warm-up build on the first tenth of the aux indices"}

    # ---- errors: split vs FP64 engine (all entries), both vs the oracle ----
    peaks, peak_src = load_peaks()
    error = None
    if rank == 0 and not args.no_oracle and fp64 is not None:
        import oracle
        Lh = torch.from_numpy(Lhost) if Lhost is not None else torch.empty(Ld.shape, dtype=Ld.dtype).copy_(Ld)
        s, mu, nu = sample_entries(np.random.default_rng(2), len(ks), n, args.samples)
        t0 = time.perf_counter()
        Jo, Ko = oracle.sample(Lh.numpy(), m.X, m.Y, s, mu, nu)
        t_or = time.perf_counter() - t0
        del Lh
        phase(f"oracle samples: {t_or:.1f} s")
        Jn, Kn, Jfn, Kfn = (t.cpu().numpy() for t in (J, K, Jf, Kf))
        err = {
            "split_vs_fp64_J": float(np.abs(Jn - Jfn).max()), "split_vs_fp64_K": float(np.abs(Kn - Kfn).max()),
            "split_vs_oracle_J": float(np.abs(Jn[s, mu, nu] - Jo).max()),
            "split_vs_oracle_K": float(np.abs(Kn[s, mu, nu] - Ko).max()),
            "fp64_vs_oracle_J": float(np.abs(Jfn[s, mu, nu] - Jo).max()),
            "fp64_vs_oracle_K": float(np.abs(Kfn[s, mu, nu] - Ko).max()),
            "max_abs_J": float(np.abs(Jfn).max()), "max_abs_K": float(np.abs(Kfn).max())}
        gate_j = max(SPLIT_GATE, err["fp64_vs_oracle_J"])
        gate_k = max(SPLIT_GATE, err["fp64_vs_oracle_K"])
        error = dict(err, samples=int(args.samples), oracle_seconds=t_or,
                     split_gate_abs=SPLIT_GATE, fp64_gate_rel=FP64_GATE,
                     split_within_gate=bool(err["split_vs_oracle_J"] <= gate_j and
                                            err["split_vs_oracle_K"] <= gate_k),
                     fp64_within_gate=bool(err["fp64_vs_oracle_J"] <= FP64_GATE * err["max_abs_J"] and
                                           err["fp64_vs_oracle_K"] <= FP64_GATE * err["max_abs_K"]),
                     how="max |error| over all entries (split vs the FP64 engine) and over sampled entries "
                         "(both engines vs the CPU oracle, long-double accumulation)")

    # ---- end to end through the public API, host buffers -------------------
    # the oracle's CPU baseline below takes the first aux indices of the factor
    Lcpu = np.ascontiguousarray(Lhost[:CPU_SAMPLE[case][1]]) if Lhost is not None else \
        Ld[:CPU_SAMPLE[case][1]].cpu().numpy()
    e2e = None
    if not args.no_e2e:
        packed_link = args.e2e_link == "packed"
        src = jk.pack_factor(Ld) if packed_link else Ld          # packed on the device: half the upload
        Lup = torch.empty(src.shape, dtype=src.dtype, pin_memory=True)
        Lup.copy_(src)
        del src
        Xh = [torch.from_numpy(x).pin_memory() for x in m.X]
        Yh = [torch.from_numpy(y).pin_memory() for y in m.Y]
        Jh = torch.empty((len(ks), n, n), dtype=torch.float64).pin_memory()
        Kh = torch.empty((len(ks), n, n), dtype=torch.float64).pin_memory()
        h2d = Lup.numel() * 8 + sum(x.numel() * 8 for x in Xh) + sum(y.numel() * 8 for y, s in zip(Yh, sym) if not s)
        d2h = (Jh.numel() + Kh.numel()) * 8
        e2e_steps = max(1, min(args.steps, 3))
        eng.set_option("packed_factor", 0)      # the host builds take the factor from host memory
        eng.build_host(Lup, Xh, Yh, sym, "split", J=Jh, K=Kh, stream=st, packed=packed_link)
        barrier(world)
        ms_e2e = timed(lambda: eng.build_host(Lup, Xh, Yh, sym, "split", J=Jh, K=Kh, stream=st, sync=False,
                                              packed=packed_link), e2e_steps, 0, st)
        eng.sync_status(st)
        ms_e2e = max_over_ranks(ms_e2e, world, dev)
        phase(f"end to end: {ms_e2e:.1f} ms per build")
        e2e = {"value": job_tflops(flops, ms_e2e, world), "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": ms_e2e,
               "steps": e2e_steps, "packed_factor": packed_link,
               "path": ("jk_build_host_packed" if packed_link else "jk_build_host") +
                       ": pinned host inputs and outputs, the factor streamed in aux chunks on the library's copy "
                       "stream, overlapped with the chunk builds; J, K read back"}
        del Lup

    # ---- rooflines ----------------------------------------------------------
    fp64_tf = fp64_peak(eng, st)
    roofline = gemm_roofline(prof, panel_rank_flops(n, naux, ks, sym), issued, args.steps, peaks, peak_src)
    # three J kernels per aux chunk (exponents, digits, scatter)
    nchunks = max(1, round(prof.get("j_tri", (0.0, 0))[1] / (3 * args.steps)))
    jstream = jstream_roofline(prof, n, naux, len(ks), args.steps, peaks, fp64_tf, nchunks)
    if fp64 is not None:
        fp64["fp64_pipe_peak_tflops"] = fp64_tf
        fp64["fp64_pipe_frac"] = fp64["value"] / fp64_tf

    del Ld, Lfac, Xd, Yd, J, K, Jf, Kf
    eng.close()
    torch.cuda.empty_cache()

    configs = None
    if not args.headline_only and case == "large_single":
        configs = other_configs(dev, st)

    if rank != 0:
        return
    cpu = cpu_baseline_sample(case, Lcpu)
    phase("cpu baseline measured")
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16-slices/fp32-tmem/int64 -> f64",
        "data": "synthetic (seeded; the paper's molecules stand in)",
        "config": {"workload": WORKLOADS[case], "engine": "split", "nbf": n, "naux": naux, "nd": len(ks),
                   "k": ks[0], "l2": "inputs larger than L2 (factor %.1f GB FP64), no flush" % (8e-9 * n * n * naux),
                   "parallelism": f"replicas x{world}", "tuned": tuned, "slicer": args.slicer,
                   "syrk": args.syrk, "packed_factor": bool(args.packed_factor), "j_path": args.j_path},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "launches_per_step": launches / args.steps,
        "kernels_ms": kernels_ms,
        "fp64_gpu": fp64,
        "error": error,
        "roofline": roofline,
        "j_stream": jstream,
        "cpu_baseline": {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "clocks": clk,
        "configs": configs,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# The other workloads, reported beside the headline (same JSON line)
# ---------------------------------------------------------------------------
def measure_small(dev, st, reps=200):
    """One molecule small: latency-bound; microseconds per build, both engines."""
    import torch
    from paper_2608_06536_b300 import inputs, jk
    m = inputs.one_molecule_small()
    L = torch.from_numpy(m.L).to(dev)
    X = [torch.from_numpy(x).to(dev) for x in m.X]
    Y = [torch.from_numpy(y).to(dev) for y in m.Y]
    eng = jk.Engine(dev)
    out = {"workload": WORKLOADS["small"]}
    for prec in ("split", "fp64"):
        J, K = eng.build(L, X, Y, m.sym, prec)
        l0 = eng.launch_count()
        ms = timed(lambda: eng.build(L, X, Y, m.sym, prec, J=J, K=K), reps, 10, st)
        nl = (eng.launch_count() - l0) / (reps + 10)
        eng.sync_status()
        out[prec] = {"us_per_build": ms * 1e3, "launches_per_build": nl,
                     "value": build_flops(m.n, m.naux, m.ks, m.sym) / (ms * 1e-3) / 1e12}
    eng.close()
    return out


def measure_multi_state(dev, st, steps=5, warmup=2):
    """Multi-state workload, both engines (FP64: one timed build)."""
    import torch
    from paper_2608_06536_b300 import inputs, jk
    m = inputs.multi_state()
    L = torch.from_numpy(m.L).to(dev)
    X = [torch.from_numpy(x).to(dev) for x in m.X]
    Y = [torch.from_numpy(y).to(dev) for y in m.Y]
    eng = jk.Engine(dev)
    fl = build_flops(m.n, m.naux, m.ks, m.sym)
    cfg, _ = eng.autotune(L, X, Y, m.sym, "split", reps=1)
    out = {"workload": WORKLOADS["multi_state"], "tuned": cfg}
    for prec, (s_, w_) in (("split", (steps, warmup)), ("fp64", (1, 1))):
        J, K = eng.build(L, X, Y, m.sym, prec)
        ms = timed(lambda: eng.build(L, X, Y, m.sym, prec, J=J, K=K), s_, w_, st)
        eng.sync_status()
        out[prec] = {"ms_per_step": ms, "value": fl / (ms * 1e-3) / 1e12, "steps": s_}
    out["speedup_split_over_fp64"] = out["fp64"]["ms_per_step"] / out["split"]["ms_per_step"]
    eng.close()
    return out


def measure_adjoint(dev, st, steps=2, warmup=1, slices=7):
    """Adjoint case: dX, dY and the symmetrized dL, split (7 slices per
    operand unless `slices` says 6) and FP64 engines."""
    import numpy as np
    import torch
    from paper_2608_06536_b300 import inputs, jk
    m, W, V = inputs.adjoint_case(with_factor=False)
    L = inputs.factor_device(m.n, m.naux, m.tau, m.seed, device=dev)
    X = [torch.from_numpy(x).to(dev) for x in m.X]
    Y = [torch.from_numpy(y).to(dev) for y in m.Y]
    Wd = torch.tensor(np.array(W), device=dev)
    Vd = torch.tensor(np.array(V), device=dev)
    eng = jk.Engine(dev)
    eng.set_option("adjoint_slices", slices)
    fl = adjoint_flops(m.n, m.naux, m.ks, m.sym)
    out = {"workload": "adjoint: nbf=600 naux=3600, 8 non-symmetric densities k=60, W, V N(0,1); dX, dY and the "
                       "symmetrized dL", "algorithmic_flop": fl, "split_slices": slices}
    for prec, (s_, w_) in (("split", (steps, warmup)), ("fp64", (1, 1))):
        ms = timed(lambda: eng.adjoint(L, X, Y, m.sym, Wd, Vd, precision=prec), s_, w_, st)
        eng.sync_status()
        out[prec] = {"ms_per_step": ms, "value": fl / (ms * 1e-3) / 1e12, "steps": s_}
    out["speedup_split_over_fp64"] = out["fp64"]["ms_per_step"] / out["split"]["ms_per_step"]
    eng.close()
    del L
    torch.cuda.empty_cache()
    return out


def measure_batched(dev, st, steps=2, warmup=1):
    """Uneven batch: one batched split build of 64 molecules, captured in a
    CUDA graph and replayed; launches counted at capture."""
    import torch
    from paper_2608_06536_b300 import inputs, jk
    mols = inputs.uneven_batch(with_factor=False)
    eng = jk.Engine(dev)
    args_b = [(inputs.factor_device(mm.n, mm.naux, mm.tau, mm.seed, device=dev),
               [torch.from_numpy(x).to(dev) for x in mm.X], [torch.from_numpy(y).to(dev) for y in mm.Y], mm.sym)
              for mm in mols]
    flops = sum(build_flops(mm.n, mm.naux, mm.ks, mm.sym) for mm in mols)
    eng.build_batched(args_b, "split")
    torch.cuda.synchronize(dev)
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream(dev)
    cs.wait_stream(st)
    l0 = eng.launch_count()
    with torch.cuda.stream(cs):
        with torch.cuda.graph(g, stream=cs):
            eng.build_batched(args_b, "split", stream=cs)
    captured = eng.launch_count() - l0
    st.wait_stream(cs)
    ms = timed(g.replay, steps, warmup, st)
    eng.sync_status()
    out = {"workload": "uneven batch: 64 molecules nbf U{100..600}, naux 6 nbf, 560 non-symmetric densities "
                       "k = nbf/10 (208 GB of factors), one batched split build replayed as a CUDA graph",
           "ms_per_step": ms, "value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s (algorithmic)",
           "launches_per_build": captured, "steps": steps}
    eng.close()
    del args_b, g
    torch.cuda.empty_cache()
    return out


def other_configs(dev, st):
    out = {}
    for name, fn in (("one_molecule_small", measure_small), ("multi_state", measure_multi_state),
                     ("adjoint", measure_adjoint), ("uneven_batch", measure_batched)):
        t0 = time.perf_counter()
        try:
            out[name] = fn(dev, st)
            phase(f"{name} measured")
        except Exception as e:          # reported, never silently dropped
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = time.perf_counter() - t0
    return out


# ---------------------------------------------------------------------------
# Single extra cases (bench.py --case ...), one JSON line each
# ---------------------------------------------------------------------------
PAIR_WORKLOAD = ("bra-ket pairings: nbf=400 naux=2400 tau=400, 8 left x 8 right non-symmetric densities k=40; "
                 "jk_pair Jp and Kp")
LAPLACE_WORKLOAD = ("Laplace (LT-AO) builds: nbf=400 naux=2400 tau=400, 8 Gauss-Laguerre points, m=40 occupied "
                    "against virtual coefficient columns; jk_build_laplace weighted J and K")
DENSE_WORKLOAD = ("dense densities: nbf=400 naux=2400 tau=400, 8 general non-symmetric D_s "
                  "(N(0, 1/nbf^2) entries); jk_build_dense J and K, and jk_density_grad K(W) + J(V)")


def run_extra_case(args, rank, local):
    import numpy as np
    import torch
    from paper_2608_06536_b300 import inputs, jk

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    st = torch.cuda.current_stream(dev)
    if args.case == "adjoint":
        out = measure_adjoint(dev, st, args.steps, args.warmup, args.adjoint_slices)
    elif args.case == "batched":
        out = measure_batched(dev, st, args.steps, args.warmup)
    elif args.case == "dense":
        eng = jk.Engine(dev)
        n, naux, nd = 400, 2400, 8
        L = inputs.factor_device(n, naux, 400.0, 0, device=dev)
        D = torch.from_numpy(inputs.dense_densities(n, nd, seed=0)).to(dev)
        W = torch.from_numpy(inputs.dense_densities(n, nd, seed=1)).to(dev)
        out = {"workload": DENSE_WORKLOAD, "unit": "TFLOP/s (algorithmic)"}
        for name, call in (("build_dense", lambda: eng.build_dense(L, D, args.precision)),
                           ("density_grad", lambda: eng.density_grad(L, W, D, args.precision))):
            ms = timed(call, args.steps, args.warmup, st)
            eng.sync_status()
            out[name] = {"ms_per_step": ms, "value": dense_flops(n, naux, nd) / (ms * 1e-3) / 1e12}
    else:
        eng = jk.Engine(dev)
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
        ms = timed(call, args.steps, args.warmup, st)
        eng.sync_status()
        out = {"workload": workload, "ms_per_step": ms, "value": flops / (ms * 1e-3) / 1e12,
               "unit": "TFLOP/s (algorithmic)"}
    out = {"case": args.case, "engine": args.precision, **out}
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["split", "fp64"], default="split",
                    help="engine of the single extra cases (the headline times both)")
    ap.add_argument("--case", default="large_single",
                    choices=["large_single", "multi_state", "small", "profile", "adjoint", "batched", "dense",
                             "pairs", "laplace"],
                    help="large_single: the headline workload; multi_state, small: the other build workloads in "
                         "the headline's form; profile: the large single molecule with naux=400 for ncu captures; "
                         "adjoint, batched, dense, pairs, laplace: single extra cases")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="skip the autotuner (default configuration)")
    ap.add_argument("--config", default="",
                    help="fixed run-time configuration aux_chunk,schedule,raster[,tile] (skips the autotuner)")
    ap.add_argument("--slicer", type=int, choices=[0, 1], default=0,
                    help="digit extraction of the vector slicer: 0 integer, 1 FP32 additions")
    ap.add_argument("--syrk", type=int, choices=[0, 1], default=0,
                    help="symmetric densities: 0 full rank update, 1 blocked symmetric rank update")
    ap.add_argument("--j-path", dest="j_path", type=int, choices=[-1, 0, 1], default=-1,
                    help="split builds' J: -1 automatic, 0 FP64 pass on a second stream, 1 tensor cores")
    ap.add_argument("--packed-factor", dest="packed_factor", action="store_true",
                    help="device factor stored as packed upper triangles (half the memory)")
    ap.add_argument("--e2e-link", dest="e2e_link", choices=["packed", "full"], default="packed",
                    help="end-to-end leg: packed (jk_build_host_packed, the factor's upper triangles: half the "
                         "bytes over the host link; default) or full (jk_build_host)")
    ap.add_argument("--quick", action="store_true", help="device-resident timing only")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 engine (and the error comparison)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle's sampled entries")
    ap.add_argument("--samples", type=int, default=24, help="oracle-sampled entries of the error check")
    ap.add_argument("--headline-only", action="store_true", help="skip the other workloads")
    ap.add_argument("--adjoint-slices", dest="adjoint_slices", type=int, choices=[6, 7], default=7,
                    help="--case adjoint: BF16 slices per operand of the split adjoint")
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
