"""Benchmark of the fused D1Q3Q3 collide-stream step on one lattice of N = 2^26 nodes.

Workload (steepening acoustic wave): rho = 1 + 0.1 sin(2 pi j/N), u = 0.1 sin(2 pi j/N),
adiabatic pressure, periodic, lambda = 1, free rate s_e = 1.2 with the paper's coupled rates.
One benchmark "step" is one lattice time step (every stage of the hot path over all N nodes).
The headline is FP32 on shifted populations; FP64 is measured on the same workload beside it.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (the single lattice is not partitioned:
replicas only); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GLUPS (both distributions) & % HBM peak; batched-FP32 and adjoint vs plain FP64"
UNIT = "GLUPS"
N_NODES = 1 << 26
S_E = 1.2
AMP = 0.1
# Algorithmic bytes per node-update: the six populations read and written once (FP32 / FP64).
BYTES_PER_NODE = {"f32": 48, "f64": 96}
WORKLOAD = "steepening acoustic wave, single periodic lattice N=2^26, lambda=1, s_e=1.2"
# DRAM bytes per node per launch of the step kernel, measured with ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) on the same workload at N = 2^23 and scaled to a full launch by the node
# count (traffic is proportional to the nodes); keyed by (precision, k, block_threads,
# nodes_per_thread) of the current kernel version. Summaries: profiles/step_tiles_*.md.
# Arithmetic per node-update for the ALU roofline (halo recomputation excluded). FP32: the scaled node
# update as the step kernel implements it (moments, equation of state with the series log1p and
# expm1, equilibria, relaxation, source, M^-1): 19 add/sub + 22 mul + 33 fma (2 flops) + 3 reciprocals
# (1 flop) = 110 flops. FP64: the kernel's executed FP64 arithmetic per node-update from ncu at (1, 256, 2),
# N = 2^23: (2 DFMA + DADD + DMUL) / nodes = 95.8 (its log1p and expm1 run in double-float on the FP32
# pipes, the reciprocals as FP32 estimates refined by FP64 Newton steps; the FP64 pipe is 85 % busy).
# The same FP32 node update in FMA-pipe lane operations (an add, a multiply or a fused multiply-add is
# one): 19 + 22 + 33 = 74 per node-step, the 3 reciprocals running on the multi-function unit (ncu's
# paired-instruction counts at (8, 128, 4), N = 2^23, ghost-refresh tiles: 2 (FADD2 + FFMA2 + FMUL2) /
# computed node-steps = 2 x 2,788,102,144 / (18397 x 512 x 8) = 74.0; profiles/step_tiles_f32_k8_128x4_N8M.md).
LANE_OPS_PER_NODE_F32 = 74.0
FLOPS_PER_NODE = {"f32": 110.0, "f64": (2 * 236744704 + 177558528 + 152193024) / 8388608}
METHOD_FLOPS_PER_NODE = 110.0
# Peak arithmetic per SM per clock from the unit counts: 128 FP32 FMA lanes (256 flops); FP64 at
# 2 FMA per SM per clock (4 flops; the nominal 1.25 TFLOP/s of the part at 152 SMs, 2.07 GHz).
FLOPS_PER_SM_CLOCK = {"f32": 256.0, "f64": 4.0}
# FP32 operations (each lane of FADD2 / FFMA2 / FMUL2 one lane-operation) per computed node-step of
# the double-float step kernel on paired lanes, from ncu at N = 2^23, (8, 128, 4), entropy source in
# FP32 where it is below 2^-32 of the field scale: 2 x (8,805,052,416 FADD2 + 18,397,548,544 FFMA2 +
# 2,183,366,656 FMUL2) thread-instructions (no scalar FADD / FFMA / FMUL) over 17,477 x 512 x 8
# node-steps = 821.0 (profiles/step_tiles_df_N8M.md).
DF_FP32_OPS_PER_COMPUTED = 2 * (8805052416 + 18397548544 + 2183366656) / (17477 * 512 * 8)
TRAFFIC_BYTES_PER_NODE = {("f32", 8, 128, 4): (201.492224e6 + 153.174272e6) / 8388608,
                          ("f32", 8, 64, 4): (201.407232e6 + 153.744896e6) / 8388608,
                          ("f32", 8, 256, 4): (201.421568e6 + 152.067072e6) / 8388608,
                          ("f64", 1, 256, 2): (403.062016e6 + 347.52768e6) / 8388608}


def tile_span_f32(nt: int, v: int) -> int:
    """Nodes an FP32 tile of nt threads x v nodes spans: with four nodes per thread its warps overlap by
    4 ghost nodes per side (the step kernel's ghost-refresh tiles)."""
    return nt * v - (2 * 4 * (nt // 32 - 1) if v == 4 else 0)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.dev = device_index
        # The raw samples go to LBM_CLOCKS_DIR (default: the system's temporary directory).
        out_dir = os.environ.get("LBM_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_rank{device_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


_FIELDS = {}


def workload_fields(N: int):
    if N not in _FIELDS:
        from paper_1802_02369_gb300 import workloads as W

        _FIELDS[N] = W.steepening_wave(N, AMP, W.reference_pressure())
    return _FIELDS[N]


# ---------------------------------------------------------------------------------------------

def cpu_oracle_rate(N_sample: int, budget_s: float, nthreads: int):
    """Times the oracle (as it stands) on the first N_sample nodes of the workload, periodic,
    for as many steps as fit about budget_s seconds. Returns (GLUPS, steps, seconds)."""
    import oracle as O

    ph = O.default_phys()
    rho, u, p = workload_fields(N_SAMPLE_FULL)
    rho, u, p = rho[:N_sample], u[:N_sample], p[:N_sample]
    fd = O.init(ph, rho, u, p=p)
    r = O.coupled_rates(S_E)
    t0 = time.perf_counter()
    fd = O.run(ph, r, fd, 1, nthreads)
    t1 = time.perf_counter() - t0
    steps = max(1, int(budget_s / max(t1, 1e-6)))
    t0 = time.perf_counter()
    O.run(ph, r, fd, steps, nthreads)
    dt = time.perf_counter() - t0
    return N_sample * steps / dt / 1e9, steps, dt


N_SAMPLE_FULL = N_NODES
N_SAMPLE = 1 << 22


def run_reference(args, rank: int):
    """The CPU oracle as the reference arm (rank 0 only). Each benchmark step is one oracle time
    step on a periodic sample of the workload's first n nodes, n sized from a calibration run so
    that the whole run takes about two minutes."""
    if rank != 0:
        return
    import oracle as O

    O.build()
    cores = os.cpu_count() or 1
    ph = O.default_phys()
    r = O.coupled_rates(S_E)
    rho, u, p = workload_fields(N_NODES)
    cal_n = 1 << 20
    fd = O.init(ph, rho[:cal_n], u[:cal_n], p=p[:cal_n])
    t0 = time.perf_counter()
    O.run(ph, r, fd, 2, cores)
    rate = 2 * cal_n / (time.perf_counter() - t0)
    nsteps = args.warmup + args.steps
    n = int(min(1 << 22, max(4096, rate * 120.0 / max(1, nsteps))))
    fd = O.init(ph, rho[:n], u[:n], p=p[:n])
    fd = O.run(ph, r, fd, args.warmup, cores)
    t0 = time.perf_counter()
    O.run(ph, r, fd, args.steps, cores)   # the K timed steps in one oracle call
    tsum = time.perf_counter() - t0
    value = n * args.steps / tsum / 1e9
    sample = f"first {n} nodes of the workload (periodic), {args.steps} oracle steps in one call, FP64"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tsum / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N_NODES, "precision": "f64 (CPU oracle)", "sample_nodes": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(value: float, dist, device: str = "cuda") -> float:
    """The largest value over all ranks (the whole-job time of replicas started together)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


MIN_TIMED_MS = 200.0
MAX_REPEATS = 200


def time_device_repeats(lat, torch, steps: int, warmup: int, dist, world: int, min_ms: float = MIN_TIMED_MS):
    """Device-resident timing: `warmup` untimed lattice steps, then timed regions of exactly `steps`
    lattice steps, each between CUDA events on the library's stream and bracketed by a barrier and a
    device synchronisation on both sides, the maximum over ranks taken per region. Regions are repeated
    (the state keeps advancing) until they add up to min_ms; returns the list of region times in ms (the
    same count on every rank, since each rank sees the same maxima)."""
    st = lat.stream
    if warmup > 0:
        lat.step(warmup)
    times = []
    while True:
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        lat.step(steps)
        e1.record(st)
        torch.cuda.synchronize()
        times.append(max_over_ranks(e0.elapsed_time(e1), dist))
        if dist is not None:
            dist.barrier()
        if sum(times) >= min_ms or len(times) >= MAX_REPEATS:
            return times


def time_device(lat, torch, steps: int, warmup: int, dist, world: int, min_ms: float = MIN_TIMED_MS):
    """Median time in ms of the timed regions of time_device_repeats."""
    return float(np.median(time_device_repeats(lat, torch, steps, warmup, dist, world, min_ms)))


BATCH_ENTROPY_BAND = (-0.15, 0.0)
BATCH_ORACLE_LATTICES = 4


def run_batched(args, lbm, torch, hbm_peak, world):
    """Ragged batch of independent Riemann problems (4096 lattices, lengths U[512, 65536], s_e
    U[1.0, 1.9], pressures in units of p0, periodic or bounce-back), FP32, autotuned tile shape.

    The timed set is the draw restricted to Riemann problems that stay inside the scheme's linearly
    stable region, as the stability tests pin it: both states with -0.15 c_p <= s - s0 <= 0, and the
    velocity of the exact solution's star region below the stable flow speed of the lattice's s_e
    (workloads.STABLE_FLOW_SPEED). Every lattice then stays finite over the 2000 steps, so the throughput is that of the method's hot path at its stated
    accuracy (L1(rho) against the oracle: the CPU leg and the parity tests). It runs as one persistent
    launch replayed from a CUDA graph (the configuration's mode, the value) and, for comparison, as one
    launch per k steps. The unrestricted draw, on which most lattices blow up (linear instability of the
    scheme at entropies above about 0.1 c_p), is reported as a record beside it: its flag count and its
    rate, which times NaN arithmetic on the flagged lattices."""
    from paper_1802_02369_gb300 import workloads as W

    nlat = args.batched_lattices
    steps = args.batched_steps
    out = {}
    for which, band in (("stable", BATCH_ENTROPY_BAND), ("literal", None)):
        bat = W.ragged_batch(nlat, 1802, W.reference_pressure(), entropy_range=band, stable_flow=band is not None)
        ntot = int(bat.offsets[-1])
        fields = [torch.from_numpy(x).cuda() for x in (bat.rho, bat.u, bat.p)]
        lat = lbm.Lattice(bat.lengths, s_e=bat.s_e, bc=bat.bc, precision="f32")
        lat.set_state(*fields)
        if args.batched_config:
            lat.set_config(*[int(x) for x in args.batched_config.split(",")])
            k, nt, vpt = lat.get_config()
        else:
            k, nt, vpt = lat.autotune(1)
        timings, flagged, rho_small = {}, {}, None
        for mode in (("graph", "launch") if which == "stable" else ("launch",)):
            lat.set_mode(mode)
            lat.set_state(*fields)
            lat.step(steps)                   # warm-up (in graph mode: captures the graph)
            lat.set_state(*fields)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(lat.stream)
            lat.step(steps)                   # launch: ceil(steps / k) launches; graph: one persistent launch
            e1.record(lat.stream)
            torch.cuda.synchronize()
            timings[mode] = (e0.elapsed_time(e1), lat.status())
            _, flags, _ = lat.diagnostics()
            flagged[mode] = int((flags != 0).sum())
            if which == "stable" and mode == "graph":
                rho = lat.moments(device=True)[0]
                small = np.argsort(bat.lengths)[:BATCH_ORACLE_LATTICES]
                rho_small = {int(b): rho[int(bat.offsets[b]):int(bat.offsets[b + 1])].cpu().numpy() for b in small}
                del rho
        lat.close()
        del fields
        torch.cuda.empty_cache()
        rate = lambda t: world * ntot * steps / (t * 1e-3) / 1e9
        mode = "graph" if which == "stable" else "launch"
        ms, status = timings[mode]
        glups = rate(ms)
        launches = (steps + k - 1) // k
        alg = ntot * BYTES_PER_NODE["f32"] * launches   # one state read + write per block of k steps
        achieved = alg / (ms * 1e-3) / 1e9
        r = {"value": glups, "unit": UNIT, "lattices": nlat, "nodes": ntot, "steps": steps, "ms": ms,
             "steps_per_launch_block": k, "block_threads": nt, "nodes_per_thread": vpt,
             "mode": {"launch": "one kernel launch per k steps",
                      "graph": "one persistent kernel launch replayed from a CUDA graph"}[mode],
             "value_by_mode": {m: rate(t[0]) for m, t in timings.items()}, "status": status,
             "lattices_flagged_unstable": flagged[mode],
             "lattices_flagged_by_mode": flagged,
             "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                          "frac": achieved / hbm_peak, "traffic": BATCH_TRAFFIC_BYTES_PER_NODE.get((k, nt, vpt)),
                          "effective_gbs": glups / world * BYTES_PER_NODE["f32"],
                          "effective_frac": glups / world * BYTES_PER_NODE["f32"] / hbm_peak}}
        if r["roofline"]["traffic"] is not None:
            r["roofline"]["traffic"] *= ntot
        if which == "stable":
            r["selection"] = (f"Riemann states restricted to {BATCH_ENTROPY_BAND[0]} <= (s - s0)/c_p <= "
                              f"{BATCH_ENTROPY_BAND[1]} on both sides and exact-solution star velocity |u*| below "
                              f"the linear stability limit of the lattice's s_e (rejection sampling of the same "
                              f"draw)")
            r["_rho_small"] = rho_small
            r["_batch"] = bat
            out = r
        else:
            r["note"] = ("unrestricted draw: most lattices blow up (scheme instability at entropies above "
                         "about 0.1 c_p); the rate includes NaN arithmetic on the flagged lattices")
            out["literal_draw"] = r
    return out


SWEEP_WINDOW = 64          # lattice steps; every lattice is still unflagged (first flags: FP32 96, FP64 200)
SWEEP_CHECKPOINTS = (16, 32, 48, 64)
SWEEP_SUBSAMPLE = 16       # every 16th node: the 2^16-node subsampled copy of a 2^20-node lattice


def run_sweep(args, lbm, torch):
    """Precision and scale sweep: 64 lattices of 2^20 nodes, steepening wave of amplitude 0.2, lattice b
    with s_e = (1.2, 1.6, 1.9)[b mod 3], FP32 shifted populations and FP64, autotuned.

    The amplitude-0.2 wave is linearly unstable for every one of these rates (|u| = 0.2 lambda; the
    stability tests pin the radius above 1.03), so every lattice blows up from rounding noise (first
    flags after 96 steps in FP32, 200 in FP64) and the configured 10 000 steps would only propagate NaN.
    The sweep is therefore measured over the window of the first 64 steps, on live lattices: each timed
    region re-initialises the state (untimed) and advances exactly 64 steps. Reported per precision: the
    GLUPS of the window, the lattices flagged at its end (0), the per-step drift of the mass and
    momentum sums, |sum(64) - sum(0)| / (64 sum rho(0)), and the FP32-against-FP64 L1(rho) on the
    2^16-node subsample (every 16th node of all 64 lattices) at steps 16, 32, 48, 64; the L1(rho)
    against the oracle at step 64 is computed in the CPU leg from the subsamples kept here."""
    from paper_1802_02369_gb300 import workloads as W

    B, N, T = 64, 1 << 20, SWEEP_WINDOW
    s_vals = np.array([1.2, 1.6, 1.9])
    s_e = s_vals[np.arange(B) % 3]
    rho, u, p = W.steepening_wave(N, 0.2, W.reference_pressure())
    fields = [torch.from_numpy(np.tile(x, B)).cuda() for x in (rho, u, p)]
    out, snaps = {}, {}
    for prec in ("f32", "f64"):
        lat = lbm.Lattice(np.full(B, N), s_e=s_e, precision=prec)
        lat.set_state(*fields)
        k, nt, v = lat.autotune(1)
        times = []
        while True:
            lat.set_state(*fields)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(lat.stream)
            lat.step(T)
            e1.record(lat.stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            if sum(times) >= MIN_TIMED_MS or len(times) >= MAX_REPEATS:
                break
        ms = float(np.median(times))
        _, flags, _ = lat.diagnostics()
        flagged_timed = int((flags != 0).sum())
        # Untimed rerun of the window with read-backs: sums at 0 and T, subsampled rho at the checkpoints.
        lat.set_state(*fields)
        s0, _, _ = lat.diagnostics()
        snaps[prec] = {}
        done = 0
        for c in SWEEP_CHECKPOINTS:
            lat.step(c - done)
            done = c
            r = lat.moments(device=True)[0].view(B, N)[:, ::SWEEP_SUBSAMPLE].contiguous()
            snaps[prec][c] = r
        s1, flags, _ = lat.diagnostics()
        lat.close()
        drift = np.abs(s1[:, :2] - s0[:, :2]).max(axis=0) / (T * s0[:, 0].max())
        out[prec] = {"value": B * N * T / (ms * 1e-3) / 1e9, "unit": UNIT, "lattices": B, "N": N, "steps": T,
                     "timed_regions": len(times), "steps_per_launch": k, "block_threads": nt, "nodes_per_thread": v,
                     "mass_drift_per_step": float(drift[0]), "momentum_drift_per_step": float(drift[1]),
                     "lattices_flagged_unstable": max(flagged_timed, int((flags != 0).sum()))}
    del fields
    growth = {}
    for c in SWEEP_CHECKPOINTS:
        growth[str(c)] = float(torch.mean(torch.abs(snaps["f32"][c] - snaps["f64"][c])).item())
    out["l1_rho_f32_vs_f64"] = growth
    out["window"] = (f"first {T} of the configured 10000 steps: the amplitude-0.2 wave is linearly unstable at "
                     f"every s_e of the sweep and blows up from rounding noise after 96 (FP32) / 200 (FP64) steps")
    out["_subsample"] = {prec: {b: snaps[prec][T][b].cpu().numpy() for b in range(3)} for prec in snaps}
    del snaps
    torch.cuda.empty_cache()
    return out


def run_df(args, lbm, torch, N: int, sm_clock_mhz: float):
    """The benchmark workload with FP64 storage and the time step in double-float on the FP32 pipes
    (precision LBM_F64_DF), autotuned, beside the native FP64 figure."""
    rho, u, p = workload_fields(N)
    d = [torch.from_numpy(x).cuda() for x in (rho, u, p)]
    lat = lbm.Lattice(N, s_e=S_E, precision="f64df")
    lat.set_state(*d)
    if args.df_config:
        lat.set_config(*[int(x) for x in args.df_config.split(",")])
        k, nt, v = lat.get_config()
    else:
        k, nt, v = lat.autotune(2)
    lat.set_state(*d)
    steps = max(k, (args.df_steps // k) * k)
    ms = time_device(lat, torch, steps, 3 * k, None, 1)
    _, flags, _ = lat.diagnostics()
    lat.close()
    del d
    torch.cuda.empty_cache()
    glups = N * steps / (ms * 1e-3) / 1e9
    r = {"value": glups, "unit": UNIT, "steps": steps, "steps_per_launch": k, "block_threads": nt,
         "nodes_per_thread": v, "launch_ms": ms / (steps // k), "flags": int(flags[0]),
         "arithmetic": "double-float (two FP32 numbers per value) on the FP32 pipes, FP64 storage",
         "effective_gbs": glups * BYTES_PER_NODE["f64"]}
    if DF_FP32_OPS_PER_COMPUTED is not None:
        ops = DF_FP32_OPS_PER_COMPUTED * nt * v / (nt * v - 4 * k)
        a = glups * ops / 1e3
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        pk = props.multi_processor_count * 128 * sm_clock_mhz * 1e6 / 1e12
        r["roofline"] = {"bound": "alu", "achieved": a, "peak": pk, "unit": "T FP32 op/s", "frac": a / pk,
                         "fp32_ops_per_node_update": ops,
                         "peak_kind": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x "
                                      f"{sm_clock_mhz:.0f} MHz (one operation per lane per clock)"}
    return r


def run_linear(args, lbm, torch):
    """The section 7 linear scheme (linear equilibria around u0 = 0.15, s0 = 0.2, sigma_eps = 1.5,
    no source) on a small acoustic wave, N = 2^26, autotuned, FP32 and FP64."""
    N = N_NODES
    x = 2 * np.pi * np.arange(N) / N
    rho = torch.from_numpy(1.0 + 1e-3 * np.sin(x)).cuda()
    u = torch.from_numpy(0.15 + 0.5e-3 * np.sin(x)).cuda()
    s = torch.full((N,), 0.2, dtype=torch.float64, device="cuda")
    out = {}
    for prec, steps in (("f32", 1000), ("f64", 200)):
        lat = lbm.Lattice(N, s_e=1.9, s_eps=0.5, precision=prec,
                          phys=dict(equilibria=1, u0_lin=0.15, s0_lin=0.2, source_on=0))
        lat.set_state_entropy(rho, u, s)
        k, nt, v = lat.autotune(1)
        lat.set_state_entropy(rho, u, s)
        steps = (steps // k) * k
        ms = time_device(lat, torch, steps, 3 * k, None, 1)
        lat.close()
        out[prec] = {"value": N * steps / (ms * 1e-3) / 1e9, "unit": UNIT, "steps": steps, "steps_per_launch": k,
                     "block_threads": nt, "nodes_per_thread": v}
    del rho, u, s
    torch.cuda.empty_cache()
    return out


# DRAM bytes per node and block of k steps of the persistent launch on the ragged batch, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum of one persistent launch over 25 blocks of 8 steps, on
# the batch selection at 1024 lattices, 33.8 M nodes: (20,723.5 + 20,387.7) MB / (33,783,937 x 25)),
# keyed by (k, NT, V); profiles/persistent_vs_launch_batch256.md.
BATCH_TRAFFIC_BYTES_PER_NODE = {(8, 128, 4): (20729.632512e6 + 20420.880128e6) / (33783937 * 25)}
# DRAM bytes of the backward sweep over its algorithmic bytes, from ncu (dram__bytes_read.sum +
# dram__bytes_write.sum of every recompute and adjoint-block launch between the misfit seed and the
# initial-state adjoint) on 256 x 65536 nodes (larger than L2), T = 64 (FP32, 4 reverse steps per
# launch) and T = 16 (FP64, 1; double-float, 4): 23.13 / 24, 211.78 / 216 and 35.49 / 36 B per
# differentiated node-step. The benchmark reports this ratio times its own algorithmic bytes.
ADJOINT_TRAFFIC_RATIO = {"f32": 23.13 / 24.0, "f64": 211.78 / 216.0, "f64df": 35.49 / 36.0}


def adjoint_bytes_per_node_step(word: int, k: int, T: int) -> float:
    """Algorithmic bytes per differentiated node-step of the backward sweep: per block of k reverse steps
    one adjoint-block launch (state and a(t + k) read, a(t) written: 18 words) and, for every block that
    does not start at a checkpoint, one k-step recompute launch of its starting state (12 words); a
    segment of S = round(sqrt(T)) steps holds ceil(S / k) blocks, one starting at its checkpoint."""
    S = max(1, int(round(T ** 0.5)))
    nb = -(-S // k)
    return word * (18.0 + 12.0 * (nb - 1) / nb) / k


def run_adjoint(args, lbm, torch, hbm_peak: float):
    """Gradient of sum (rho_T - rho*)^2 for 256 lattices of 65536 nodes (Gaussian density bumps,
    seed 2369; target from seed 2370), sqrt(T) checkpointing. Reported: node-steps of the
    differentiated run per second, over forward + backward. An untimed forward run first allocates the
    checkpoints (about sqrt(T) states, tens of GB), which torch's caching allocator then keeps for the
    timed run, and computes the seed once, so that torch's lazy loading of its elementwise kernels
    (about a second, once per process) stays out of the timed region too."""
    from paper_1802_02369_gb300 import workloads as W

    B, N = args.adjoint_lattices, 65536
    out = {}
    for prec, T in (("f32", args.adjoint_steps_f32), ("f64", args.adjoint_steps_f64),
                    ("f64df", args.adjoint_steps_f64)):
        base = "f64" if prec == "f64df" else prec  # the double-float leg runs with the FP64 one
        if base not in args.precisions.split(","):
            continue
        rho, u, p = W.gaussian_bumps(B, N, 2369, W.reference_pressure())
        rho_t, u_t, p_t = W.gaussian_bumps(B, N, 2370, W.reference_pressure())
        tgt_lat = lbm.Lattice(np.full(B, N), s_e=1.5, precision=prec)
        tgt_lat.set_state(rho_t.ravel(), u_t.ravel(), p_t.ravel())
        tgt_lat.step(T)
        target = tgt_lat.moments(device=True)[0]
        tgt_lat.close()
        lat = lbm.Lattice(np.full(B, N), s_e=1.5, precision=prec)
        adj_k = lat.get_adjoint_config()
        d = [torch.from_numpy(x.ravel()).cuda() for x in (rho, u, p)]
        lat.set_state(*d)
        lat.adjoint_forward(T)   # warm-up: allocates the checkpoints and loads the seed's torch kernels
        seed = 2.0 * (lat.moments(device=True)[0] - target)
        lat.adjoint_release()
        del seed
        lat.set_state(*d)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.adjoint_forward(T)
        rho_T = lat.moments(device=True)[0]
        seed = 2.0 * (rho_T - target)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(lat.stream)
        g_rho, g_u, g_rates, _ = lat.adjoint_backward(seed, device=True)
        e1.record(lat.stream)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        bwd_s = e0.elapsed_time(e1) * 1e-3
        lat.adjoint_release()
        lat.close()
        del d, target, rho_T, seed, g_rho, g_u
        torch.cuda.empty_cache()
        word = 4 if prec == "f32" else 8
        bpn = adjoint_bytes_per_node_step(word, adj_k, T)
        ach = B * N * T * bpn / bwd_s / 1e9
        out[prec] = {"value": B * N * T / dt / 1e9, "unit": "GLUPS (differentiated node-steps / s)", "T": T,
                     "lattices": B, "N": N, "seconds": dt, "backward_seconds": bwd_s,
                     "checkpoint_segment": int(round(T ** 0.5)), "reverse_steps_per_launch": adj_k,
                     "dL_dse_first_lattice": float(g_rates[0, 0]),
                     "roofline": {"bound": "hbm", "scope": "backward sweep (recompute launches + adjoint block "
                                                            "launches), CUDA events on the library stream",
                                  "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                                  "algorithmic_bytes_per_node_step": bpn,
                                  "traffic": ADJOINT_TRAFFIC_RATIO[prec] * bpn * B * N * T,
                                  "traffic_unit": "bytes of the whole backward sweep (ncu ratio x algorithmic)",
                                  "note": "arithmetic-bound in practice (ncu: DRAM well below peak)"}}
    return out


# Finite-difference comparison solver (section 9) on the same steepening wave: dx = 1, nu = the
# lattice Boltzmann viscosity at s_e = 1.2 in lattice units (sigma_e lambda dx = 1/3), dt = 1 (one
# lattice time step), source on. Bytes per node per launch: three words read and written.
FD_NU = 1.0 / S_E - 0.5
FD_DT = 1.0
FD_BYTES_PER_NODE = {"f32": 24, "f64": 48}
# Arithmetic per computed node-step of the finite-difference kernel (halo included). FP64: executed on the
# FP64 pipe, from ncu at N = 2^23, (4, 256, 1): (2 DFMA + DADD + DMUL) = 2,736,388,096 over 33,826 x 256 x 4
# node-steps = 79.0 (log1p and expm1 run in double-float on the FP32 pipes). FP32 runs two nodes
# per paired lane, which ncu's per-opcode counters do not split out; counted from the source (fma = 2):
# 57 for the nodal quantities (series log1p 20 and expm1 13 included) + 37 for the update = 94. Per
# output node-update this is multiplied by the tile's computed / stored nodes, NT V / (NT V - 2K).
FD_FLOPS_PER_COMPUTED = {"f64": 2736388096 / 34637824, "f32": 94.0}


def run_fd(args, lbm, torch, N: int, hbm_peak: float, sm_clock_mhz: float):
    """Forward-Euler centred finite differences of eq. (NS-rho-J-zeta) on the benchmark wave,
    FP64 and FP32, autotuned (or the fixed --fd-config)."""
    rho, u, p = workload_fields(N)
    d_rho, d_u = torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda()
    d_s = torch.zeros(N, dtype=torch.float64, device="cuda")   # adiabatic: p = p0 rho^gamma, s = 0
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    out = {}
    for prec in args.precisions.split(","):
        steps = args.fd_steps_f64 if prec == "f64" else args.fd_steps_f32
        g = lbm.FdGrid(N, 1.0, FD_DT, FD_NU, precision=prec)
        g.set_state(d_rho, d_u, d_s)
        if args.fd_config:
            g.set_config(*[int(x) for x in args.fd_config.split(",")])
            k, nt, v = g.get_config()
        else:
            k, nt, v = g.autotune(2)
        g.set_state(d_rho, d_u, d_s)
        steps = max(k, (steps // k) * k)
        ms = time_device(g, torch, steps, 3 * k, None, 1)
        _, flags, _ = g.diagnostics()
        g.close()
        glups = N * steps / (ms * 1e-3) / 1e9
        launch_ms = ms / (steps // k)
        achieved = N * FD_BYTES_PER_NODE[prec] / (launch_ms * 1e-3) / 1e9
        r = {"value": glups, "unit": UNIT, "steps": steps, "steps_per_launch": k, "block_threads": nt,
             "nodes_per_thread": v, "launch_ms": launch_ms, "flags": int(flags),
             "roofline_hbm": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                              "frac": achieved / hbm_peak,
                              "effective_gbs": glups * FD_BYTES_PER_NODE[prec],
                              "algorithmic_bytes_per_launch": N * FD_BYTES_PER_NODE[prec]}}
        fl = FD_FLOPS_PER_COMPUTED[prec] * nt * v / (nt * v - 2 * k)
        a = glups * fl / 1e3
        pk = props.multi_processor_count * FLOPS_PER_SM_CLOCK[prec] * sm_clock_mhz * 1e6 / 1e12
        r["roofline"] = {"bound": "alu", "achieved": a, "peak": pk, "unit": "TFLOP/s", "frac": a / pk,
                         "flops_per_node_update": fl,
                         "peak_kind": f"derived: {props.multi_processor_count} SMs x {FLOPS_PER_SM_CLOCK[prec]:.0f} "
                                      f"{prec.upper()} flops/clock x {sm_clock_mhz:.0f} MHz"}
        out[prec] = r
    del d_rho, d_u, d_s
    torch.cuda.empty_cache()
    return out


# Single-distribution D1Q3 schemes (sections 2 and 4) on N = 2^26 nodes, lambda = 1: the fluid scheme
# on the steepening wave (rho = 1 + 0.1 sin, J = rho 0.1 sin, s_e = 1.2, isentropic p0 (rho)^1.4) and
# the advection-diffusion scheme on zeta = 1 + 0.1 sin (u0 = 0.1, alpha = 0, s_psi = 1.2, s_eps = 1.5).
# Bytes per node per launch: three populations read and written.
D1Q3_BYTES_PER_NODE = {"f32": 24, "f64": 48}
# Arithmetic per computed node-step (halo included), keyed by (scheme, precision). FP64: executed on the
# FP64 pipe (2 DFMA + DADD + DMUL) from ncu at N = 2^23, (16, 256, 4), over 8457 x 1024 x 16 node-steps:
# fluid 5,265,260,544 / 138,559,488 = 38.0 (its log1p and expm1 in double-float on the FP32 pipes),
# advection-diffusion 3,048,308,736 / 138,559,488 = 22.0.
# FP32 runs on paired lanes, which ncu's per-opcode counters do not split out; counted from the source
# instead (fma = 2): fluid 60 (moments 5, 1/(1+r) 2, series log1p 20 and expm1 13, equilibrium and
# relaxation 11, M^-1 9), advection-diffusion 22 (the FP64 count).
D1Q3_FLOPS_PER_COMPUTED = {("fluid", "f64"): 5265260544 / 138559488, ("advection_diffusion", "f64"): 22.0,
                           ("fluid", "f32"): 60.0, ("advection_diffusion", "f32"): 22.0}


def run_d1q3(args, lbm, torch, N: int, hbm_peak: float, sm_clock_mhz: float):
    x = 2 * np.pi * np.arange(N) / N
    rho = torch.from_numpy(1.0 + 0.1 * np.sin(x)).cuda()
    J = rho * torch.from_numpy(0.1 * np.sin(x)).cuda()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    out = {}
    for scheme in ("fluid", "advection_diffusion"):
        out[scheme] = {}
        for prec in args.precisions.split(","):
            steps = args.d1q3_steps_f64 if prec == "f64" else args.d1q3_steps_f32
            if scheme == "fluid":
                lat = lbm.D1q3Lattice(N, "fluid", s_e=S_E, precision=prec)
                state = (rho, J)
            else:
                lat = lbm.D1q3Lattice(N, "advection_diffusion", u0=0.1, alpha=0.0, s_psi=1.2, precision=prec)
                state = (rho,)
            lat.set_state(*state)
            if args.d1q3_config:
                lat.set_config(*[int(v) for v in args.d1q3_config.split(",")])
                k, nt, v = lat.get_config()
            else:
                k, nt, v = lat.autotune(2)
            lat.set_state(*state)
            steps = max(k, (steps // k) * k)
            ms = time_device(lat, torch, steps, 3 * k, None, 1)
            _, flags, _ = lat.sums()
            lat.close()
            glups = N * steps / (ms * 1e-3) / 1e9
            launch_ms = ms / (steps // k)
            achieved = N * D1Q3_BYTES_PER_NODE[prec] / (launch_ms * 1e-3) / 1e9
            r = {"value": glups, "unit": UNIT, "steps": steps, "steps_per_launch": k, "block_threads": nt,
                 "nodes_per_thread": v, "launch_ms": launch_ms, "flags": int(flags),
                 "roofline_hbm": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                                  "frac": achieved / hbm_peak, "effective_gbs": glups * D1Q3_BYTES_PER_NODE[prec],
                                  "effective_frac": glups * D1Q3_BYTES_PER_NODE[prec] / hbm_peak,
                                  "algorithmic_bytes_per_launch": N * D1Q3_BYTES_PER_NODE[prec]}}
            fl = D1Q3_FLOPS_PER_COMPUTED.get((scheme, prec))
            if fl is not None:
                fl = fl * nt * v / (nt * v - 2 * k)
                a = glups * fl / 1e3
                pk = props.multi_processor_count * FLOPS_PER_SM_CLOCK[prec] * sm_clock_mhz * 1e6 / 1e12
                r["roofline"] = {"bound": "alu", "achieved": a, "peak": pk, "unit": "TFLOP/s", "frac": a / pk,
                                 "flops_per_node_update": fl,
                                 "peak_kind": f"derived: {props.multi_processor_count} SMs x "
                                              f"{FLOPS_PER_SM_CLOCK[prec]:.0f} {prec.upper()} flops/clock x "
                                              f"{sm_clock_mhz:.0f} MHz"}
            out[scheme][prec] = r
    del rho, J
    torch.cuda.empty_cache()
    return out


# The two-dimensional D2Q9-D2Q5 scheme: 14 populations read and written once per node-update.
D2_BYTES_PER_NODE = {"f32": 14 * 2 * 4, "f64": 14 * 2 * 8, "f64df": 14 * 2 * 8}
# DRAM bytes per node-update of its step kernel from ncu (dram__bytes_read.sum + dram__bytes_write.sum of
# one launch on a 4096 x 4096 lattice, scaled by the node count): profiles/step2d_kernel_4096.md.
D2_TRAFFIC_BYTES_PER_NODE = {"f32": (942.33984e6 + 895.275264e6) / 16777216,
                             "f64": (1882.121984e6 + 1831.835136e6) / 16777216}


def run_2d(args, lbm, torch, side: int, hbm_peak: float):
    """The two-dimensional scheme on a periodic side x side lattice of smooth seeded waves (density,
    velocity and entropy modes of relative amplitude 0.05), s_e = 1.2: one launch per step, timed on
    the device as the other legs."""
    from paper_1802_02369_gb300 import workloads as W

    fields = W.waves_2d(side, side, 2369, amp=0.05)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields]
    del fields
    N = side * side
    out = {"lattice": f"{side} x {side} periodic", "workload": "seeded smooth waves, amplitude 0.05, s_e = 1.2, "
                                                                "beta = 9/2"}
    precs = args.precisions.split(",")
    if "f64" in precs:
        precs.append("f64df")  # FP64 planes, double-float arithmetic: FP64 accuracy on the FP32 pipes
    for prec in precs:
        steps = {"f64": args.d2_steps_f64, "f64df": args.d2_steps_f64df}.get(prec, args.d2_steps_f32)
        lat = lbm.Lattice2D(side, side, precision=prec, s_e=S_E)
        lat.set_state(*d)
        ms = time_device(lat, torch, steps, 3, None, 1)
        rho = lat.fields(device=True)[0]
        finite = bool(torch.isfinite(rho).all().item())
        del rho
        lat.close()
        glups = N * steps / (ms * 1e-3) / 1e9
        launch_ms = ms / steps
        achieved = N * D2_BYTES_PER_NODE[prec] / (launch_ms * 1e-3) / 1e9
        tb = D2_TRAFFIC_BYTES_PER_NODE.get(prec)
        out[prec] = {"value": glups, "unit": UNIT, "steps": steps, "steps_per_launch": 1, "launch_ms": launch_ms,
                     "finite": finite,
                     "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                                  "frac": achieved / hbm_peak, "traffic": None if tb is None else tb * N,
                                  "algorithmic_bytes_per_launch": N * D2_BYTES_PER_NODE[prec]}}
        torch.cuda.empty_cache()
    del d
    torch.cuda.empty_cache()
    return out


# Algorithmic bytes of one node update of the three-dimensional scheme: 26 populations read and 26
# written.
D3_BYTES_PER_NODE = {"f32": 26 * 2 * 4, "f64": 26 * 2 * 8, "f64df": 26 * 2 * 8}
# DRAM bytes per node per launch, read + write, from one ncu capture of step3d_kernel each: FP32
# (shared-buffer variant) on a 128^3 lattice, FP64 on 96^3 (both states above L2), scaled by the nodes.
D3_TRAFFIC_BYTES_PER_NODE = {"f32": (222.251008e6 + 177.752576e6) / 128 ** 3,
                             "f64": (188.406528e6 + 146.721792e6) / 96 ** 3}


def run_3d(args, lbm, torch, side: int, hbm_peak: float):
    """The three-dimensional scheme on a periodic side^3 lattice of smooth seeded waves (density and
    velocity modes of relative amplitude 0.05, entropy 0.0125 c_p), s_e = 1.2: one launch per step,
    timed on the device as the other legs."""
    from paper_1802_02369_gb300 import workloads as W

    fields = W.waves_3d(side, side, side, 2369, amp=0.05)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields]
    del fields
    N = side ** 3
    out = {"lattice": f"{side} x {side} x {side} periodic",
           "workload": "seeded smooth waves, amplitude 0.05, s_e = 1.2, beta = 9"}
    precs = args.precisions.split(",")
    if "f64" in precs:
        precs.append("f64df")  # FP64 planes, double-float arithmetic: FP64 accuracy on the FP32 pipes
    for prec in precs:
        steps = {"f64": args.d3_steps_f64, "f64df": args.d3_steps_f64df}.get(prec, args.d3_steps_f32)
        lat = lbm.Lattice3D(side, side, side, precision=prec, s_e=S_E)
        if args.d3_config:
            ty, zc, keep = (int(v) for v in args.d3_config.split(","))
            lat.set_config(ty=ty, zc=zc, keep=keep)
        lat.set_state(*d)
        ms = time_device(lat, torch, steps, 3, None, 1)
        rho = lat.fields(device=True)[0]
        finite = bool(torch.isfinite(rho).all().item())
        del rho
        cfg = lat.get_config()
        lat.close()
        glups = N * steps / (ms * 1e-3) / 1e9
        launch_ms = ms / steps
        achieved = N * D3_BYTES_PER_NODE[prec] / (launch_ms * 1e-3) / 1e9
        tb = D3_TRAFFIC_BYTES_PER_NODE.get(prec)
        out[prec] = {"value": glups, "unit": UNIT, "steps": steps, "steps_per_launch": 1, "launch_ms": launch_ms,
                     "finite": finite, "tile_rows": cfg[0], "planes_per_cta": cfg[1] or "auto", "keep": cfg[2],
                     "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                                  "frac": achieved / hbm_peak, "traffic": None if tb is None else tb * N,
                                  "algorithmic_bytes_per_launch": N * D3_BYTES_PER_NODE[prec]}}
        torch.cuda.empty_cache()
    del d
    torch.cuda.empty_cache()
    return out


def oracle_accuracy(O, batched, sweep, cores: int):
    """The CPU leg's accuracy statements (the oracle as it stands, on bounded samples): L1(rho) of the
    ragged batch's shortest lattices after the timed 2000 steps, and of the precision sweep's three rates
    on the 2^16-node subsample at the end of its window, against the FP64 oracle on the same inputs."""
    if batched is not None and "_rho_small" in batched:
        bat = batched["_batch"]
        l1 = {}
        for b, got in batched["_rho_small"].items():
            phb = O.default_phys(bc=int(bat.bc[b]))
            r, u, p = bat.lattice(b)
            fd = O.run(phb, O.coupled_rates(bat.s_e[b]), O.init(phb, r, u, p=p), batched["steps"], cores)
            _, oflag = O.diagnostics(phb, fd)
            l1[str(b)] = {"length": int(bat.lengths[b]), "bc": int(bat.bc[b]), "s_e": float(bat.s_e[b]),
                          "oracle_flags": oflag,
                          "l1_rho": float(np.mean(np.abs(got - O.moments(phb, fd)[:, 0])) / phb.rho0)}
        batched["accuracy_vs_oracle"] = {
            "metric": "L1(rho) = mean |rho_gpu - rho_oracle| / rho0 after the timed steps (bound 1e-4)",
            "lattices": l1, "max": max(v["l1_rho"] for v in l1.values())}
    if sweep is not None and "_subsample" in sweep:
        from paper_1802_02369_gb300 import workloads as W

        N = sweep["f32"]["N"]
        T = sweep["f32"]["steps"]
        rho, u, p = W.steepening_wave(N, 0.2, W.reference_pressure())
        ph = O.default_phys()
        acc = {"f32": {}, "f64": {}}
        for b, s_e in enumerate((1.2, 1.6, 1.9)):
            fd = O.run(ph, O.coupled_rates(s_e), O.init(ph, rho, u, p=p), T, cores)
            ref = O.moments(ph, fd)[::SWEEP_SUBSAMPLE, 0]
            for prec in ("f32", "f64"):
                acc[prec][str(s_e)] = float(np.mean(np.abs(sweep["_subsample"][prec][b] - ref)) / ph.rho0)
        sweep["l1_rho_vs_oracle"] = {"step": T, "subsample": f"every {SWEEP_SUBSAMPLE}th node of lattices 0, 1, 2",
                                     "by_precision_and_s_e": acc}


def run_ours(args, rank: int, world: int, local: int, dist):
    import torch

    from paper_1802_02369_gb300 import build, lbm

    torch.cuda.set_device(local)
    build.build()
    hbm_peak, peak_kind = measured_peaks()
    if args.batched_only:
        res = run_batched(args, lbm, torch, hbm_peak, world)
        for key in [x for x in res if x.startswith("_")]:
            res.pop(key)
        if rank == 0:
            print(json.dumps({"profiling_case": True, "solver": "ragged batch", "results": res}), flush=True)
        return
    if args.df_only:
        with ClockSampler(local) as clk:
            res = run_df(args, lbm, torch, args.nodes, 2070.0)
        if rank == 0:
            print(json.dumps({"profiling_case": True, "solver": "double-float", "nodes": args.nodes, "results": res,
                              "clocks": clk.summary()}), flush=True)
        return
    if args.adjoint_only:
        res = run_adjoint(args, lbm, torch, hbm_peak)
        if rank == 0:
            print(json.dumps({"profiling_case": True, "solver": "adjoint", "results": res}), flush=True)
        return
    if args.d1q3_only:
        with ClockSampler(local) as clk:
            res = run_d1q3(args, lbm, torch, args.nodes, hbm_peak, 2070.0)
        if rank == 0:
            print(json.dumps({"profiling_case": True, "solver": "D1Q3 schemes", "nodes": args.nodes,
                              "results": res, "clocks": clk.summary()}), flush=True)
        return
    if args.d2_only:
        with ClockSampler(local) as clk:
            res = run_2d(args, lbm, torch, args.d2_side, hbm_peak)
        if rank == 0:
            print(json.dumps({"profiling_case": True, "solver": "two-dimensional D2Q9-D2Q5", "results": res,
                              "clocks": clk.summary()}), flush=True)
        return
    if args.d3_only:
        with ClockSampler(local) as clk:
            res = run_3d(args, lbm, torch, args.d3_side, hbm_peak)
        if rank == 0:
            print(json.dumps({"profiling_case": True, "solver": "three-dimensional D3Q19-D3Q7", "results": res,
                              "clocks": clk.summary()}), flush=True)
        return
    if args.fd_only:
        with ClockSampler(local) as clk:
            fd = run_fd(args, lbm, torch, args.nodes, hbm_peak, 2070.0)
        if rank == 0:
            print(json.dumps({"profiling_case": True, "solver": "finite differences", "nodes": args.nodes,
                              "results": fd, "clocks": clk.summary()}), flush=True)
        return
    NN = args.nodes
    rho, u, p = workload_fields(NN)
    d_rho, d_u, d_p = (torch.from_numpy(x).cuda() for x in (rho, u, p))
    results = {}
    precs = args.precisions.split(",")
    with ClockSampler(local) as clk:
        for prec in precs:
            lat = lbm.Lattice(NN, s_e=S_E, precision=prec)
            lat.set_state(d_rho, d_u, d_p)
            if args.config:
                lat.set_config(*[int(x) for x in args.config.split(",")])
                k, nt, vpt = lat.get_config()
            else:
                k, nt, vpt = lat.autotune(2)
            lat.set_state(d_rho, d_u, d_p)
            # Exactly --steps lattice steps per timed region (FP64, about 60x slower, at most 200) after
            # exactly --warmup (at least 3) untimed ones; lbm_step runs a shorter last launch for a
            # remainder of the steps per launch.
            steps = args.steps if prec == "f32" else max(1, min(args.steps, 200))
            warm = max(args.warmup, 3)
            times = time_device_repeats(lat, torch, steps, warm, dist, world)
            ms = float(np.median(times))
            launches = (steps + k - 1) // k                     # per timed region
            glups = world * NN * steps / (ms * 1e-3) / 1e9
            launch_ms = ms / launches
            # Every launch, whatever its depth, reads and writes the state once.
            alg_bytes = NN * BYTES_PER_NODE[prec] * launches
            achieved = alg_bytes / (ms * 1e-3) / 1e9
            sums, flags, rc = lat.diagnostics()
            results[prec] = dict(value=glups, ms_per_step=ms / steps, steps=steps, warmup=warm, k=k, block_threads=nt,
                                 nodes_per_thread=vpt, launches=launches, launch_ms=launch_ms, achieved=achieved,
                                 repeats=len(times), region_ms=[round(t, 4) for t in times],
                                 effective_gbs=glups / world * BYTES_PER_NODE[prec], flags=int(flags[0]))
            lat.close()
            torch.cuda.empty_cache()
    clocks = clk.summary()
    if NN != N_NODES or len(precs) != 2:
        if rank == 0:
            print(json.dumps({"profiling_case": True, "nodes": NN, "results": results, "clocks": clocks}), flush=True)
        return

    # End to end through the C-ABI with pinned host buffers: state in, K steps, (rho, J, zeta) out.
    r32 = results["f32"]
    K = r32["steps"]
    h = [torch.from_numpy(x).pin_memory() for x in (rho, u, p)]
    outs = [torch.empty(N_NODES, dtype=torch.float64).pin_memory() for _ in range(3)]
    lat = lbm.Lattice(N_NODES, s_e=S_E, precision="f32")
    lat.set_config(r32["k"], r32["block_threads"], r32["nodes_per_thread"])
    lat.set_state(*h)
    lat.step(r32["warmup"])
    lat.moments(out=outs + [None, None, None])
    e2e_times = []
    while True:  # regions of: host state in, exactly K steps, (rho, J, zeta) back to host memory
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        lat.set_state(*h)
        lat.step(K)
        lat.moments(out=outs + [None, None, None])
        torch.cuda.synchronize()
        e2e_times.append(max_over_ranks(time.perf_counter() - t0, dist))
        if dist is not None:
            dist.barrier()
        if sum(e2e_times) >= MIN_TIMED_MS * 1e-3 or len(e2e_times) >= MAX_REPEATS:
            break
    e2e_s = float(np.median(e2e_times))
    lat.close()
    e2e = {"value": world * N_NODES * K / e2e_s / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": 3 * 8 * N_NODES / K, "d2h_bytes_per_step": 3 * 8 * N_NODES / K,
           "timed_regions": len(e2e_times), "region_s_median": e2e_s,
           "path": "lbm_set_state from pinned host arrays, lbm_step(K), lbm_moments into pinned host arrays"}

    batched = None if args.no_batched else run_batched(args, lbm, torch, hbm_peak, world)
    linear = None if args.no_linear else run_linear(args, lbm, torch)
    sweep = None if args.no_sweep else run_sweep(args, lbm, torch)
    dfl = None if args.no_df else run_df(args, lbm, torch, N_NODES, clocks.get("sm_max_mhz") or 2070.0)
    adjoint = None if args.no_adjoint else run_adjoint(args, lbm, torch, hbm_peak)
    fdiff = None if args.no_fd else run_fd(args, lbm, torch, N_NODES, hbm_peak, clocks.get("sm_max_mhz") or 2070.0)
    d1q3 = None if args.no_d1q3 else run_d1q3(args, lbm, torch, N_NODES, hbm_peak, clocks.get("sm_max_mhz") or 2070.0)
    two_d = None if args.no_2d else run_2d(args, lbm, torch, args.d2_side, hbm_peak)
    three_d = None if args.no_3d else run_3d(args, lbm, torch, args.d3_side, hbm_peak)

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle as O

        O.build()
        cores = os.cpu_count() or 1
        g, st, dt = cpu_oracle_rate(N_SAMPLE, 15.0, cores)
        g1, st1, dt1 = cpu_oracle_rate(1 << 18, 4.0, 1)
        cpu = {"value": g, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first 2^22 nodes of the workload (periodic), {st} steps, {dt:.1f} s, FP64",
               "single_core": {"value": g1, "unit": UNIT, "cores": 1,
                               "sample": f"first 2^18 nodes (periodic), {st1} steps, {dt1:.1f} s, FP64"}}
        oracle_accuracy(O, batched, sweep, cores)
    for leg in (batched, sweep):   # host-side samples kept for the oracle comparison only
        if leg is not None:
            for key in [x for x in leg if x.startswith("_")]:
                leg.pop(key)

    props = torch.cuda.get_device_properties(local)
    sm_clock_mhz = clocks.get("sm_max_mhz") or 2070.0

    def roof_alu(r, prec):
        # Both precisions count the method's node update as the FP32 kernel implements it (110 flops);
        # for FP64 the executed count (CUDA's log1p / expm1 internals and correctly rounded reciprocals
        # included) is reported beside it.
        tb = TRAFFIC_BYTES_PER_NODE.get((prec, r["k"], r["block_threads"], r["nodes_per_thread"]))
        achieved = r["value"] / world * METHOD_FLOPS_PER_NODE / 1e3          # TFLOP/s
        peak = props.multi_processor_count * FLOPS_PER_SM_CLOCK[prec] * sm_clock_mhz * 1e6 / 1e12
        out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
               "traffic": None if tb is None else tb * N_NODES, "flops_per_node_update": METHOD_FLOPS_PER_NODE,
               "peak_kind": f"derived: {props.multi_processor_count} SMs x {FLOPS_PER_SM_CLOCK[prec]:.0f} "
                            f"{prec.upper()} flops/clock x {sm_clock_mhz:.0f} MHz"}
        if prec == "f64":
            ex = r["value"] / world * FLOPS_PER_NODE["f64"] / 1e3
            out["executed_flops_per_node_update"] = FLOPS_PER_NODE["f64"]
            out["executed_achieved"] = ex
            out["executed_frac"] = ex / peak
        return out

    def roof_lane_ops(r):
        # FMA-pipe view of the FP32 kernel: every add, multiply and fused multiply-add is one lane
        # operation, 128 per SM per clock; halo and ghost recomputation included (computed / stored
        # nodes of a tile).
        nt, v = r["block_threads"], r["nodes_per_thread"]
        ops = LANE_OPS_PER_NODE_F32 * nt * v / (tile_span_f32(nt, v) - 4 * r["k"])
        achieved = r["value"] / world * ops / 1e3
        peak = props.multi_processor_count * 128 * sm_clock_mhz * 1e6 / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP32 lane-op/s",
                "frac": achieved / peak, "lane_ops_per_node_update": ops,
                "peak_kind": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x {sm_clock_mhz:.0f} MHz"}

    def roof(r, prec):
        tb = TRAFFIC_BYTES_PER_NODE.get((prec, r["k"], r["block_threads"], r["nodes_per_thread"]))
        return {"bound": "hbm", "achieved": r["achieved"], "peak": hbm_peak, "unit": "GB/s",
                "frac": r["achieved"] / hbm_peak, "traffic": None if tb is None else tb * N_NODES,
                "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": N_NODES * BYTES_PER_NODE[prec],
                "steps_per_launch": r["k"], "launch_ms": r["launch_ms"],
                "effective_gbs": r["effective_gbs"], "effective_frac": r["effective_gbs"] / hbm_peak}

    f32, f64 = results["f32"], results["f64"]
    line = {"metric": METRIC, "value": f32["value"], "unit": UNIT, "n_gpus": world, "steps": f32["steps"],
            "warmup": f32["warmup"], "ms_per_step": f32["ms_per_step"], "higher_is_better": True,
            "timed_regions": f32["repeats"], "region_ms": f32["region_ms"],
            "timing": f"median over {f32['repeats']} timed regions of exactly {f32['steps']} lattice steps each "
                      f"(CUDA events, barrier and synchronize on both sides, max over ranks), repeated until "
                      f"{MIN_TIMED_MS:.0f} ms",
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N_NODES, "precision": "f32 shifted populations",
                       "steps_per_launch": f32["k"], "block_threads": f32["block_threads"],
                       "nodes_per_thread": f32["nodes_per_thread"],
                       "l2": "inputs larger than L2 (FP32 state 1.6 GB, FP64 3.2 GB)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof_alu(f32, "f32"), "roofline_lane_ops": roof_lane_ops(f32),
            "roofline_hbm": roof(f32, "f32"),
            "fp64_double_float": dfl,
            "fp64": {"value": f64["value"], "unit": UNIT, "ms_per_step": f64["ms_per_step"], "steps": f64["steps"],
                     "timed_regions": f64["repeats"],
                     "steps_per_launch": f64["k"], "block_threads": f64["block_threads"],
                     "nodes_per_thread": f64["nodes_per_thread"], "roofline": roof_alu(f64, "f64"),
                     "roofline_hbm": roof(f64, "f64")},
            "batched_fp32": batched, "adjoint": adjoint, "linear_variant": linear,
            "finite_differences": fdiff, "d1q3_schemes": d1q3, "d2q9_d2q5": two_d, "d3q19_d3q7": three_d, "precision_sweep": sweep,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": f32["launches"],
            "gpu_launches_note": "step-kernel launches per timed region of K lattice steps (K / steps per launch, "
                                 "rounded up: a remainder runs as one shorter launch)",
            "clocks": clocks,
            "diagnostic_flags": {"f32": f32["flags"], "f64": f64["flags"]}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # Profiling of smaller cases (not the benchmark line): lattice size, precisions, fixed config.
    ap.add_argument("--nodes", type=int, default=N_NODES)
    ap.add_argument("--precisions", default="f32,f64")
    ap.add_argument("--config", default="", help="k,block_threads,nodes_per_thread instead of autotuning")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-linear", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=2000)
    ap.add_argument("--batched-lattices", type=int, default=4096)
    ap.add_argument("--batched-only", action="store_true", help="only the ragged-batch leg")
    ap.add_argument("--batched-config", default="", help="k,block_threads,nodes_per_thread of the batch")
    ap.add_argument("--adjoint-steps-f32", type=int, default=4000)
    ap.add_argument("--adjoint-steps-f64", type=int, default=4000)
    ap.add_argument("--no-fd", action="store_true")
    ap.add_argument("--fd-only", action="store_true", help="only the finite-difference leg at --nodes")
    ap.add_argument("--fd-config", default="", help="k,block_threads,nodes_per_thread of the finite-difference kernel")
    ap.add_argument("--fd-steps-f64", type=int, default=200)
    ap.add_argument("--fd-steps-f32", type=int, default=1000)
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-df", action="store_true")
    ap.add_argument("--df-only", action="store_true", help="only the double-float leg at --nodes")
    ap.add_argument("--df-config", default="", help="k,block_threads,nodes_per_thread of the double-float kernel")
    ap.add_argument("--df-steps", type=int, default=200)
    ap.add_argument("--adjoint-only", action="store_true", help="only the adjoint leg")
    ap.add_argument("--adjoint-lattices", type=int, default=256)
    ap.add_argument("--no-d1q3", action="store_true")
    ap.add_argument("--d1q3-only", action="store_true", help="only the single-distribution D1Q3 leg at --nodes")
    ap.add_argument("--d1q3-config", default="", help="k,block_threads,nodes_per_thread of the D1Q3 kernels")
    ap.add_argument("--d1q3-steps-f64", type=int, default=500)
    ap.add_argument("--d1q3-steps-f32", type=int, default=2000)
    ap.add_argument("--no-2d", action="store_true")
    ap.add_argument("--d2-only", action="store_true", help="only the two-dimensional D2Q9-D2Q5 leg")
    ap.add_argument("--d2-side", type=int, default=8192)
    ap.add_argument("--d2-steps-f32", type=int, default=200)
    ap.add_argument("--d2-steps-f64", type=int, default=20)
    ap.add_argument("--d2-steps-f64df", type=int, default=40)
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--d3-only", action="store_true", help="only the three-dimensional D3Q19-D3Q7 leg")
    ap.add_argument("--d3-side", type=int, default=256)
    ap.add_argument("--d3-steps-f32", type=int, default=100)
    ap.add_argument("--d3-steps-f64", type=int, default=10)
    ap.add_argument("--d3-steps-f64df", type=int, default=20)
    ap.add_argument("--d3-config", default="", help="ty,zc,keep of the 3-D kernel (0 / -1: default)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist_mod

        torch.cuda.set_device(local)
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    run_ours(args, rank, world, local, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
