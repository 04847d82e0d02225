#!/usr/bin/env python3
"""Benchmark of the HHS-FSI hot path: acc + gradient interactions per second.

Workload (default): Plummer sphere N = 65536, equal masses, Henon units (G = M = 1),
seed 2, eta = 0.2, top-level pivot step 2^-7, mixed precision (FP32 pair bodies on
float-float separations, FP64 state and sums).

One timed step = one top-level HHS-FSI step (Algorithm hhs-fsi on all particles: time-step
pass, partition, inter-level acc / gradient passes and kicks, FSI steps of the slow sets,
recursion into the fast sets).  The energy / momentum / angular momentum reduction (the
on-the-fly analysis) runs once at the end of the timed region, as the paper samples it on a
cadence rather than every step.  `value` = acc + gradient pair interactions evaluated in the
timed region / device time; L2 is flushed (256 MiB write) before every timed step.

Extra keys: full_pass (one acc + gradient pass over all N), fp64 (the same workload in FP64
mode: full pass and 16 hierarchical steps), energy (|dE/E| after 16 steps from the initial
state in both precisions), roofline (dominant pair kernel vs the CUDA-core peak),
cpu_baseline (the FP64 oracle on the host cores), e2e (through the C-ABI with host buffers).

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_PER_PAIR = {"acc": 20.0, "grad": 38.0, "tstep": 45.0}
SM_COUNT = 152
FP32_LANES_PER_SM = 128
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 rate
METRIC = "acc+gradient interactions/s"
UNIT = "interactions/s"
# DRAM bytes (read + write) per launch of the Newtonian kind in one 64k hierarchical step:
# ncu dram__bytes_read.sum + dram__bytes_write.sum over the step's 396 launches of that kind,
# captured on the current kernels
TRAFFIC_ACC_PLUMMER64K = 388752.0


# the bars the GPU tests hold the CUDA path to against the FP64 oracle (tests/test_gpu_parity.py)
PARITY_BARS = {
    "mixed": "a_i, g_i and a~_i within 1e-6 relative at the 99.9th percentile of the particles "
             "(every particle of plummer_64k; sampled at 262144 and 1048576); the cross pass "
             "whose every dominant slot is full, reversed, within 1e-7 x sum_j |term_ij|",
    "fp64": "a_i, g_i and a~_i within 1e-12 relative for every particle; near tight pairs "
            "(hard binaries, cross passes with every dominant slot full) g_i within 1e-12 x "
            "sum_j |m_j K(x_ji) a_ji|, the bound of an FP64 sum of those terms, which exceeds "
            "1e-12 |g_i| where the partners' terms cancel",
    "timesteps": "FP64 1e-12 relative; mixed 2e-6 at the 99.9th percentile",
    "partition, kick, drift": "bit-exact",
    "trajectories": "FP64 positions within 1e-10 of the oracle over several hierarchical steps "
                    "(N <= 2000; 16 steps at N = 1024); mixed vs FP64 |dE/E| within 2x",
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=16)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="frost", choices=["frost", "reference"])
    p.add_argument("--workload", default="plummer_64k")
    p.add_argument("--dt", type=float, default=2.0 ** -7)
    p.add_argument("--eta", type=float, default=0.2)
    p.add_argument("--fp64-steps", type=int, default=16)
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--passes-only", action="store_true",
                   help="time one full acc+gradient pass and one time-step pass and report the "
                        "time-step level histogram (workloads whose hierarchy cannot be "
                        "integrated in minutes, e.g. hard binaries without regularisation)")
    p.add_argument("--integrator", default="hhs_fsi", choices=["hhs_fsi", "hold2"],
                   help="hhs_fsi: the fourth-order method (default); hold2: the second-order HOLD "
                        "integrator of Eq. hhs2, the paper's point of comparison")
    p.add_argument("--flyby-exact", action="store_true",
                   help="exact fly-by derivative in the time-steps (first line of Eq. "
                        "dt-flyby-derivative)")
    p.add_argument("--subtree-blocks", type=int, default=0,
                   help="thread blocks (a cluster) per single-set subtree-solver launch; 0 = library default")
    p.add_argument("--subtree-max", type=int, default=0,
                   help="largest set whose hhs_fsi subtree runs in one block (0 = library default)")
    p.add_argument("--branch-streams", type=int, default=0,
                   help="0: fsi(S) of grid-level hhs_fsi calls concurrently with hhs_fsi(F) (library "
                        "default); -1: one stream")
    p.add_argument("--sym-cross", type=int, default=0,
                   help="0: the Newtonian kick_sf evaluates each S x F pair once where that fills the "
                        "GPU (library default); 1: always; -1: two one-sided passes")
    p.add_argument("--integrate", action="store_true",
                   help="integrate the workload for --steps top-level steps of --dt (or to --t-end) "
                        "with per-step hierarchy statistics, the energy, momentum and angular "
                        "momentum errors, and the time extrapolated to --t-end")
    p.add_argument("--t-end", type=float, default=None,
                   help="--integrate: the end time of the configuration (the run may stop earlier, "
                        "see --max-seconds); cluster batches: advance every cluster to t-end in one "
                        "frost_step call")
    p.add_argument("--max-seconds", type=float, default=None,
                   help="--integrate: stop after the first step that ends past this wall time")
    p.add_argument("--compare-fp64", action="store_true",
                   help="--integrate: also run the FP64 mode from the same state and compare")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


# ---------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"frost_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------------------
def oracle_sample(workload, n_sample, seed=0):
    from paper_2011_14984_gb300 import ics
    m, x, v = ics.workload(workload)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(m.size, n_sample, replace=False)).astype(np.int32)
    return m, x, v, idx


def time_oracle_pass(m, x, idx, eps_grad):
    import oracle
    t0 = time.perf_counter()
    oracle.accel_gradient(m, x, idx, idx, eps_grad)
    dt = time.perf_counter() - t0
    n = idx.size
    return 2.0 * n * (n - 1), dt  # acc + gradient interactions of the pass


def cpu_baseline(workload, seconds, n_sample=16384):
    import oracle
    m, x, v, idx = oracle_sample(workload, n_sample)
    pairs = 0.0
    elapsed = 0.0
    reps = 0
    while elapsed < seconds or reps == 0:
        p, dt = time_oracle_pass(m, x, idx, 2.0 ** -7)
        pairs += p
        elapsed += dt
        reps += 1
    return {"value": pairs / elapsed, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{reps} FP64 acc+gradient passes (same-set, a~ with eps=2^-7) over a random "
                      f"{n_sample}-particle subset of {workload}, {elapsed:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    n_sample = 8192
    m, x, v, idx = oracle_sample(args.workload, n_sample)
    for _ in range(max(args.warmup, 0)):
        time_oracle_pass(m, x, idx, args.dt)
    pairs = 0.0
    elapsed = 0.0
    for _ in range(args.steps):
        p, dt = time_oracle_pass(m, x, idx, args.dt)
        pairs += p
        elapsed += dt
    value = pairs / elapsed
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * elapsed / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "sample": f"{n_sample}-particle subset",
                       "step": "one FP64 acc+gradient pass over the subset"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{args.steps} FP64 acc+gradient passes over a random "
                                       f"{n_sample}-particle subset of {args.workload}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate_ranks(ms_total, work, world, device):
    """Whole-job numbers over replicas: the slowest rank's time and the sum of the work.
    Every rank must call this (collectives); with world == 1 the inputs come back as they are."""
    if world <= 1:
        return float(ms_total), float(work)
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_total, work], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


# ---------------------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------------------
def work_stream(dev=None):
    """The stream every measured call runs on (made current for torch too): the device's
    highest priority, so that the library's concurrent branch lanes, created at the lowest
    priority, yield to the recursion on the context stream (its critical path)."""
    import torch
    s = torch.cuda.Stream(device=dev, priority=-100)  # mapped to the greatest priority
    torch.cuda.set_stream(s)
    return s


# ---------------------------------------------------------------------------------------
def method_pairs(st):
    """acc + gradient interactions of the method's steps: the evaluated pairs, plus the
    Newtonian pairs of the second fsi(S) that reuse the stored end-of-first-fsi a^SS (exact,
    S has not moved), plus the second side of every pair of a symmetric S x F pass (one
    evaluation serves both interactions); the evaluated count alone is reported beside it."""
    return float(st["acc_pairs"] + st.get("acc_pairs_reused", 0) + st.get("acc_pairs_symmetric", 0)
                 + st["grad_pairs"] + st.get("grad_pairs_symmetric", 0))


def subtree_rate(st, fp32_peak, probe):
    """Algorithmic flop rate of the single-block subtree-solver launches (all passes of the
    small sets: Newtonian, gradient and time-step pairs at 20 / 38 / 45 flops) over their
    CUDA-event time, against the FP32 peak of the whole GPU (the launches use one SM each)."""
    ms = st["timed_ms"][3]
    pairs = st.get("subtree_pairs", [0, 0, 0])
    flops = pairs[0] * FLOPS_PER_PAIR["acc"] + pairs[1] * FLOPS_PER_PAIR["grad"] + pairs[2] * FLOPS_PER_PAIR["tstep"]
    if ms <= 0:
        return None
    tf = flops / (ms * 1e-3) / 1e12
    return {"launches": st["timed_launches"][3], "ms": ms, "pairs": list(pairs), "tflops": tf,
            "frac_of_gpu": tf / fp32_peak, "frac_of_one_sm": tf / (fp32_peak / SM_COUNT),
            "frac_of_probe": tf / max(probe["ffma_tflops"], probe["ffma2_tflops"])}


def run_frost(args):
    import torch
    import torch.distributed as dist

    from paper_2011_14984_gb300 import build as fbuild
    from paper_2011_14984_gb300 import frost as fr
    from paper_2011_14984_gb300 import ics

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    fbuild.build()
    fr.load()
    dev = torch.device("cuda", local)
    stream = work_stream(dev)

    m, x, v = ics.workload(args.workload)
    n = m.size
    E0_ref = None

    def new(prec):
        return fr.Frost(m, x, v, G=1.0, eta=args.eta, precision=prec, stream=stream.cuda_stream,
                        subtree_max=args.subtree_max, subtree_blocks=args.subtree_blocks,
                        branch_streams=args.branch_streams, sym_cross=args.sym_cross,
                        sym=fr.FROST_SYM_HARMONIC | (fr.FROST_FLYBY_EXACT if args.flyby_exact else 0),
                        integrator=fr.FROST_HOLD2 if args.integrator == "hold2" else fr.FROST_HHS_FSI)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB

    def ev():
        return torch.cuda.Event(enable_timing=True)

    # ---- timed hierarchical steps (mixed) ----
    f = new("mixed")
    tuned = f.autotune()  # launch shapes of the pair kernels, outside the timed region
    for _ in range(args.warmup):
        f.step(args.dt, 1)
    torch.cuda.synchronize()
    # the state at the start of the timed region, replayed by the event-timed pass and e2e
    xs = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    vs = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    t_start = fr.frost_get_state(f.ctx, xs.numpy(), vs.numpy())
    e_start = f.energy()

    def timed_steps(per_launch_events):
        """K steps + E/P/L once; returns (device ms, stats).  Per-launch events (for the
        roofline's kernel durations) cost host time per launch, so the headline pass runs
        without them and a second pass over the same steps takes them."""
        fr.frost_set_state(f.ctx, xs.numpy(), vs.numpy(), t_start)
        torch.cuda.synchronize()
        f.reset_stats()
        f.set_timing(per_launch_events)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        total = 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)
            a, b = ev(), ev()
            a.record(stream)
            f.step(args.dt, 1)
            b.record(stream)
            b.synchronize()
            total += a.elapsed_time(b)
        a, b = ev(), ev()
        a.record(stream)
        e_end = f.energy()
        b.record(stream)
        b.synchronize()
        ms_e = a.elapsed_time(b)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        st_ = f.stats()
        f.set_timing(False)
        return total + ms_e, ms_e, e_end, st_

    clocks = ClockSampler(local)
    clocks.start()
    t_wall0 = time.perf_counter()
    ms_total, ms_energy, e_end, st = timed_steps(False)
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    interactions = method_pairs(st)
    evaluated = float(st["acc_pairs"] + st["grad_pairs"])
    launches = st["kernel_launches"] + 3  # + the energy pass kernels
    ms_max, interactions = aggregate_ranks(ms_total, interactions, world, dev)
    value = interactions / (ms_max * 1e-3)
    ms_timed_pass, _, _, st_ev = timed_steps(True)
    assert st_ev["acc_pairs"] == st["acc_pairs"], "the event-timed pass replays the same steps"

    # measured rates of the pipes the pair passes run on (FFMA, packed FFMA2, DFMA, MUFU)
    probe = fr.frost_peak_probe(stream.cuda_stream)

    # roofline of the dominant pair kernel (largest share of kernel time)
    kinds = ["acc", "grad", "tstep"]
    kms = st_ev["timed_ms"][:3]
    dom = int(np.argmax(kms))
    kname = kinds[dom]
    achieved_tf = st_ev["timed_pairs"][dom] * FLOPS_PER_PAIR[kname] / (kms[dom] * 1e-3) / 1e12
    sm_max = (clk.get("sm_max_mhz") or peaks().get("sm_max_mhz") or 2070.0)
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    sm_med = clk.get("sm_mhz")
    default_run = (args.workload == "plummer_64k" and args.integrator == "hhs_fsi" and not args.flyby_exact
                   and args.subtree_max == 0 and args.subtree_blocks == 0 and args.branch_streams == 0
                   and args.sym_cross == 0)
    traffic = TRAFFIC_ACC_PLUMMER64K if (default_run and kname == "acc") else None
    roofline = {"bound": "alu", "kernel": f"{kname} pass (mixed, FP32 pipe)",
                "achieved": achieved_tf, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved_tf / fp32_peak, "traffic": traffic,
                "traffic_basis": ("DRAM bytes per launch of the kind, averaged over one step's launches "
                                  "(ncu capture of this workload)") if traffic else None,
                "peak_basis": f"152 SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz (max SM clock)",
                "frac_at_median_clock": (achieved_tf / (fp32_peak * sm_med / sm_max)) if sm_med else None,
                "probe": probe,
                "frac_of_probe": achieved_tf / max(probe["ffma_tflops"], probe["ffma2_tflops"]),
                "probe_basis": "frost_peak_probe on the same GPU before the timed region: the faster of "
                               "scalar and packed FP32 FMA chains at full occupancy (2 flop per FMA)",
                "flops_per_pair": FLOPS_PER_PAIR[kname],
                "launches": st_ev["timed_launches"][dom], "kernel_ms": kms[dom],
                "kernel_share": kms[dom] / max(ms_timed_pass - ms_energy, 1e-9),
                "timing": "kernel durations from per-launch CUDA events in a second pass over the same K steps (the headline pass runs without them)",
                "per_kind": {kinds[k]: {"launches": st_ev["timed_launches"][k], "ms": kms[k],
                                        "pairs": st_ev["timed_pairs"][k],
                                        "tflops": (st_ev["timed_pairs"][k] * FLOPS_PER_PAIR[kinds[k]]
                                                   / (kms[k] * 1e-3) / 1e12) if kms[k] > 0 else 0.0}
                             for k in range(3)}}
    dE_timed = abs((e_end["E"] - e_start["E"]) / e_start["E"])

    # ---- end to end through the C-ABI with host buffers: the same K steps and E/P/L ----
    xh = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    vh = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    x_np, v_np = xh.numpy(), vh.numpy()
    x_np[:] = xs.numpy()
    v_np[:] = vs.numpy()
    tt = t_start
    e2e_steps = args.steps
    f.reset_stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        fr.frost_set_state(f.ctx, x_np, v_np, tt)
        fr.frost_step(f.ctx, args.dt, 1)
        tt = fr.frost_get_state(f.ctx, x_np, v_np)
    f.energy()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    st2 = f.stats()
    e2e_value = method_pairs(st2) / e2e_s * (world if world > 1 else 1)
    f.close()

    # ---- one full acc + gradient pass (both precisions) ----
    def full_pass(prec, reps):
        g = new(prec)
        g.accel_gradient(None, None, eps_grad=args.dt)  # warm-up
        g.set_timing(True)
        g.reset_stats()
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        for _ in range(reps):
            g.accel_gradient(None, None, eps_grad=args.dt, want=("acc_tilde",))
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / reps
        s = g.stats()
        g.close()
        inter = 2.0 * n * (n - 1)
        out = {"ms": ms, "value": inter / (ms * 1e-3), "unit": UNIT}
        for k, nm in ((0, "acc"), (1, "grad")):
            if s["timed_ms"][k] > 0:
                tf = s["timed_pairs"][k] * FLOPS_PER_PAIR[nm] / (s["timed_ms"][k] * 1e-3) / 1e12
                out[f"{nm}_kernel_ms"] = s["timed_ms"][k] / max(s["timed_launches"][k], 1)
                out[f"{nm}_tflops"] = tf
                out[f"{nm}_frac"] = tf / (fp32_peak if prec == "mixed" else FP64_PEAK_TFLOPS)
                out[f"{nm}_frac_of_probe"] = tf / (max(probe["ffma_tflops"], probe["ffma2_tflops"])
                                                   if prec == "mixed" else probe["dfma_tflops"])
        return out

    fp_mixed = full_pass("mixed", 5)
    extra = {"full_pass": fp_mixed}

    # ---- FP64 mode and |dE/E| at equal steps from the initial state ----
    if not args.no_fp64:
        fp_64 = full_pass("fp64", 1)
        en = {}
        for prec in ("mixed", "fp64"):
            g = new(prec)
            E0 = g.energy()["E"]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.step(args.dt, args.fp64_steps)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            s = g.stats()
            E1 = g.energy()
            en[prec] = {"dE_over_E": abs((E1["E"] - E0) / E0), "seconds": secs,
                        "interactions_per_s": method_pairs(s) / secs,
                        "dP": float(np.linalg.norm(E1["P"])), "max_depth": s["max_depth_seen"]}
            g.close()
        extra["fp64"] = {"full_pass": fp_64, "steps": args.fp64_steps}
        extra["energy"] = {"steps": args.fp64_steps, "t_end": args.fp64_steps * args.dt, **en,
                           "mixed_speedup": en["fp64"]["seconds"] / en["mixed"]["seconds"],
                           "dE_ratio_mixed_over_fp64": en["mixed"]["dE_over_E"] / en["fp64"]["dE_over_E"]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        try:
            import oracle
            oracle.build()
            cpu = cpu_baseline(args.workload, args.cpu_seconds)
        except Exception as exc:  # the baseline is a report, never the product path
            cpu = {"value": None, "unit": UNIT, "error": str(exc)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": args.workload, "N": int(n), "eta": args.eta,
                           "dt_pivot": args.dt, "precision": "mixed (FP32 pair body, float-float "
                           "separations, FP64 state and sums)",
                           "step": "one top-level HHS-FSI step; E/P/L once per timed region",
                           "l2": "flushed before every timed step (256 MiB write)",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "subtree_max": args.subtree_max or "library default",
                           "integrator": args.integrator,
                           "branch_streams": "concurrent" if args.branch_streams >= 0 else "one stream",
                           "sym_cross": {0: "where it fills the GPU", 1: "always", -1: "off"}[max(-1, min(1, args.sym_cross))],
                           "flyby_derivative": "exact" if args.flyby_exact else "two-body"},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "steps": e2e_steps,
                        "h2d_bytes_per_step": int(2 * n * 3 * 8),
                        "d2h_bytes_per_step": int(2 * n * 3 * 8)},
                "gpu_launches": int(launches), "clocks": clk,
                "wall_s_timed_region": wall, "energy_ms": ms_energy,
                "dE_over_E_timed_run": dE_timed, "max_depth": st["max_depth_seen"],
                "autotune_waves": tuned,
                "value_evaluated": evaluated / (ms_max * 1e-3),
                "interactions": {"method": interactions, "evaluated": evaluated,
                                 "reused_acc_pairs": int(st.get("acc_pairs_reused", 0)),
                                 "symmetric_second_side_pairs": int(st.get("acc_pairs_symmetric", 0)
                                                                    + st.get("grad_pairs_symmetric", 0)),
                                 "note": "value counts the method's acc+gradient pairs; the "
                                         "reused ones are the first Newtonian pass of each "
                                         "second fsi(S), taken bit for bit from the first; "
                                         "the symmetric second side is the F-side interaction "
                                         "of an S x F pair (Newtonian or gradient) evaluated "
                                         "once for both particles, counted in method, not in "
                                         "evaluated"},
                "hhs_calls": st["hhs_calls"], "subtree_launches": st["subtree_launches"],
                "subtree_fsi_beside": int(st.get("subtree_fsi_beside", 0)),
                "subtree_ms": st_ev["timed_ms"][3],
                "subtree": subtree_rate(st_ev, fp32_peak, probe),
                "levels": {"calls": list(st["level_calls"][:st["max_depth_seen"] + 1]),
                           "particles": list(st["level_particles"][:st["max_depth_seen"] + 1]),
                           "note": "hhs_fsi calls and particles per hierarchy depth, timed steps"},
                "parity": PARITY_BARS,
                **extra}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batch(args):
    """Batch of independent clusters (config: 256 Plummer clusters, N log-uniform 64..4096):
    every timed step is one launch that advances all clusters by one top-level step."""
    import torch

    from paper_2011_14984_gb300 import build as fbuild
    from paper_2011_14984_gb300 import frost as fr
    from paper_2011_14984_gb300 import ics

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    fbuild.build()
    fr.load()
    stream = work_stream()
    off, m, x, v = ics.batch_workload(args.workload)
    ncl = off.size - 1
    f = fr.Frost(m, x, v, G=1.0, eta=args.eta, precision="mixed", stream=stream.cuda_stream,
                 offsets=off)
    tuned = f.autotune()  # the team split of the batch launch, outside the timed region
    e0 = f.cluster_energies()
    # steps per frost_step call: 1, or (with --t-end) every step to t_end in one call, which is
    # one launch (one replay of the captured step graph) for all clusters
    per_call = 1
    if args.t_end is not None:
        import math
        per_call = int(math.ceil(args.t_end / args.dt - 1e-9))
        n0 = m.size
        x0 = torch.empty((n0, 3), dtype=torch.float64).pin_memory().numpy()
        v0 = torch.empty((n0, 3), dtype=torch.float64).pin_memory().numpy()
        t0_state = fr.frost_get_state(f.ctx, x0, v0)
        f.step(args.dt, per_call)  # captures the graph of this call shape (untimed)
        fr.frost_set_state(f.ctx, x0, v0, t0_state)
    else:
        for _ in range(args.warmup):
            f.step(args.dt, 1)
        e0 = f.cluster_energies()
    f.reset_stats()
    f.set_timing(True)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.synchronize()
    clocks.start()
    ms = 0.0
    calls = 1 if args.t_end is not None else args.steps
    for _ in range(calls):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        f.step(args.dt, per_call)
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    torch.cuda.synchronize()
    clk = clocks.stop()
    st = f.stats()
    f.set_timing(False)
    e1 = f.cluster_energies()
    dE = np.abs((e1["E"] - e0["E"]) / e0["E"])
    inter = method_pairs(st)
    value = inter / (ms * 1e-3)
    flops = (st["acc_pairs"] * FLOPS_PER_PAIR["acc"] + st["grad_pairs"] * FLOPS_PER_PAIR["grad"]
             + st["tstep_pairs"] * FLOPS_PER_PAIR["tstep"])
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    ach = flops / (st["timed_ms"][3] * 1e-3) / 1e12 if st["timed_ms"][3] > 0 else 0.0
    # end to end with host buffers
    n = m.size
    xh = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    vh = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    tt = fr.frost_get_state(f.ctx, xh, vh)
    f.reset_stats()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 4))
    for _ in range(e2e_steps):
        fr.frost_set_state(f.ctx, xh, vh, tt)
        fr.frost_step(f.ctx, args.dt, 1)
        tt = fr.frost_get_state(f.ctx, xh, vh)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    st2 = f.stats()
    f.close()
    nsteps = calls * per_call
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": nsteps,
            "warmup": args.warmup, "ms_per_step": ms / nsteps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "clusters": int(ncl), "N_total": int(n),
                       "N_min": int(np.diff(off).min()), "N_max": int(np.diff(off).max()),
                       "eta": args.eta, "dt_pivot": args.dt, "t_end": args.t_end,
                       "step": ("one launch (one replay of the captured step graph): every cluster "
                                f"advances {per_call} top-level HHS-FSI steps, to t = {per_call * args.dt:g}")
                               if per_call > 1 else
                               "one launch: every cluster in its own thread block advances one "
                               "top-level HHS-FSI step",
                       "l2": "flushed before every timed step (256 MiB write)"},
            "roofline": {"bound": "alu", "kernel": "k_hhs_subtree (batch; all passes)", "achieved": ach,
                         "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                         "flops_counted": "acc 20, grad 38, tstep 45 per pair"},
            "cpu_baseline": None,
            "e2e": {"value": method_pairs(st2) / e2e_s, "unit": UNIT,
                    "steps": e2e_steps, "h2d_bytes_per_step": int(2 * n * 24),
                    "d2h_bytes_per_step": int(2 * n * 24)},
            "gpu_launches": calls, "clocks": clk, "seconds_timed": ms * 1e-3,
            "dE_over_E_clusters": {"median": float(np.median(dE)), "max": float(dE.max())},
            "autotuned_teams": tuned,
            "max_depth": st["max_depth_seen"], "hhs_calls": st["hhs_calls"]}
    print(json.dumps(line), flush=True)


def run_passes(args):
    """Full passes of a workload: acc+gradient and time-step, timed with CUDA events, and the
    hierarchy level each particle's time-step would put it on (level = number of halvings of
    dt_pivot until tau_i >= pivot)."""
    import torch

    from paper_2011_14984_gb300 import build as fbuild
    from paper_2011_14984_gb300 import frost as fr
    from paper_2011_14984_gb300 import ics

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    fbuild.build()
    fr.load()
    stream = work_stream()
    m, x, v = ics.workload(args.workload)
    n = m.size
    f = fr.Frost(m, x, v, G=1.0, eta=args.eta, precision="mixed", stream=stream.cuda_stream)
    for _ in range(args.warmup):
        f.accel_gradient(None, None, eps_grad=args.dt, want=("acc_tilde",))
    f.set_timing(True)
    f.reset_stats()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    ms = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        f.accel_gradient(None, None, eps_grad=args.dt, want=("acc_tilde",))
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    tau = f.timesteps()
    b.record(stream)
    b.synchronize()
    ms_tau = a.elapsed_time(b)
    clk = clocks.stop()
    st = f.stats()
    f.close()
    t = tau.cpu().numpy()
    lev = np.maximum(0, np.ceil(np.log2(args.dt / t))).astype(int)
    hist = np.bincount(lev)
    value = 2.0 * n * (n - 1) * args.steps / (ms * 1e-3)
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    kinds = ["acc", "grad", "tstep"]
    per = {kinds[k]: {"launches": st["timed_launches"][k], "ms": st["timed_ms"][k],
                      "tflops": st["timed_pairs"][k] * FLOPS_PER_PAIR[kinds[k]] / (st["timed_ms"][k] * 1e-3) / 1e12
                      if st["timed_ms"][k] > 0 else 0.0} for k in range(3)}
    dom = max(range(3), key=lambda k: st["timed_ms"][k])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "N": int(n), "eta": args.eta, "dt_pivot": args.dt,
                       "step": "one full acc + gradient pass over all N (no hierarchical steps)",
                       "l2": "flushed before every timed pass (256 MiB write)"},
            "roofline": {"bound": "alu", "kernel": kinds[dom] + " pass (mixed)", "achieved": per[kinds[dom]]["tflops"],
                         "peak": peak, "unit": "TFLOP/s", "frac": per[kinds[dom]]["tflops"] / peak,
                         "traffic": None, "per_kind": per},
            "timestep_pass_ms": ms_tau,
            "level_histogram": {"levels": hist.tolist(), "max_level": int(lev.max()),
                                "tau_min": float(t.min()), "tau_median": float(np.median(t)),
                                "note": "level of tau_i below dt_pivot on the first partition"},
            "clocks": clk}
    print(json.dumps(line), flush=True)


def binary_energies(fr, stream, m, x, v, pairs):
    """Energy bookkeeping of a system with binaries (pairs [k, 2] of member indices): the
    internal two-body energies of the binaries (FP64, host) and the energy of the system with
    every binary replaced by its centre of mass (the potential through the library's FP64
    energy pass on the GPU).  Their sum differs from the total energy by the binaries' tidal
    terms only."""
    i1, i2 = pairs[:, 0], pairs[:, 1]
    m1, m2 = m[i1], m[i2]
    mt = m1 + m2
    r = np.linalg.norm(x[i1] - x[i2], axis=1)
    u = v[i1] - v[i2]
    e_int = 0.5 * (m1 * m2 / mt) * (u * u).sum(1) - m1 * m2 / r
    single = np.ones(m.size, dtype=bool)
    single[i1] = single[i2] = False
    xc = (m1[:, None] * x[i1] + m2[:, None] * x[i2]) / mt[:, None]
    vc = (m1[:, None] * v[i1] + m2[:, None] * v[i2]) / mt[:, None]
    mm = np.concatenate([m[single], mt])
    xm = np.concatenate([x[single], xc])
    vm = np.concatenate([v[single], vc])
    g = fr.Frost(mm, xm, vm, G=1.0, precision="fp64", stream=stream.cuda_stream)
    e = g.energy()
    g.close()
    return e["E"], e_int


def run_integrate(args):
    """Integration of a single-set workload: --steps top-level HHS-FSI steps of --dt (all of
    them, or those that fit in --max-seconds), each timed with CUDA events, with the hierarchy
    of every step (depth, hhs_fsi calls and set sizes per level), the errors of E, P and L,
    and the wall time extrapolated to --t-end at the measured rate.  With --compare-fp64 the
    FP64 mode runs the same steps from the same state, and the positions, velocities and
    conservation errors of the two are compared."""
    import math

    import torch

    from paper_2011_14984_gb300 import build as fbuild
    from paper_2011_14984_gb300 import frost as fr
    from paper_2011_14984_gb300 import ics

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    fbuild.build()
    fr.load()
    stream = work_stream()
    m, x, v = ics.workload(args.workload)
    n = m.size
    steps = args.steps
    if args.t_end is not None and not args.max_seconds:
        steps = int(math.ceil(args.t_end / args.dt - 1e-9))
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    runs = {}
    for prec in (("mixed", "fp64") if args.compare_fp64 else ("mixed",)):
        f = fr.Frost(m, x, v, G=1.0, eta=args.eta, precision=prec, stream=stream.cuda_stream,
                     subtree_max=args.subtree_max, branch_streams=args.branch_streams,
                     sym_cross=args.sym_cross)
        tuned = f.autotune() if prec == "mixed" else None
        e0 = f.energy()
        bpairs = ics.binary_pairs(n) if args.workload == "plummer_kroupa_binaries_256k" else None
        if bpairs is not None:
            eb0, eint0 = binary_energies(fr, stream, m, x, v, bpairs)
        per = []
        ms_total = 0.0
        pairs = 0.0
        lev_calls = np.zeros(48, dtype=np.int64)
        lev_part = np.zeros(48, dtype=np.int64)
        wall0 = time.perf_counter()
        for k in range(steps):
            f.reset_stats()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            f.step(args.dt, 1)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            st = f.stats()
            d = st["max_depth_seen"]
            lc = np.array(st["level_calls"], dtype=np.int64)
            lp = np.array(st["level_particles"], dtype=np.int64)
            lev_calls += lc
            lev_part += lp
            ms_total += ms
            pairs += method_pairs(st)
            per.append({"ms": ms, "max_depth": d, "hhs_calls": int(lc.sum()),
                        "deepest_level_calls": int(lc[d]), "interactions": method_pairs(st)})
            if args.max_seconds and time.perf_counter() - wall0 > args.max_seconds:
                break
        done = len(per)
        e1 = f.energy()
        xs, vs, t = f.state()
        f.close()
        binaries = None
        if bpairs is not None:
            eb1, eint1 = binary_energies(fr, stream, m, xs, vs, bpairs)
            de = eint1 - eint0
            worst = np.argsort(-np.abs(de))[:5]
            i1, i2 = bpairs[:, 0], bpairs[:, 1]
            mt = m[i1] + m[i2]
            r0 = x[i1] - x[i2]
            u0 = v[i1] - v[i2]
            a0 = 1.0 / (2.0 / np.linalg.norm(r0, axis=1) - (u0 * u0).sum(1) / mt)
            h0 = np.linalg.norm(np.cross(r0, u0), axis=1)
            peri0 = a0 * (1.0 - np.sqrt(np.maximum(0.0, 1.0 - h0 * h0 / (mt * a0))))
            binaries = {
                "dE_bulk_over_E": abs((eb1 - eb0) / e0["E"]),
                "dE_binaries_internal_over_E": float(abs(de.sum()) / abs(e0["E"])),
                "dE_total_over_E": abs((e1["E"] - e0["E"]) / e0["E"]),
                "worst_binaries": [{"pair": int(k), "pericentre_t0": float(peri0[k]), "a_t0": float(a0[k]),
                                    "E_internal_t0": float(eint0[k]), "dE_internal": float(de[k])}
                                   for k in worst],
                "note": "bulk: every binary replaced by its centre of mass; internal: the binaries' "
                        "two-body energies; their sum is the total up to the tidal terms"}
        dmax = int(max(p["max_depth"] for p in per))
        secs = ms_total * 1e-3
        L0 = np.linalg.norm(e0["L"])
        runs[prec] = {
            "steps_done": done, "t_reached": t, "device_s": secs,
            "value": pairs / secs, "unit": UNIT,
            "top_level_steps_per_s": done / secs,
            "deepest_level_calls_per_s": sum(p["deepest_level_calls"] for p in per) / secs,
            "depth_per_step": [p["max_depth"] for p in per],
            "ms_per_step": [p["ms"] for p in per],
            "levels": {"calls": lev_calls[:dmax + 1].tolist(),
                       "mean_set_size": [float(lev_part[k] / lev_calls[k]) if lev_calls[k] else 0.0
                                         for k in range(dmax + 1)],
                       "calls_per_s": (lev_calls[:dmax + 1] / secs).tolist()},
            "dE_over_E": abs((e1["E"] - e0["E"]) / e0["E"]),
            "dP": float(np.linalg.norm(e1["P"] - e0["P"])),
            "dL_over_L": float(np.linalg.norm(e1["L"] - e0["L"]) / L0) if L0 > 0 else None,
            "autotune_waves": tuned, "binaries": binaries, "_x": xs, "_v": vs}
        if args.t_end is not None:
            runs[prec]["extrapolated_s_to_t_end"] = secs * args.t_end / t
            runs[prec]["t_end"] = args.t_end
    clk = clocks.stop()
    mixed = runs["mixed"]
    out = {"metric": METRIC, "value": mixed["value"], "unit": UNIT, "n_gpus": 1,
           "steps": mixed["steps_done"], "warmup": 0,
           "ms_per_step": 1e3 * mixed["device_s"] / mixed["steps_done"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": args.workload, "N": int(n), "eta": args.eta, "dt_pivot": args.dt,
                      "t_end": args.t_end, "mode": "integration, per-step statistics"},
           "clocks": clk}
    if args.compare_fp64:
        fp = runs["fp64"]
        k = min(mixed["steps_done"], fp["steps_done"])
        assert k == mixed["steps_done"] == fp["steps_done"], "compare equal step counts"
        dx = np.linalg.norm(mixed["_x"] - fp["_x"], axis=1)
        dv = np.linalg.norm(mixed["_v"] - fp["_v"], axis=1)
        out["fp64_comparison"] = {
            "dE_over_E": {"mixed": mixed["dE_over_E"], "fp64": fp["dE_over_E"]},
            "dP": {"mixed": mixed["dP"], "fp64": fp["dP"]},
            "dL_over_L": {"mixed": mixed["dL_over_L"], "fp64": fp["dL_over_L"]},
            "mixed_speedup": fp["device_s"] / mixed["device_s"],
            "position_difference": {"p50": float(np.median(dx)), "p999": float(np.percentile(dx, 99.9)),
                                    "max": float(dx.max())},
            "velocity_difference": {"p50": float(np.median(dv)), "p999": float(np.percentile(dv, 99.9)),
                                    "max": float(dv.max())}}
    for prec, r in runs.items():
        r.pop("_x")
        r.pop("_v")
        out[prec] = r
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload.startswith("cluster_batch"):
        run_batch(args)
    elif args.passes_only:
        run_passes(args)
    elif args.integrate:
        run_integrate(args)
    else:
        run_frost(args)


if __name__ == "__main__":
    main()
