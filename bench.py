#!/usr/bin/env python
"""Benchmark of the WCSPH hot path on GB300: SPH particle-steps/s.

One step = one full pass of the method over the whole particle set: cell
hash + radix sort + cell ranges + reorder, two evaluations (colour, normal,
forces) with the predictor-corrector update in between, inflow/outflow, and
(every 100 steps) the breakup-length evaluation.

Default workload (N = 1): the large 2D planar jet, Re = 100, We = 10,
Wendland kernel, dx = D/100, 100 D domain (~1M particles), FP32 pair sums with
FP64 positions and time, adaptive dt (Eqs. 30-32).  Inputs are seeded
synthetic states (workloads.py).  The K timed steps start with a forced cell
rebuild and include the breakup length every 100 steps; a second window of at
least 64 rebuild cadences gives the steady-state rate.  Beside the line: the
64-jet batched ensemble (batched and member by member), the GPU's FP32 / FP64
FMA peaks measured by the library's probe, and the FP64 CPU oracle on 1 thread
and on every host core.  Small states (below twice the L2 size) are timed step
by step with a 256 MiB L2 flush before each step (outside the events); large
ones back to back.

Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload jet_c2|jet_c3|dam_c1]
  python bench.py --workload ensemble_c4 [--steps K]   (64-jet batched ensemble,
      one graph launch per ensemble step, against the same members run one after
      another with their own step graphs)
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)
Under torchrun each rank simulates its own jet (seed = rank): weak scaling,
no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1603_02421_gb300 import workloads as wl  # noqa: E402

METRIC = "SPH particle-steps/s on 1 GB300, plain vs batched/surrogate, at fixed error"
UNIT = "particle-steps/s"
BREAKUP_EVERY = 100
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def workload(name: str, seed: int):
    if name == "jet_c2":
        case = wl.jet(seed=seed, Re=200.0, We=20.0, dx=1.0 / 40, length=60.0,
                      kernel="wendland", prec="fp32")
        desc = ("2D planar jet, Re=200, We=20, Wendland, dx=D/40, 60D domain, "
                "FP32 pair sums / FP64 positions, adaptive dt")
    elif name == "jet_c3":
        case = wl.jet(seed=seed, Re=100.0, We=10.0, dx=1.0 / 100, length=100.0,
                      kernel="wendland", prec="fp32", capacity_factor=1.15)
        desc = ("2D planar jet, Re=100, We=10, Wendland, dx=D/100, 100D domain, "
                "FP32 pair sums / FP64 positions, adaptive dt")
    elif name == "dam_c1":
        case = wl.dam_break(seed=seed, dx=0.01, prec="fp64")
        desc = "2D dam break with obstacle, cubic spline, dx=0.01 m, FP64, dt=1e-4"
    else:
        raise SystemExit("unknown workload %s" % name)
    return case, desc


# Algorithmic FP32 operations per interacting pair (r < 2h) (Wendland),
# counting a fused multiply-add as 2 and rsqrt, sqrt and division as 1 each;
# compares and selects are not counted.  Geometry (offset difference with the
# cell shift, r^2, 1/r, q, 1/q) 11; W(q) 7; F(q) 4; colour accumulate 2;
# normal weight 3 + accumulate 4; forces: continuity 9 + viscosity 10 +
# pressure 8 + Eq. 31 term 3 = 30.
#   pairsum (with surface tension: colour and the state-only forces in one
#           list walk): geometry + W + F + colour 2 + forces 30 = 54
#   normal: geometry + F + 7 = 22 per pair walked
#   forces (without surface tension, one walk): geometry + F + 30 = 45
# The method itself (colour, normal and forces each with its own geometry,
# as the equations are written) is 20 + 22 + 45 = 87 per pair and evaluation.
FLOP_PER_PAIR = {"pairsum": 54, "pairsum_correct": 54, "normal": 22}
FLOP_PER_PAIR_NO_CSF = {"forces": 45, "forces_correct": 45}
FLOP_PER_PARTICLE = {"pairsum": 22, "pairsum_correct": 22, "normal": 8, "forces": 20,
                     "forces_correct": 30}
FLOP_METHOD_PER_PAIR = 87
FLOP_METHOD_PER_PAIR_NO_CSF = 45
STEP_BYTES_PER_SORT = 100.0


def step_bytes_lower(fp64: bool, csf: bool, rebuild_fraction: float) -> float:
    """Lower bound of the HBM bytes per particle-step of the method: two
    evaluations, each reading the state S (position 16 B, velocity and
    density: 28 B in FP32, 40 B in FP64) and, with surface tension, writing
    and reading the colour and the normal (24 B in FP32, 48 B in FP64); the
    predictor's half-step save and reload (2 S); the final state write (S);
    ~100 B per cell sort (key and index passes, state permutation) at the
    fraction of steps that rebuild.  Neighbour re-reads are not counted (cache
    reuse).  FP32 with surface tension: 188 B + 100 B per sort."""
    S = 40.0 if fp64 else 28.0
    c = (48.0 if fp64 else 24.0) if csf else 0.0
    return 2.0 * (S + c) + 2.0 * S + S + STEP_BYTES_PER_SORT * rebuild_fraction
# Algorithmic HBM bytes per particle of the streaming kernel groups (FP32 path).
BYTES_PER_PARTICLE = {"cell_sort": 16 + 1 + 4 + 4 + 4 + 4 + 4, "reorder": 2 * 41 + 4 + 4 + 32,
                      "predict": 41 + 12 + 48, "spawn": 0}


# Batched ensemble: 64 jets on the Re x We grid of the paper's sweeps
# (Table 1 ranges), dx from D/30 to D/80 and 20k-400k particles per member.
ENS_RE = [100, 200, 400, 700, 1000, 1500, 2000, 3000]
ENS_WE = [5, 10, 15, 20, 30, 40, 50, 60]


def ensemble_members():
    """(member, Re, We, dx, strip length) of the 64 members: member m = 8i + j
    has Re_i, We_j, dx = D / (30 + 50 m/63) and a strip holding about
    20k * 20^(m/63) particles (geometric from 20k to 400k)."""
    out = []
    for i, re in enumerate(ENS_RE):
        for j, we in enumerate(ENS_WE):
            m = 8 * i + j
            f = m / 63.0
            dx = 1.0 / (30.0 + 50.0 * f)
            n_target = 20000.0 * 20.0 ** f
            out.append((m, float(re), float(we), dx, n_target * dx * dx))
    return out


def ensemble_case(m, re, we, dx, length, skin):
    case = wl.jet(seed=m, Re=re, We=we, dx=dx, length=length, kernel="wendland", prec="fp32",
                  capacity_factor=1.15)
    case["params"]["skin_over_h"] = skin
    return case


# Sources that define the SPH step kernels (the host runtime is not among them).
KERNEL_SOURCES = ("sph_sweeps.cu", "sph_device.cuh", "sph_internal.cuh")


def sources_sha256() -> str:
    """Hash of the sources that define libsph's step kernels."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1603_02421_gb300", "csrc")
    hsh = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            hsh.update(name.encode() + b"\0" + f.read())
    return hsh.hexdigest()


# Fallback roofline denominators when MEASURED_PEAKS.json (measured on this
# pool's GPUs) is absent: one earlier measurement on a GB300.
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def pool_peak(key: str):
    """(value, "of measured" | "of fallback") of a MEASURED_PEAKS.json entry."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)[key]), "of measured"
    except (OSError, ValueError, KeyError, TypeError):
        return FALLBACK_PEAKS[key], "of fallback"


def measured_step_traffic(workload: str):
    """DRAM bytes per particle of a step that keeps its cell build, summed over
    the step's launches in an ncu capture summarised under profiles/ (a line
    'step-traffic: workload=... bytes_per_particle=... sources_sha256=...');
    None when no capture of this workload exists or the sources changed."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    want = sources_sha256()
    for name in sorted(os.listdir(pdir)):
        if not name.endswith(".md"):
            continue
        for line in open(os.path.join(pdir, name)):
            if not line.startswith("step-traffic:"):
                continue
            kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
            if kv.get("workload") == workload and kv.get("sources_sha256") == want:
                return float(kv["bytes_per_particle"])
    return None


def measured_traffic(group: str, particles: float):
    """DRAM bytes (read + write) per launch of a kernel group from an ncu
    capture summarised under profiles/ (a line 'traffic: group=... bytes=...
    particles=... sources_sha256=...'), scaled to `particles`; None when no
    capture exists or the sources changed since it was taken."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    want = sources_sha256()
    for name in sorted(os.listdir(pdir)):
        if not name.endswith(".md"):
            continue
        for line in open(os.path.join(pdir, name)):
            if not line.startswith("traffic:"):
                continue
            kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
            if kv.get("group") == group and kv.get("sources_sha256") == want:
                return float(kv["bytes"]) * particles / float(kv["particles"])
    return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="jet_c3",
                    choices=["jet_c2", "jet_c3", "dam_c1", "ensemble_c4", "surrogate_c5",
                             "surrogate_step"])
    ap.add_argument("--train-seconds", type=float, default=60.0,
                    help="surrogate_c5: GPU training time of the network")
    ap.add_argument("--threshold", type=float, default=1e-3,
                    help="surrogate_c5: residual threshold above which plain SPH takes over")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="jet_c3: skip the 64-jet batched ensemble reported beside the line")
    ap.add_argument("--ensemble-steps", type=int, default=100,
                    help="jet_c3: ensemble steps timed for the batched_c4 keys")
    ap.add_argument("--cpu-seconds", type=float, default=24.0)
    ap.add_argument("--tune", default="auto",
                    help="auto (autotuner), or LANES,CADENCE[,gated|conditional] (e.g. 4,1 for "
                         "every-step cell builds; the third field picks how a step at cadence > 1 "
                         "chooses its start on the device, default gated)")
    ap.add_argument("--skin", type=float, default=None,
                    help="skin / h of the cell search (default 0.15 for the jets, whose lists "
                         "are kept in the velocity frame, 0.3 for the dam break, whose walls "
                         "keep the absolute rebuild test)")
    args = ap.parse_args()
    if args.skin is None:
        args.skin = 0.3 if args.workload == "dam_c1" else 0.15
    return args


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample(case, max_particles=24000):
    """A bounded sample of the workload for the CPU oracle: the upstream part
    of the jet (all particles with x below a cut chosen so that at most
    max_particles remain), with its inflow."""
    st = case["fluid"]
    x = st["x"]
    if len(x) > max_particles:
        cut = np.sort(x)[max_particles]
        keep = x < cut
        st = {k: v[keep] for k, v in st.items()}
        p = dict(case["params"])
        p["xmax"] = float(cut)
        case = dict(case, fluid=st, params=p)
    return case


def run_oracle(case, seconds, max_steps=None):
    from oracle import oracle as orc
    orc.build()
    sim = orc.OracleSim(case["params"], case["fluid"], case.get("boundary"))
    inf = case.get("inflow")
    if inf is not None:
        sim.add_inflow(inf["x_exit"], inf["y0"], inf["y1"], inf["U"], inf["amp"], inf["k"],
                       inf["phase"], inf["layers"])
    psteps = 0
    nsteps = 0
    t0 = time.perf_counter()
    while True:
        n = len(sim.st["x"])
        sim.step()
        psteps += n
        nsteps += 1
        el = time.perf_counter() - t0
        if (max_steps is not None and nsteps >= max_steps) or \
                (max_steps is None and el >= seconds):
            break
    return psteps, nsteps, time.perf_counter() - t0, len(sim.st["x"])


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload in ("ensemble_c4", "surrogate_c5"):
        m, re, we, dx, length = ensemble_members()[0]
        case = ensemble_case(m, re, we, dx, length, args.skin)
        desc = "member 0 of the 64-jet ensemble"
    else:
        case, desc = workload(args.workload, seed=0)
    from oracle import oracle as orc
    orc.build()
    cores = orc.max_threads()
    orc.set_threads(cores)
    # the oracle runs ~6e6 particle-steps/s on the 16 cores of the GPU host:
    # the sample is sized so that the K steps take well under a minute
    budget = 1.2e8 / max(args.steps, 1)
    sample = oracle_sample(case, int(min(24000, max(2000, budget))))
    run_oracle(sample, 0, max_steps=max(args.warmup, 0) or 1)
    psteps, nsteps, el, n = run_oracle(sample, 0, max_steps=args.steps)
    v = psteps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / nsteps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload + ": " + desc, "particles": n,
                   "sample": "upstream %d particles of the workload" % n},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "FP64 CPU oracle (OpenMP over particles, %d threads), %d "
                                   "steps of the upstream %d particles" % (cores, nsteps, n)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the first reading takes a moment: start timing only once it is in
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = [r[0] for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, val in zip(names, r[2:]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1603_02421_gb300 import binding, build
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()

    from paper_1603_02421_gb300.replicas import rank_members
    if args.workload == "ensemble_c4":
        bench_ensemble(args, binding, dist, dev, rank, world, local)
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.workload == "surrogate_step":
        bench_surrogate_step(args, binding, dev, rank, local)
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.workload == "surrogate_c5":
        bench_surrogate(args, binding, dist, dev, rank, world, local)
        if dist is not None:
            dist.destroy_process_group()
        return
    case, desc = workload(args.workload, seed=rank_members(rank, world, world)[0])
    case["params"]["skin_over_h"] = args.skin
    line, sim = bench_plain(args, binding, dist, dev, rank, world, local, case, desc)
    sim.close()
    if world == 1 and args.workload == "jet_c3" and not args.no_ensemble:
        # the metric compares plain with batched: the 64-jet ensemble of the
        # paper's Re x We sweeps, batched and member by member, beside it
        # (one GPU only: with N > 1 the other GPUs would idle meanwhile; the
        # ensemble's own scaling run is --workload ensemble_c4)
        ens = bench_ensemble(args, binding, None, dev, 0, 1, local, steps=args.ensemble_steps,
                             emit=False, cpu=False)
        line["batched_c4"] = {k: ens[k] for k in ("value", "plain_value", "batched_over_plain",
                                                  "ms_per_step", "steps", "particles_total",
                                                  "tuning", "clocks", "gpu_launches")}
        line["batched_c4"]["workload"] = ens["workload"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def measured_peaks(binding, local):
    """FP32 and FP64 FMA rates of this GPU from the library's own probe
    (CUDA events, best of 5 launches), with the SM clocks sampled while it
    ran."""
    clocks = ClockSampler(local)
    f32, ms32 = binding.sph_fma_peak(local, 0)
    f64, ms64 = binding.sph_fma_peak(local, 1)
    clk = clocks.stop()
    return {"fp32_tflops": f32, "fp64_tflops": f64, "fp32_launch_ms": ms32,
            "fp64_launch_ms": ms64, "clocks": clk,
            "how": "sph_fma_peak: every SM filled with threads running 8 independent FMA "
                   "chains, 2 x FMAs / time of the best of 5 launches (CUDA events)"}


def bench_plain(args, binding, dist, dev, rank, world, local, case, desc):
    """One jet (or the dam break): autotune, W warm-up steps, then exactly K
    timed steps starting with a forced cell rebuild, then a steady-state
    window of at least 64 rebuild cadences, per-kernel attribution, the
    roofline of the dominant kernel group, end to end through the ABI, and
    the CPU oracle."""
    import torch
    peaks = measured_peaks(binding, local)
    free0 = torch.cuda.mem_get_info(dev)[0]
    stream = torch.cuda.Stream(device=dev)
    sim = binding.Simulation(case, stream=stream.cuda_stream, device=local)
    ctx = sim.ctx
    resident = max(free0 - torch.cuda.mem_get_info(dev)[0], 0)
    l2_bytes = 129 * 1024 * 1024
    flush_l2 = resident < 2 * l2_bytes
    if args.tune == "auto":
        lanes, cadence, _ = binding.sph_autotune(ctx, 24)
        form = binding.sph_get_start_form(ctx)
    else:
        lanes, cadence, form = parse_tune(args.tune)
        binding.sph_set_tuning(ctx, lanes, cadence)
        binding.sph_set_start_form(ctx, form)
    per_full, per_reuse, per_breakup = binding.sph_kernel_counts(ctx)
    has_inflow = case.get("inflow") is not None

    # interacting pairs of the initial state (for the algorithmic FLOP count)
    n0 = binding.sph_get_time(ctx)["n"]
    pa, _ = binding.sph_get_pairs(ctx, int(n0 * 40))
    pairs_per_particle = len(pa) / max(n0, 1)
    del pa

    flush = (torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
             if flush_l2 else None)
    for _ in range(max(args.warmup, 0)):
        binding.sph_run_async(ctx, 1)
        binding.sph_sync(ctx)

    def timed(K, profile):
        """K steps.  Small states (resident set below twice the L2): each step
        bracketed by CUDA events on the library's stream with an L2 flush
        before it, outside the events.  Large states: the K steps back to
        back between two events (the inputs do not fit in L2).  The breakup
        length (every 100 steps) is inside the timed region."""
        nact = np.zeros(K, np.int64)
        Ls = []
        n_now = binding.sph_get_time(ctx)["n"]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        if flush is not None or profile:
            ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
            ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
            for k in range(K):
                nact[k] = n_now
                if flush is not None:
                    with torch.cuda.stream(stream):
                        flush.zero_()
                ev0[k].record(stream)
                binding.sph_run_async(ctx, 1)
                if has_inflow and not profile and (k + 1) % BREAKUP_EVERY == 0:
                    Ls.append(binding.sph_breakup_length(ctx)[0])
                ev1[k].record(stream)
                binding.sph_sync(ctx)
                if (k + 1) % 50 == 0:
                    n_now = binding.sph_get_time(ctx)["n"]
            torch.cuda.synchronize(dev)
            ms = np.array([ev0[k].elapsed_time(ev1[k]) for k in range(K)])
            return ms, nact, Ls
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        done = 0
        while done < K:
            chunk = min(BREAKUP_EVERY - done % BREAKUP_EVERY, K - done)
            nact[done:done + chunk] = n_now
            binding.sph_run_async(ctx, chunk)
            done += chunk
            if has_inflow and done % BREAKUP_EVERY == 0:
                Ls.append(binding.sph_breakup_length(ctx)[0])
                n_now = binding.sph_get_time(ctx)["n"]
        e1.record(stream)
        binding.sph_sync(ctx)
        torch.cuda.synchronize(dev)
        total = e0.elapsed_time(e1)
        return np.full(K, total / K), nact, Ls

    def window(K):
        """K timed steps from a forced rebuild; (ms per step, active counts,
        breakup lengths, steps that rebuilt, wall seconds, clocks)."""
        binding.sph_request_rebuild(ctx)
        clocks = ClockSampler(local)
        b0 = binding.sph_get_rebuild_stats(ctx)[0]
        t0 = time.perf_counter()
        ms, nact, Ls = timed(K, profile=False)
        wall = time.perf_counter() - t0
        clk = clocks.stop()
        # cell sorts in the window: one per rebuilding step and one per
        # breakup-length evaluation
        full = binding.sph_get_rebuild_stats(ctx)[0] - b0 - len(Ls)
        return ms, nact, Ls, full, wall, clk

    K = args.steps
    step_ms, nact, Ls, full_steps, wall, clk = window(K)
    nbreak = len(Ls)
    from paper_1603_02421_gb300.replicas import reduce_rate
    value, total_s, units = reduce_rate(step_ms.sum() / 1e3, float(nact.sum()), dist, dev)
    if dist is not None:
        dist.barrier()
    # steady state: enough steps for many rebuild cycles and inflow layers
    Ks = max(K, 64 * cadence, 1000)
    s_ms, s_nact, s_Ls, s_full, s_wall, s_clk = window(Ks)
    steady_value = float(s_nact.sum()) / (s_ms.sum() / 1e3)

    # per-kernel attribution: the same steps with a CUDA event before each
    # kernel group (captured into the step graph)
    binding.sph_profile(ctx, 1)
    binding.sph_run_async(ctx, 1)
    binding.sph_sync(ctx)
    binding.sph_profile(ctx, 1)
    Kp = min(Ks, 200)
    prof_ms, _, _ = timed(Kp, profile=True)
    prof = binding.sph_profile_report(ctx)
    binding.sph_profile(ctx, 0)

    # ---- roofline of the dominant kernel group --------------------------
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_launches = prof[dom]
    avg_s = dom_ms / 1e3 / max(dom_launches, 1)
    n_mean = float(nact.mean())
    csf = float(case["params"].get("sigma", 0.0)) > 0.0
    per_pair = dict(FLOP_PER_PAIR) if csf else dict(FLOP_PER_PAIR_NO_CSF)
    if csf:
        per_pair.pop("normal")       # walked only near the surface: not a full-pair count
    if dom in per_pair:
        flops = n_mean * (pairs_per_particle * per_pair[dom] + FLOP_PER_PARTICLE[dom])
        achieved = flops / avg_s / 1e12
        fp64 = case["params"].get("prec") == "fp64"
        peak = peaks["fp64_tflops" if fp64 else "fp32_tflops"]
        roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": measured_traffic(dom, n_mean),
                "peak_source": "measured on this GPU by the library's FMA probe (sph_fma_peak, "
                               "%s, median SM clock %s MHz during the probe)"
                               % ("FP64" if fp64 else "FP32",
                                  peaks["clocks"]["sm_mhz"] if peaks["clocks"] else "n/a"),
                "algorithmic_per_launch": flops}
    else:
        hbm, hbm_src = pool_peak("hbm_gbs")
        nbytes = n_mean * BYTES_PER_PARTICLE.get(dom, 0)
        achieved = nbytes / avg_s / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm,
                "traffic": measured_traffic(dom, n_mean),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % hbm_src,
                "algorithmic_per_launch": nbytes}

    # ---- the whole step against both rooflines ----------------------------
    # at the steady-state rate: the method's FLOPs (each equation with its own
    # geometry, pairs r < 2h, two evaluations per step), the lower-bound bytes
    # and the DRAM bytes ncu measured for a step that keeps its build
    fp64 = case["params"].get("prec") == "fp64"
    mp_hbm, hbm_src = pool_peak("hbm_gbs")
    s_rebuild = s_full / Ks
    step_flop = 2.0 * pairs_per_particle * (FLOP_METHOD_PER_PAIR if csf
                                            else FLOP_METHOD_PER_PAIR_NO_CSF)
    step_lower = step_bytes_lower(fp64, csf, s_rebuild)
    step_meas = measured_step_traffic(args.workload)
    arith_peak = peaks["fp64_tflops" if fp64 else "fp32_tflops"]
    step_roof = {
        "rate": steady_value,
        "flop_per_particle_step": step_flop,
        "arith_tflops": step_flop * steady_value / 1e12,
        "arith_peak_tflops": arith_peak,
        "arith_frac": step_flop * steady_value / 1e12 / arith_peak,
        "bytes_lower_bound_per_particle_step": step_lower,
        "hbm_frac_lower_bound": step_lower * steady_value / 1e9 / mp_hbm,
        "dram_bytes_measured_per_particle_step": step_meas,
        "hbm_frac_measured": (step_meas * steady_value / 1e9 / mp_hbm
                              if step_meas is not None else None),
        "hbm_peak_gbs": mp_hbm,
        "hbm_peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % hbm_src,
        "how": "steady-state particle-steps/s times the method's FLOPs (%d per pair r < 2h, "
               "two evaluations) over the measured %s FMA peak, and times bytes per "
               "particle-step over MEASURED_PEAKS hbm_gbs: the method's lower bound (188 B "
               "in FP32 with surface tension, + 100 B x the fraction of steps that rebuild), "
               "and the DRAM traffic ncu measured for a "
               "step that keeps its build (profiles/, null when the kernels changed since)"
               % (FLOP_METHOD_PER_PAIR if csf else FLOP_METHOD_PER_PAIR_NO_CSF,
                  "FP64" if fp64 else "FP32"),
    }

    # ---- end to end through the public API with host buffers -------------
    e2e = None
    if rank == 0:
        e2e = end_to_end(binding, case, stream, local, K=min(K, 100), tuning=(lanes, cadence, form))

    # ---- CPU baseline (oracle) on a bounded sample: 1 thread, all cores ---
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(case, args.cpu_seconds)

    launches = full_steps * per_full + (K - full_steps) * per_reuse + nbreak * per_breakup
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if case["params"].get("prec") == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": args.workload + ": " + desc,
                   "particles_mean": n_mean, "parallelism": "replicas (one jet per GPU)",
                   "l2": ("flushed between timed steps (256 MiB write)" if flush_l2 else
                          "inputs larger than L2 (%.2f GB resident), steps back to back"
                          % (resident / 1e9)),
                   "tuning": {"lanes": lanes, "cadence": cadence,
                              "start_form": FORM_NAMES[form], "skin_over_h": args.skin,
                              "chosen_by": "autotuner" if args.tune == "auto" else "flag",
                              "rebuild_fraction": full_steps / K,
                              "first_timed_step": "forced cell rebuild"},
                   "breakup_every": BREAKUP_EVERY if has_inflow else None,
                   "pairs_per_particle": pairs_per_particle,
                   "wall_s": wall},
        "steady_state": {"value": steady_value, "steps": Ks,
                         "ms_per_step": float(s_ms.sum()) / Ks,
                         "rebuild_fraction": s_full / Ks, "breakups": len(s_Ls),
                         "clocks": s_clk,
                         "how": "a second window of max(K, 64 x cadence, 1000) steps from a "
                                "forced rebuild"},
        "roofline": roof,
        "step_roofline": step_roof,
        "measured_peaks": peaks,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "kernel_ms_per_step": {k: v[0] / Kp for k, v in prof.items()},
        "attribution": {"steps": Kp, "ms_per_step_with_events": float(prof_ms.mean()),
                        "how": "CUDA event before each kernel group inside the step graph"},
        "breakup_L_over_D": Ls,
    }
    return line, sim


def cpu_baseline(case, seconds):
    """The FP64 oracle on a bounded sample of the workload (its upstream part),
    timed with 1 thread and with every host core."""
    from oracle import oracle as orc
    orc.build()
    sample = oracle_sample(case)
    cores = orc.max_threads()
    orc.set_threads(1)
    p1, n1, e1, n = run_oracle(sample, seconds / 3.0)
    orc.set_threads(cores)
    pa, na, ea, n = run_oracle(sample, 2.0 * seconds / 3.0)
    orc.set_threads(1)
    return {"value": pa / ea, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread": {"value": p1 / e1, "cores": 1, "steps": n1, "seconds": e1},
            "sample": "FP64 CPU oracle on the upstream %d particles of the same workload: "
                      "%d steps on %d threads (OpenMP over particles) in %.1f s, and %d steps "
                      "on 1 thread in %.1f s" % (n, na, cores, ea, n1, e1)}


def parse_tune(text):
    """'LANES,CADENCE[,gated|conditional]' -> (lanes, cadence, start form)."""
    from paper_1603_02421_gb300 import binding
    parts = text.split(",")
    forms = {"gated": binding.START_GATED, "conditional": binding.START_CONDITIONAL}
    form = forms[parts[2]] if len(parts) > 2 else binding.START_GATED
    return int(parts[0]), int(parts[1]), form


FORM_NAMES = {0: "gated", 1: "conditional"}


def end_to_end(binding, case, stream, local, K, tuning):
    """Particle-steps/s through the public C ABI with host buffers: upload the
    state from pinned host memory (sph_set_state), K x sph_step (each reads
    the step's dt back to the host), download the state (sph_get_state)."""
    import torch
    sim = binding.Simulation(case, stream=stream.cuda_stream, device=local)
    ctx = sim.ctx
    binding.sph_set_tuning(ctx, *tuning[:2])
    binding.sph_set_start_form(ctx, tuning[2])
    st = binding.sph_get_state(ctx)
    n = len(st["x"])
    pinned = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy()
              for k, v in st.items()}
    binding.sph_step(ctx)              # warm (captures the step graphs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    binding.sph_set_state(ctx, pinned)
    for _ in range(K):
        binding.sph_step(ctx)
    psteps = n * K
    out = binding.sph_get_state(ctx)
    el = time.perf_counter() - t0
    sim.close()
    h2d = n * (16 + 8 + 4 + 4 + 4 + 1 + 4)
    # the state's arrays, plus the types once more for the binding's count query
    d2h_state = len(out["x"]) * (16 + 8 + 4 + 4 + 1 + 4 + 8 + 4 + 1)
    scal = 736   # bytes of the device scalars read back by each sph_step
    return {"value": psteps / el, "unit": UNIT,
            "h2d_bytes_per_step": h2d / K,
            "d2h_bytes_per_step": scal + d2h_state / K,
            "how": "sph_set_state from pinned host arrays, %d x sph_step (dt read back "
                   "each step), sph_get_state; host wall clock" % K}


def bench_ensemble(args, binding, dist, dev, rank, world, local, steps=None, emit=True,
                   cpu=True):
    """The 64-member ensemble: ensemble steps (one graph launch advancing
    every member one step) against the plain form (each member's own step
    graph, one member after another) on the same stream.  Ranks own members
    round-robin (weak scaling over members, no exchange).  Returns the bench
    line (printed by rank 0 when emit)."""
    import torch
    from paper_1603_02421_gb300.replicas import rank_members, reduce_rate
    specs = [ensemble_members()[m] for m in rank_members(rank, world, 64)]
    stream = torch.cuda.Stream(device=dev)
    sims = []
    for (m, re, we, dx, length) in specs:
        sims.append(binding.Simulation(ensemble_case(m, re, we, dx, length, args.skin),
                                       stream=stream.cuda_stream, device=local))
    ens = binding.Ensemble(sims, stream=stream.cuda_stream)
    if args.tune == "auto":
        lanes, cadence, _ = ens.autotune(8)
        form = sims[0].start_form()
    else:
        lanes, cadence, form = parse_tune(args.tune)
        for sm in sims:
            sm.set_tuning(lanes, cadence)
            sm.set_start_form(form)
    counts = [binding.sph_kernel_counts(sm.ctx) for sm in sims]
    # interacting pairs per particle (the same h/dx in every member)
    n_first = sims[0].time()["n"]
    pa, _ = binding.sph_get_pairs(sims[0].ctx, int(n_first * 40))
    pairs_pp = len(pa) / max(n_first, 1)
    del pa

    def live():
        return sum(sm.time()["n"] for sm in sims)

    def builds():
        return [sm.rebuild_stats()[0] for sm in sims]

    K = args.steps if steps is None else steps
    ens.run(max(args.warmup, 1))
    # plain: every member's own step graph (captured on first use), then timed
    for sm in sims:
        binding.sph_run_async(sm.ctx, 1)
    torch.cuda.synchronize(dev)
    n0 = live()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for sm in sims:
        binding.sph_run_async(sm.ctx, K)
    e1.record(stream)
    for sm in sims:
        binding.sph_sync(sm.ctx)
    torch.cuda.synchronize(dev)
    plain_s = e0.elapsed_time(e1) / 1e3
    n1 = live()
    plain_units = 0.5 * (n0 + n1) * K
    # batched
    ens.run(1)
    b0 = builds()
    n0 = live()
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter()
    e0.record(stream)
    ens.run_async(K)
    e1.record(stream)
    ens.sync()
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    batched_s = e0.elapsed_time(e1) / 1e3
    n1 = live()
    b1 = builds()
    units = 0.5 * (n0 + n1) * K
    value, total_s, total_units = reduce_rate(batched_s, units, dist, dev)
    plain_value, _, _ = reduce_rate(plain_s, plain_units, dist, dev)
    launches = 0
    for (pf, pr, _), bb0, bb1 in zip(counts, b0, b1):
        full = bb1 - bb0
        launches += full * pf + (K - full) * pr
    Ls = [binding.sph_breakup_length(sm.ctx)[0] for sm in sims]

    # end to end: members' states from pinned host arrays, K ensemble steps,
    # states back to the host
    Ke = min(K, 20)
    states = [binding.sph_get_state(sm.ctx) for sm in sims]
    pinned = [{k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy()
               for k, v in st.items()} for st in states]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for sm, st in zip(sims, pinned):
        binding.sph_set_state(sm.ctx, st)
    ens.run(Ke)
    outs = [binding.sph_get_state(sm.ctx) for sm in sims]
    e2e_s = time.perf_counter() - t0
    n_e2e = sum(len(st["x"]) for st in states)
    h2d = n_e2e * (16 + 8 + 4 + 4 + 4 + 1 + 4)
    d2h = sum(len(o["x"]) for o in outs) * (16 + 8 + 4 + 4 + 1 + 4 + 8 + 4)
    e2e_value, _, _ = reduce_rate(e2e_s, n_e2e * Ke, dist, dev)

    # whole-step FP32 work against the FP32 peak (algorithmic FLOPs per
    # particle-step of the six pair sweeps and the per-particle work)
    flop_ps = 2 * (pairs_pp * FLOP_METHOD_PER_PAIR + 2 + FLOP_PER_PARTICLE["normal"] +
                   FLOP_PER_PARTICLE["forces_correct"])
    sm_mhz = clk["sm_mhz"] if clk else 1900.0
    peaks = None
    if emit:
        # the ensemble's own line: the FP32 FMA peak measured on this GPU
        peaks = measured_peaks(binding, local)
        peak = peaks["fp32_tflops"]
        peak_source = ("measured on this GPU by the library's FMA probe (sph_fma_peak, FP32, "
                       "median SM clock %s MHz during the probe)"
                       % (peaks["clocks"]["sm_mhz"] if peaks["clocks"] else "n/a"))
    else:
        peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        peak_source = "152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % sm_mhz
    achieved = flop_ps * value / world / 1e12
    cpu_line = None
    if cpu and rank == 0 and world == 1 and not args.no_cpu_baseline:
        m, re, we, dx, length = specs[0]
        cpu_line = cpu_baseline(ensemble_case(m, re, we, dx, length, args.skin), args.cpu_seconds)
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "ensemble_c4: 64 planar jets, Re in %s x We in %s, "
                                   "dx = D/30 .. D/80, 20k-400k particles each, Wendland, "
                                   "FP32 pair sums / FP64 positions, adaptive dt per member"
                                   % (ENS_RE, ENS_WE),
                       "members_per_gpu": len(sims), "particles_total": 0.5 * (n0 + n1),
                       "parallelism": "members round-robin over ranks (no exchange)",
                       "l2": "inputs larger than L2 (all members resident, several GB)",
                       "tuning": {"lanes": lanes, "cadence": cadence,
                                  "start_form": FORM_NAMES[form], "skin_over_h": args.skin,
                                  "chosen_by": "ensemble autotuner" if args.tune == "auto"
                                  else "flag"},
                       "plain_value": plain_value,
                       "batched_over_plain": value / plain_value,
                       "plain_how": "each member's own step graph, members one after "
                                    "another on the same stream",
                       "wall_s": wall},
            "roofline": {"kernel": "whole ensemble step (all kernels)", "bound": "alu",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "peak_source": peak_source,
                         "algorithmic_per_particle_step": flop_ps,
                         "pairs_per_particle": pairs_pp},
            "measured_peaks": peaks,
            "cpu_baseline": cpu_line,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d / Ke,
                    "d2h_bytes_per_step": d2h / Ke,
                    "how": "sph_set_state of every member from pinned host arrays, %d "
                           "ensemble steps, sph_get_state of every member; host wall clock"
                           % Ke},
            "gpu_launches": launches,
            "clocks": clk,
            "breakup_L_over_D_mean": float(np.mean(Ls)),
        }
        # flat copies of the keys the plain line quotes
        line["workload"] = line["config"]["workload"]
        line["plain_value"] = line["config"]["plain_value"]
        line["batched_over_plain"] = line["config"]["batched_over_plain"]
        line["particles_total"] = line["config"]["particles_total"]
        line["tuning"] = line["config"]["tuning"]
        if emit:
            print(json.dumps({k: v for k, v in line.items()
                              if k not in ("workload", "plain_value", "batched_over_plain",
                                           "particles_total", "tuning")}), flush=True)
    ens.close()
    for sm in sims:
        sm.close()
    return line


# Learned-surrogate workload: training jets on the ensemble's Re x We grid and
# 16 held-out (Re, We) pairs between its grid points at about 200k particles.
SUR_TRAIN = [(100, 5), (200, 20), (400, 40), (700, 10), (1000, 60), (1500, 15), (2000, 30),
             (3000, 50)]
SUR_HELD_RE = [150, 300, 550, 850, 1250, 1750, 2500, 2750]
SUR_HELD_WE = [7.5, 25.0]
SUR_K = 4


def bench_surrogate_step(args, binding, dev, rank, local):
    """The cost of one surrogate step against k plain steps on one C5-shaped
    member (a 200k-particle held-out jet at D/60), every step accepted
    (threshold 1e30) and the network untrained: the speed of the path, apart
    from how often the judge accepts (which surrogate_c5 measures)."""
    import torch
    dx = 1.0 / 60
    case = wl.jet(seed=201, Re=300, We=7.5, dx=dx, length=200000 * dx * dx, kernel="wendland",
                  prec="fp32", capacity_factor=1.15)
    case["params"]["skin_over_h"] = 0.3
    stream = torch.cuda.Stream(device=dev)
    sim = binding.Simulation(case, stream=stream.cuda_stream, device=local)
    sim.set_tuning(2, 8)
    sim.run(20)
    n = sim.time()["n"]
    net = binding.Mpnn(case["params"]["capacity"], local)
    net.set_params(wl.mpnn_init(7))
    K = max(4, min(args.steps, 200) // SUR_K * SUR_K)
    for _ in range(max(args.warmup, 3)):
        binding.sph_surrogate_step(sim.ctx, net.net, SUR_K, 1.0, 0.04, 1e30, True)
    sim.run(SUR_K * max(args.warmup, 3))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    sim.run(K)
    torch.cuda.synchronize(dev)
    plain_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    for _ in range(K // SUR_K):
        binding.sph_surrogate_step(sim.ctx, net.net, SUR_K, 1.0, 0.04, 1e30, True)
    torch.cuda.synchronize(dev)
    sur_s = time.perf_counter() - t0
    net.close()
    sim.close()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": n * K / sur_s, "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": 1e3 * sur_s / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "surrogate_step: one planar jet, Re=300, We=7.5, dx = D/60, "
                                   "%d particles; k = %d substeps per surrogate step, every "
                                   "step accepted, untrained network" % (n, SUR_K),
                       "plain_value": n * K / plain_s, "surrogate_over_plain": plain_s / sur_s,
                       "ms_per_surrogate_step": 1e3 * sur_s / (K // SUR_K),
                       "ms_per_plain_step": 1e3 * plain_s / K,
                       "timing": "host wall clock with device synchronisation around each arm"},
        }), flush=True)


def bench_surrogate(args, binding, dist, dev, rank, world, local):
    """Plain SPH (the 16 held-out members as one batched ensemble) against
    surrogate steps (k = 4 substeps per step, plain SPH as judge and fallback
    at the residual threshold) on the same members, after training the
    network on the GPU from plain trajectories of the training jets."""
    import torch
    from paper_1603_02421_gb300 import surrogate as sg
    from paper_1603_02421_gb300.replicas import rank_members, reduce_rate

    def jet_case(seed, re, we, dx, n_target):
        case = wl.jet(seed=seed, Re=re, We=we, dx=dx, length=n_target * dx * dx,
                      kernel="wendland", prec="fp32", capacity_factor=1.15)
        case["params"]["skin_over_h"] = args.skin
        return case

    # ---- training (plain trajectories -> samples -> GPU training) ----------
    t_tr = time.perf_counter()
    train_cases = [jet_case(100 + i, re, we, 1.0 / 60, 50000)
                   for i, (re, we) in enumerate(SUR_TRAIN)]
    data = [(ci, smp) for ci, c in enumerate(train_cases)
            for smp in sg.collect(c, 10, every=10, k=SUR_K, warm=20)]
    a_ref = sg.a_scale([smp for _, smp in data])
    held_all = [(200 + 2 * i + j, re, we) for i, re in enumerate(SUR_HELD_RE)
                for j, we in enumerate(SUR_HELD_WE)]
    mine = [held_all[m] for m in rank_members(rank, world, len(held_all))]
    held_cases = [jet_case(seed, re, we, 1.0 / 60, 200000) for seed, re, we in mine]
    cap = max(c["params"]["capacity"] for c in train_cases + held_cases)
    tr = sg.Trainer(train_cases, cap)
    losses = tr.train(data, a_ref, seconds=args.train_seconds, lr=1e-3)
    params = tr.net.params()
    tr.close()
    train_s = time.perf_counter() - t_tr
    # held-out prediction errors (network vs the SPH acceleration alone)
    test = [(ci, smp) for ci, c in enumerate(held_cases[:2])
            for smp in sg.collect(c, 2, every=10, k=SUR_K, warm=20, end_accel=True)]
    # the judge's residuals of the exact k-step mean of plain SPH: the lowest
    # any predictor can score (momentum balance: the judged one; acceleration
    # field: reported only)
    floor_m = sg.momentum_floor([smp for _, smp in test])
    floor_f = sg.residual_floor([smp for _, smp in test])
    floor_d = sg.density_floor([smp for _, smp in test], held_cases[0]["params"]["rho0"])
    ev = sg.Trainer(held_cases[:2], cap)
    ev.net.set_params(params)
    e_net, e_an = ev.prediction_errors(test, a_ref)
    ev.close()

    # ---- plain arm: the held-out members as one batched ensemble ----------
    K = min(args.steps, 400)
    K -= K % SUR_K
    stream = torch.cuda.Stream(device=dev)
    sims = [binding.Simulation(c, stream=stream.cuda_stream, device=local) for c in held_cases]
    for sm in sims:
        sm.set_tuning(2, 8)
    ens = binding.Ensemble(sims, stream=stream.cuda_stream)
    ens.run(max(args.warmup, 3))
    start = [binding.sph_get_state(sm.ctx) for sm in sims]
    n0 = sum(sm.time()["n"] for sm in sims)
    t_start = [sm.time()["t"] for sm in sims]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    ens.run_async(K)
    e1.record(stream)
    ens.sync()
    torch.cuda.synchronize(dev)
    plain_s = e0.elapsed_time(e1) / 1e3
    L_plain = [binding.sph_breakup_length(sm.ctx)[0] for sm in sims]
    plain_value, _, _ = reduce_rate(plain_s, n0 * K, dist, dev)
    t_plain = [sm.time()["t"] - t0_ for sm, t0_ in zip(sims, t_start)]

    # ---- surrogate arm: the same members from the same states (the state
    # is replaced; the simulated time runs on, so spans are differences) ----
    t_sur0 = []
    for sm, st in zip(sims, start):
        binding.sph_set_state(sm.ctx, st)
        t_sur0.append(sm.time()["t"])
    net = binding.Mpnn(cap, local)
    net.set_params(params)
    clocks = ClockSampler(local)
    accepted = steps = rejected_lists = 0
    rms, rds, rfs = [], [], []
    ctxs = [sm.ctx for sm in sims]
    builds0 = sum(binding.sph_get_rebuild_stats(c)[0] for c in ctxs)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(K // SUR_K):
        ok, rm, rd, rf = ens.surrogate_step(net.net, SUR_K, 1.0, a_ref, args.threshold)
        accepted += int(ok.sum())
        steps += len(ctxs)
        # rejected with both residuals within the threshold: the particles
        # moved too far for the start's neighbour lists
        rejected_lists += int(np.sum(~ok & (rm <= args.threshold) & (rd <= args.threshold)))
        rms.extend(rm.tolist())
        rds.extend(rd.tolist())
        rfs.extend(rf.tolist())
    torch.cuda.synchronize(dev)
    sur_s = time.perf_counter() - t0
    fresh_starts = sum(binding.sph_get_rebuild_stats(c)[0] for c in ctxs) - builds0
    clk = clocks.stop()
    L_sur = [binding.sph_breakup_length(sm.ctx)[0] for sm in sims]
    t_sur = [sm.time()["t"] - t0_ for sm, t0_ in zip(sims, t_sur0)]
    value, total_s, _ = reduce_rate(sur_s, n0 * K, dist, dev)
    per_full = binding.sph_kernel_counts(sims[0].ctx)[0]
    # a surrogate step launches 13 kernels when it starts from the last
    # evaluation (network 5, mean, update, spawn, refresh, 3 SPH sweeps,
    # residual), 9 more (sort 5, lists, 3 sweeps) when it starts afresh; a
    # rejected one adds k plain steps (whose rebuilds are counted as starts)
    launches = steps * 13 + fresh_starts * 9 + (steps - accepted) * SUR_K * per_full

    # ---- end to end: host state in, surrogate steps, host state out -------
    Ke = 5
    pinned = [{k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy()
               for k, v in st.items()} for st in start]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for sm, st in zip(sims, pinned):
        binding.sph_set_state(sm.ctx, st)
    for _ in range(Ke):
        ens.surrogate_step(net.net, SUR_K, 1.0, a_ref, args.threshold)
    for sm in sims:
        binding.sph_get_state(sm.ctx)
    ens.close()
    e2e_s = time.perf_counter() - t0
    e2e_value, _, _ = reduce_rate(e2e_s, n0 * Ke * SUR_K, dist, dev)
    h2d = n0 * (16 + 8 + 4 + 4 + 4 + 1 + 4)
    d2h = n0 * (16 + 8 + 4 + 4 + 1 + 4 + 8 + 4)
    net.close()

    # network GEMM work per surrogate step on the tensor cores (BF16)
    tensor_flop = 2.0 * 3 * (128 * 32 + 256 * 128) * n0 * (K // SUR_K)
    bf16, bf16_src = pool_peak("bf16_tflops")
    achieved = tensor_flop / sur_s / 1e12
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = oracle_sample(held_cases[0], 20000)
        psteps, nsteps, el, n = run_oracle(sample, args.cpu_seconds)
        cpu = {"value": psteps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "FP64 CPU oracle (single thread), %d steps of the upstream %d "
                         "particles of held-out member 0, %.1f s" % (nsteps, n, el)}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "surrogate_c5: 16 held-out planar jets, Re in %s x We in %s, "
                                   "dx = D/60, ~200k particles each; network trained on 8 jets "
                                   "of the Re x We grid at D/60, 50k particles each"
                                   % (SUR_HELD_RE, SUR_HELD_WE),
                       "members_per_gpu": len(sims), "particles_total": n0,
                       "k_substeps": SUR_K, "threshold": args.threshold,
                       "surrogate_steps": steps, "accepted": accepted,
                       "fresh_starts": fresh_starts,
                       "rejected_by_residual": steps - accepted - rejected_lists,
                       "rejected_by_lists": rejected_lists,
                       "acceptance_rate": accepted / max(steps, 1),
                       "residual_median": {
                           "momentum": float(np.median(rms)) if rms else None,
                           "density": float(np.median(rds)) if rds else None,
                           "field_reported_only": float(np.median(rfs)) if rfs else None},
                       "residual_floor": {
                           "momentum": float(np.median(floor_m)),
                           "density": float(np.median(floor_d)),
                           "field_reported_only": float(np.median(floor_f)),
                           "how": "median over held-out samples of the residuals scored by "
                                  "the exact 4-step mean acceleration of plain SPH"},
                       "prediction_error_heldout": {"network": e_net, "sph_acceleration_only": e_an},
                       "training": {"seconds": train_s, "passes": len(losses),
                                    "samples": len(data), "final_loss": losses[-1],
                                    "a_ref": a_ref},
                       "plain_value": plain_value, "surrogate_over_plain": value / plain_value,
                       "plain_how": "the same members as one batched ensemble, K plain steps",
                       "simulated_time_span": {"plain_mean": float(np.mean(t_plain)),
                                               "surrogate_mean": float(np.mean(t_sur))},
                       "breakup_L_over_D_mean": {"plain": float(np.mean(L_plain)),
                                                 "surrogate": float(np.mean(L_sur))},
                       "l2": "inputs larger than L2 (all members resident)"},
            "roofline": {"kernel": "BF16 tensor-core GEMMs of the network (whole surrogate-arm time)",
                         "bound": "tensor", "achieved": achieved, "peak": bf16,
                         "unit": "TFLOP/s", "frac": achieved / bf16,
                         "traffic": None,
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (%s)" % bf16_src},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d / (Ke * SUR_K),
                    "d2h_bytes_per_step": d2h / (Ke * SUR_K),
                    "how": "sph_set_state of every member from pinned host arrays, %d "
                           "ensemble surrogate steps of %d substeps, sph_get_state of every "
                           "member; host wall clock" % (Ke, SUR_K)},
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    for sm in sims:
        sm.close()


if __name__ == "__main__":
    main()
