#!/usr/bin/env python3
"""Throughput of the hybrid symplectic step (FP64 particle-steps/s).

Workload (one GPU): 4 giant cores (10-30 Earth masses, a in [3, 10] AU) and
100,000 gas-dragged planetesimals (a in [1, 15] AU, radius 1-100 km), power-law
gas disk Sigma = 1700 (r/AU)^-1 g/cm^2, H/r = 0.05 (r/AU)^0.25, dt = 10 days;
seeded synthetic inputs (paper_2601_16791_gb300.workloads.gas_4core_100k).

A timed step is one full hybrid step (half kick with drag, jump, Kepler drift,
encounter detection, Bulirsch-Stoer of the flagged groups, jump, half kick).
The K steps run through the production CUDA graphs of mx_step, enqueued back to
back with an L2 flush (201 MB write) before every step, followed by the
catch-up that brings every deferred planetesimal to the last step
(planetesimals whose encounter outlasts one Bulirsch-Stoer macro sub-step are
replayed from the big bodies' recorded history; long encounters continue on a
side stream while the next window runs).  The value is N K over that span's
device time minus the K flushes, timed alone right after.  Per-kernel times
come from a second pass of K steps with events between kernels.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank integrates its own disk (seed offset by rank; weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64 particle-steps/s at N=100k (plain vs batched), % FP64 peak; adjoint/fwd cost"
UNIT = "particle-steps/s"
WORKLOAD = "gas_4core_100k"

# Algorithmic FP64 work per unit (flops; FMA = 2, sqrt/div/transcendental = 1):
FLOPS_PAIR_KICK = 20       # K-weighted pair force, per (target, big) pair
FLOPS_DRAG = 88            # drag of one planetesimal: ~80 + pow, exp, 3 sqrt, 3 div
FLOPS_KICK_UPDATE = 9      # v += (h/2)(a_grav + a_drag)
FLOPS_JUMP = 3             # x += (h/2) P/m0
FLOPS_DRIFT = 340          # universal-variable solve: ~60 x 5 iterations + Stumpff ~40
FLOPS_DETECT_PAIR = 30     # endpoint distances and slopes, per (target, big) pair
# one force evaluation of a two-body Bulirsch-Stoer group (a planetesimal and
# a big body) with the Stoermer update: two star terms (12 each), the big
# body's (1-K)-weighted pull on the planetesimal (20), their sum (3), and the
# update D += d^2 A, X += D of both bodies (18); the massless body's pull on
# the big body is zero and not counted
FLOPS_BS2_FEVAL = 65
FLUSH_BYTES = 192 << 20    # L2 flush between steps: 201 MB written, 1.56x the 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="mx", choices=["mx", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the ensemble and adjoint legs")
    ap.add_argument("--ensemble-steps", type=int, default=30)
    ap.add_argument("--legs", default="batched,adjoint,ejection,growth,semiactive",
                    help="comma-separated extra legs to run")
    ap.add_argument("--budget-s", type=float, default=120.0,
                    help="reference arm: host seconds the warm-up and timed steps may take")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="another named workload (informational; the metric is quoted on the default)")
    ap.add_argument("--window", type=int, default=None,
                    help="deferral window in steps (default: the library's)")
    ap.add_argument("--tiling", default=None,
                    help="tile,order to override the autotuner (order 2: tiles per SM)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.idx), "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------- baselines
def oracle_rate(workload, target_s, warm_steps=1, threads=None):
    """Oracle particle-steps/s on the host cores (all, or `threads`) over a
    bounded sample of the workload: every big body plus a prefix of the
    planetesimals."""
    import oracle as orc
    cores = threads or os.cpu_count() or 1
    orc.set_threads(cores)
    w = workload

    def sample(ns):
        cols = np.concatenate([np.arange(w.nbig), w.nbig + np.arange(ns)])
        return cols

    # size the sample so that one step takes ~0.5 s
    ns = min(w.nsmall, 2000)
    p = orc.make_params(w.params)
    while True:
        cols = sample(ns)
        xv, mu, rc = orc.init(p, w.nbig, ns, w.m_big, w.xv_helio[:, cols])
        t0 = time.perf_counter()
        orc.step(p, w.nbig, xv, mu, rc, w.rp_km[:ns], w.rhop[:ns], 1)
        dt = time.perf_counter() - t0
        if dt > 0.3 or ns >= w.nsmall:
            break
        ns = min(w.nsmall, ns * 4)
    nsteps = max(1, int(target_s / max(dt, 1e-6)))
    for _ in range(warm_steps):
        xv, _, _, _ = orc.step(p, w.nbig, xv, mu, rc, w.rp_km[:ns], w.rhop[:ns], 1)
    t0 = time.perf_counter()
    xv, _, _, _ = orc.step(p, w.nbig, xv, mu, rc, w.rp_km[:ns], w.rhop[:ns], nsteps)
    el = time.perf_counter() - t0
    n = w.nbig + ns
    return {"value": n * nsteps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{w.nbig} bigs + {ns} of {w.nsmall} planetesimals, {nsteps} steps, "
                      f"{el:.1f} s"}, n, el / nsteps


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2601_16791_gb300 import workloads as W
    import oracle as orc
    w = W.make(WORKLOAD)
    cores = os.cpu_count() or 1
    orc.set_threads(cores)
    # bound the sample so W + K steps take about --budget-s seconds
    budget_s = args.budget_s
    per_step_target = budget_s / max(1, args.steps + args.warmup)
    ns = 256
    p = orc.make_params(w.params)
    while True:
        cols = np.concatenate([np.arange(w.nbig), w.nbig + np.arange(ns)])
        xv, mu, rc = orc.init(p, w.nbig, ns, w.m_big, w.xv_helio[:, cols])
        t0 = time.perf_counter()
        orc.step(p, w.nbig, xv, mu, rc, w.rp_km[:ns], w.rhop[:ns], 1)
        dt = time.perf_counter() - t0
        if dt * 2 > per_step_target or ns >= w.nsmall:
            break
        ns = min(w.nsmall, ns * 2)
    xv, _, _, _ = orc.step(p, w.nbig, xv, mu, rc, w.rp_km[:ns], w.rhop[:ns], args.warmup)
    t0 = time.perf_counter()
    xv, _, _, _ = orc.step(p, w.nbig, xv, mu, rc, w.rp_km[:ns], w.rhop[:ns], args.steps)
    el = time.perf_counter() - t0
    n = w.nbig + ns
    value = n * args.steps / el
    sample = f"{w.nbig} cores + first {ns} of {w.nsmall} planetesimals per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": bench_config(w),
            "reference": "CPU FP64 oracle (oracle/mx_oracle.cpp), OpenMP over targets",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(r4(line), separators=(",", ":")), flush=True)


# ---------------------------------------------------------------- roofline
def kernel_flops(kname, w, launches, nsteps):
    """Algorithmic FP64 flops of all launches of one kernel in the timed region."""
    nb, ns, n = w.nbig, w.nsmall, w.n
    if kname == "k_jump_kick":
        # gravity once per launch; drag and velocity update once per half kick
        # (two per step, however the launches split them); the jump once per step
        kicks = 2 * nsteps
        grav = launches * (ns * nb + nb * (nb - 1)) * FLOPS_PAIR_KICK
        drag = kicks * ns * FLOPS_DRAG * (1 if w.params["gas"]["enabled"] else 0)
        return grav + drag + kicks * n * FLOPS_KICK_UPDATE + FLOPS_JUMP * n * nsteps
    # k_jump_drift: no rate.  FLOPS_DRIFT counts a plain solver's 4-6 Newton
    # iterations, where the kernel makes one Halley correction on these disks,
    # so a rate against the peak would not measure executed work (its FP64
    # pipe occupancy is in the ncu summary instead).
    if kname == "k_detect":
        return FLOPS_DETECT_PAIR * (ns * nb + nb * (nb - 1) // 2) * launches
    return None


def catchup_flops(w, ops):
    """Algorithmic FP64 flops of catch-up work counted on the device
    (mx_catchup_work): body-slots through jump + drift + encounter test, half
    kicks of one body (gravity of every big body, drag, update), two-body
    Bulirsch-Stoer force evaluations of the one-try-at-a-time search."""
    slots, kicks, fevals = ops
    nb = w.nbig
    drag = FLOPS_DRAG if w.params["gas"]["enabled"] else 0
    return (slots * (FLOPS_JUMP + FLOPS_DRIFT + nb * FLOPS_DETECT_PAIR)
            + kicks * (nb * FLOPS_PAIR_KICK + drag + FLOPS_KICK_UPDATE)
            + fevals * FLOPS_BS2_FEVAL)


def source_hash(names):
    h = hashlib.sha256()
    for nm in names:
        h.update(open(os.path.join(ROOT, "paper_2601_16791_gb300", "csrc", nm), "rb").read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = {"k_jump_kick": ["k_kick.cu", "mx_kick_body.cuh", "mx_common.cuh", "mx_physics.cuh",
                                  "mx_growth.cuh"],
                  "k_jump_drift": ["k_drift.cu", "mx_drift_body.cuh", "mx_common.cuh", "mx_kepler.cuh"],
                  "k_detect": ["k_detect.cu", "mx_detect_body.cuh", "mx_common.cuh",
                               "mx_encounter.cuh"],
                  "k_bs": ["k_bs.cu", "mx_bs.cuh", "mx_common.cuh", "mx_physics.cuh"],
                  "k_catchup": ["k_bs.cu", "mx_bs.cuh", "mx_common.cuh", "mx_physics.cuh",
                                "mx_kepler.cuh", "mx_encounter.cuh"]}


def dram_traffic(kname):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel's
    source still matches the one that was profiled."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path) or kname not in KERNEL_SOURCES:
        return None
    rec = json.load(open(path)).get(kname)
    if not rec or rec.get("source_sha") != source_hash(KERNEL_SOURCES[kname]):
        return None
    return rec.get("bytes_per_launch")


# ------------------------------------------------------------ multi-rank
def rank_seed(rank):
    """Each rank integrates its own disk: same workload, seed offset by rank."""
    return 1 + rank


def reduce_max(x, device):
    """Max over ranks of a host float (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(bodies_per_rank, steps, world, t_max_s):
    """Units all ranks processed divided by the slowest rank's time."""
    return world * bodies_per_rank * steps / t_max_s


# ------------------------------------------------- ensemble and adjoint legs
def ensemble_leg(steps, nsys=256):
    """256 systems (2-50 embryos, 1e3-2e5 planetesimals each, gas with Sigma
    x U[0.3, 3]): one batched mx_system (per-kernel step graphs, then one
    persistent launch per interior step) vs a host loop calling mx_step on
    one mx_system per system.  Each advances every system by `steps` steps."""
    import torch
    from paper_2601_16791_gb300 import mx, workloads as W
    ws = W.ensemble_256(nsys=nsys)
    n_tot = sum(w.n for w in ws)
    st = torch.cuda.current_stream()
    b = mx.Batch(ws, stream=st.cuda_stream)
    tile, order = mx.mx_tiling(b.h)
    b.step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(steps)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    # the same steps with every interior step as one persistent launch
    mx.mx_set_persistent(b.h, True)
    b.step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(steps)
    torch.cuda.synchronize()
    t_persist = time.perf_counter() - t0
    b.close()
    systems = [mx.System(w, stream=st.cuda_stream) for w in ws]
    for s in systems:
        s.step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        for s in systems:
            s.step(1)
    torch.cuda.synchronize()
    t_loop = time.perf_counter() - t0
    for s in systems:
        s.close()
    return {"n_systems": nsys, "n_bodies": n_tot, "steps": steps,
            "batched_value": n_tot * steps / t_batch, "loop_value": n_tot * steps / t_loop,
            "persistent_value": n_tot * steps / t_persist,
            "speedup": t_loop / t_batch, "speedup_persistent": t_loop / t_persist,
            "tile": [tile, order]}


def adjoint_leg(nsteps=200, every=50):
    """Cost of the hand-written adjoint on the adjoint workload (4 cores +
    50,000 planetesimals with gas): bwd_over_fwd, the autograd backward's wall
    time over its forward run's; from one state, one adjoint step against one
    forward step (fwd_ms, mx_step(1)) with the groups skipped (adjoint_step_ms,
    adjoint_over_forward_step) and through every group (groups_ms,
    groups_ratio); and consecutive steps as the backward runs them, merged and
    from the forward's pre-drift states (run_ms, run_ratio)."""
    import torch
    from paper_2601_16791_gb300 import mx, workloads as W
    from paper_2601_16791_gb300.autograd import Trajectory, semimajor_loss
    w = W.adjoint_4core_50k(nsteps=nsteps, checkpoint_every=every)
    traj = Trajectory(w, stream=torch.cuda.current_stream().cuda_stream)
    g = w.params["gas"]
    xv0 = torch.tensor(w.xv_helio, dtype=torch.float64, device="cuda", requires_grad=True)
    gas = torch.tensor([g["sigma1_gcm2"], g["gamma"], g["cd_scale"]], dtype=torch.float64,
                       device="cuda", requires_grad=True)
    wts = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    wts[w.nbig:] = 1.0 / w.nsmall
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L = semimajor_loss(traj, xv0, gas, wts, nsteps, every)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    L.backward()
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    # one forward step and one adjoint step, same state, CUDA events
    z = torch.empty((6, w.n), dtype=torch.float64, device="cuda")
    mx.mx_get_state_device(traj.h, z)
    lam = torch.randn((6, w.n), dtype=torch.float64, device="cuda")
    dpar = torch.zeros(3, dtype=torch.float64, device="cuda")
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    reps = 20
    mx.mx_step(traj.h, 1)
    e[0].record()
    for _ in range(reps):
        mx.mx_set_state_device(traj.h, z)
        mx.mx_step(traj.h, 1)
    e[1].record()
    e[2].record()
    mx._check(mx.load().mx_adjoint_encounters(traj.h, 0), "mx_adjoint_encounters")
    for _ in range(reps):
        mx.mx_adjoint_step(traj.h, z, 0, lam, dpar)
    e[3].record()
    # the same step differentiated through its encounter groups
    e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mx._check(mx.load().mx_adjoint_encounters(traj.h, 1), "mx_adjoint_encounters")
    e4.record()
    for _ in range(reps):
        mx.mx_adjoint_step(traj.h, z, 0, lam, dpar)
    e5.record()
    torch.cuda.synchronize()
    f_ms = e[0].elapsed_time(e[1]) / reps
    a_ms = e[2].elapsed_time(e[3]) / reps
    g_ms = e4.elapsed_time(e5) / reps
    m_ms = merged_adjoint_ms(traj.h, w.n, z, 0)
    traj.close()
    return {"steps": nsteps, "every": every, "bwd_over_fwd": t_bwd / t_fwd, "fwd_ms": f_ms,
            "adjoint_step_ms": a_ms, "adjoint_over_forward_step": a_ms / f_ms,
            "groups_ms": g_ms, "groups_ratio": g_ms / f_ms, "run_ms": m_ms, "run_ratio": m_ms / f_ms}


def eject_leg(steps=200):
    """The ejection test of Sec. 3.5 on the gas disk (4 cores + 100,000
    planetesimals): step time with the test after every step and without it,
    the test's own launch time against the bytes it must read (the 6 state
    doubles and 2 status bytes of every body), and one element conversion of
    every body (mx_elements: momentum + k_elements)."""
    import torch
    from paper_2601_16791_gb300 import mx, workloads as W
    st = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = {"steps": steps}
    for every in (0, 1):
        w = W.make(WORKLOAD)
        w.params = dict(w.params, eject_every=every)
        s = mx.System(w, stream=st.cuda_stream)
        mx.mx_step_timed(s.h, 5, flush)
        mx.mx_step_timed(s.h, 0, flush)
        ms, cnt, tot = mx.mx_step_timed(s.h, steps, flush)
        _, _, tot0 = mx.mx_step_timed(s.h, 0, flush)
        key = "every_step" if every else "none"
        out[f"ms_per_step_{key}"] = (tot + tot0) / steps
        if every:
            n_launch = max(1, cnt["k_eject"])
            t = ms["k_eject"] / n_launch
            out["k_eject_us"] = 1e3 * t
            out["removed"] = int(mx.mx_body_status(s.h, w.n)[1][0])
            el = torch.empty((6, w.n), dtype=torch.float64, device="cuda")
            mx.mx_elements(s.h, el)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(20):
                mx.mx_elements(s.h, el)
            e1.record()
            torch.cuda.synchronize()
            out["elements_us"] = 1e3 * e0.elapsed_time(e1) / 20
        s.close()
    out["test_overhead_per_step"] = out["ms_per_step_every_step"] / out["ms_per_step_none"] - 1.0
    return out


def merged_adjoint_ms(h, n, z, mode, k=4):
    """Per-step time of the reverse of k consecutive steps from state z as
    the autograd backward runs it: mx_adjoint_merge on (each step's first half
    kick shares its pair pass with the previous step's last) and each step's
    pre-drift state from the forward (mx_adjoint_step_predrift), the final
    pending pass included."""
    import torch
    from paper_2601_16791_gb300 import mx
    seg, pre = [], []
    mx.mx_set_state_device(h, z)
    for _ in range(k):
        zi = torch.empty_like(z)
        mx.mx_get_state_device(h, zi)
        seg.append(zi)
        mx.mx_step(h, 1)
        pre.append(torch.empty_like(z))
        mx.mx_predrift_state(h, pre[-1])
    lam = torch.randn(z.shape, dtype=torch.float64, device="cuda",
                      generator=torch.Generator(device="cuda").manual_seed(6))
    dpar = torch.zeros(3, dtype=torch.float64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mx._check(mx.load().mx_adjoint_encounters(h, mode), "mx_adjoint_encounters")
    mx.mx_adjoint_merge(h, True)
    for rep in range(2):   # the first pass warms up
        if rep == 1:
            e0.record()
        for i in reversed(range(k)):
            mx.mx_adjoint_step_predrift(h, seg[i], pre[i], i, lam, dpar)
        mx.mx_adjoint_flush(h)
    e1.record()
    torch.cuda.synchronize()
    mx.mx_adjoint_merge(h, False)
    return e0.elapsed_time(e1) / k


def semiactive_adjoint(s, w, reps=3):
    """One adjoint step against one forward step (mx_step(1): both half
    kicks) from the same state of the semi-active disk: with the groups of
    big bodies only (mode 2, the masked loss) and through every group; and the
    per-step cost of consecutive steps reversed with mx_adjoint_merge (mode 2)."""
    import torch
    from paper_2601_16791_gb300 import mx
    z = torch.empty((6, w.n), dtype=torch.float64, device="cuda")
    mx.mx_get_state_device(s.h, z)
    lam = torch.randn((6, w.n), dtype=torch.float64, device="cuda",
                      generator=torch.Generator(device="cuda").manual_seed(5))
    dpar = torch.zeros(3, dtype=torch.float64, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    mx.mx_set_state_device(s.h, z)
    mx.mx_step(s.h, 1)
    ev[0].record()
    for _ in range(reps):
        mx.mx_set_state_device(s.h, z)
        mx.mx_step(s.h, 1)
    ev[1].record()
    for mode, (a, b) in ((2, (2, 3)), (1, (4, 5))):
        mx._check(mx.load().mx_adjoint_encounters(s.h, mode), "mx_adjoint_encounters")
        mx.mx_adjoint_step(s.h, z, 0, lam, dpar)
        ev[a].record()
        for _ in range(reps):
            mx.mx_adjoint_step(s.h, z, 0, lam, dpar)
        ev[b].record()
    torch.cuda.synchronize()
    f_ms = ev[0].elapsed_time(ev[1]) / reps
    a_ms = ev[2].elapsed_time(ev[3]) / reps
    g_ms = ev[4].elapsed_time(ev[5]) / reps
    m_ms = merged_adjoint_ms(s.h, w.n, z, 2, k=8)
    return {"fwd_ms": f_ms, "adjoint_step_ms": a_ms, "adjoint_over_forward_step": a_ms / f_ms,
            "groups_ms": g_ms, "groups_ratio": g_ms / f_ms, "run_ms": m_ms, "run_ratio": m_ms / f_ms}


def semiactive_leg(steps=20):
    """The O(N_big N) regime: 2,000 embryos + 200,000 planetesimals (no gas),
    where the kick is gravity of 2,000 sources on every body.  Step time, the
    kick's algorithmic FP64 rate against the measured peak, and the cost of
    an adjoint step."""
    import torch
    from paper_2601_16791_gb300 import mx, workloads as W
    st = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    w = W.semiactive_2000big_200k()
    s = mx.System(w, stream=st.cuda_stream)
    peak = mx.mx_fp64_peak(st.cuda_stream, 200.0)
    mx.mx_step_timed(s.h, 3, flush)
    mx.mx_step_timed(s.h, 0, flush)
    ms, cnt, tot = mx.mx_step_timed(s.h, steps, flush)
    ms0, cnt0, tot0 = mx.mx_step_timed(s.h, 0, flush)
    tile, order = mx.mx_tiling(s.h)
    adj = semiactive_adjoint(s, w)
    s.close()
    out = {"n_bodies": w.n, "steps": steps, "ms_per_step": (tot + tot0) / steps,
           "value": w.n * steps / ((tot + tot0) * 1e-3)}
    out.update(adj)
    # (detection's count is per pair; its FP32 screen skips most of them, so
    # it is not a rate against the FP64 peak)
    for k, key in (("k_jump_kick", "kick_frac_of_peak"),):
        f = kernel_flops(k, w, cnt[k], steps)
        if f and ms[k] > 0:
            out[key] = f / (ms[k] * 1e-3) / 1e12 / peak
    out["tile"] = [tile, order]
    return out


def growth_leg(steps=200):
    """Planet growth and gaps (Secs. 3.1, 3.3) on the two-giant disk (2
    embryos + 24,000 planetesimals with gas; tracks compressed to tau_c =
    400 d, tau_g = 200 d so that the gaps are open in the timed steps 60-259):
    step time with the tracks, against the same system with the masses fixed
    at the tracks' values at step 60 (same encounters, no growth, no gaps),
    with the per-kernel split of both."""
    import torch
    from paper_2601_16791_gb300 import mx, workloads as W
    st = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = {"steps": steps}
    m60 = None
    for grow in (True, False):
        w = W.growth_2giant(tau_c_days=400.0, tau_g_days=200.0)
        s = mx.System(w, stream=st.cuda_stream)
        if grow:
            mx.mx_step_timed(s.h, 60, flush)
            mx.mx_step_timed(s.h, 0, flush)
            m60 = mx.mx_planets(s.h, w.nbig)[0]
        else:   # same start state, masses fixed at step 60's
            s.close()
            w.growth = None
            w.m_big = m60
            s = mx.System(w, stream=st.cuda_stream)
            mx.mx_step_timed(s.h, 60, flush)
            mx.mx_step_timed(s.h, 0, flush)
        ms, cnt, tot = mx.mx_step_timed(s.h, steps, flush)
        ms0, cnt0, tot0 = mx.mx_step_timed(s.h, 0, flush)
        key = "growth" if grow else "fixed_masses"
        out[f"ms_per_step_{key}"] = (tot + tot0) / steps
        if grow:
            out["k_prep_us"] = 1e3 * ms["k_prep"] / max(1, cnt["k_prep"])
        s.close()
    return out


# ------------------------------------------------------------------- main
def r4(x):
    """Rounds floats to 4 significant digits, recursively (a short JSON line)."""
    if isinstance(x, float):
        return float(f"{x:.4g}")
    if isinstance(x, dict):
        return {k: r4(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [r4(v) for v in x]
    return x


def bench_config(w, name=WORKLOAD):
    """The `config` of both arms (the same dict)."""
    return {"workload": name, "n_bodies": w.n,
            "l2": "201 MB flush before each timed step, subtracted (GPU arm)"}


def run_mx(args):
    import torch
    from paper_2601_16791_gb300 import mx, workloads as W
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    st = torch.cuda.current_stream()
    w = W.make(args.workload, seed=rank_seed(rank))
    sysm = mx.System(w, stream=st.cuda_stream)
    if args.tiling:
        mx.mx_set_tiling(sysm.h, *[int(v) for v in args.tiling.split(",")])
    if args.window is not None:
        mx.mx_set_defer_window(sysm.h, args.window)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    peak = mx.mx_fp64_peak(st.cuda_stream, 200.0)
    mx.mx_step_timed(sysm.h, args.warmup, flush)
    mx.mx_step_timed(sysm.h, 0, flush)   # no deferred work carries into the timed region
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    # The timed region: K steps through the production step graphs, enqueued
    # back to back, each preceded by an L2 flush, then the catch-up that
    # brings every deferred planetesimal to the last step (side stream joined),
    # as one span of device time; the K flushes are then timed alone and
    # subtracted.
    wall_ms, flush_ms = mx.mx_step_wall(sysm.h, args.steps, flush)
    torch.cuda.synchronize()
    dwin, dmax, _, _ = mx.mx_defer_stats(sysm.h)
    tiling = mx.mx_tiling(sysm.h)
    barrier()
    clk = clocks.stop()
    t_max = reduce_max(wall_ms - flush_ms, "cuda")
    value = whole_job_rate(w.n, args.steps, world, t_max * 1e-3)
    # the same K steps again (from where the region ended), through the step
    # graphs' variants with an event between kernels: each kernel's time and
    # launch count, and the catch-ups' device-counted work (event nodes add
    # about 7% to a step, so this pass is not the value)
    mx.mx_catchup_work(sysm.h, reset=True)
    kms = {k: 0.0 for k in mx.KERNELS}
    kcnt = {k: 0 for k in mx.KERNELS}
    kernel_total_ms = 0.0
    for n in (args.steps, 0):
        ms, cnt, tot = mx.mx_step_timed(sysm.h, n, flush)
        for k in mx.KERNELS:
            kms[k] += ms[k]
            kcnt[k] += cnt[k]
        kernel_total_ms += tot
    torch.cuda.synchronize()
    ops_main, ops_side = mx.mx_catchup_work(sysm.h)

    # end to end through the public API with host buffers: per step the state
    # goes host->device from pinned memory, one step runs, the state comes back
    # into the other pinned buffer, which feeds the next step
    L = mx.load()
    pins = [torch.empty((6, w.n), dtype=torch.float64, pin_memory=True) for _ in range(2)]
    pins[0].copy_(torch.from_numpy(sysm.state(mx.MX_COORD_DH)))
    stepc = ctypes.c_longlong(0)
    ne = max(1, args.e2e_steps)
    barrier()
    t0 = time.perf_counter()
    for k in range(ne):
        src, dst = pins[k & 1], pins[(k + 1) & 1]
        mx._check(L.mx_set_state(sysm.h, ctypes.c_void_p(src.data_ptr()), mx.MX_COORD_DH, k),
                  "mx_set_state")
        mx._check(L.mx_step(sysm.h, 1), "mx_step")
        mx._check(L.mx_get_state(sysm.h, ctypes.c_void_p(dst.data_ptr()), mx.MX_COORD_DH,
                                 ctypes.byref(stepc)), "mx_get_state")
    e2e_s = reduce_max(time.perf_counter() - t0, "cuda")
    e2e_value = whole_job_rate(w.n, ne, world, e2e_s)

    if rank != 0:
        sysm.close()
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    def flops_of(k):
        if k == "k_catchup":
            return catchup_flops(w, ops_main)
        if k == "k_catchup_side":
            return catchup_flops(w, ops_side)
        return kernel_flops(k, w, kcnt[k], args.steps)

    # dominant kernel on the step's critical path (the side-stream catch-up
    # overlaps the steps) and its roofline
    dom = max((k for k in kms if k != "k_catchup_side"), key=lambda k: kms[k])
    flops = flops_of(dom)
    avg_ms = kms[dom] / max(1, kcnt[dom])
    achieved = (flops / max(1, kcnt[dom])) / (avg_ms * 1e-3) / 1e12 if flops and avg_ms > 0 else None
    roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None, "traffic": dram_traffic(dom),
            "peak_source": "mx_fp64_peak, this run",
            "avg_launch_ms": avg_ms, "share_of_step": kms[dom] / max(1e-12, kernel_total_ms)}
    kern = {}
    for k in mx.KERNELS:
        if kcnt[k] == 0:
            continue
        row = [kms[k] / args.steps, kcnt[k]]
        fk = flops_of(k)
        if fk and kms[k] > 0:
            row.append(fk / (kms[k] * 1e-3) / 1e12 / peak)
        kern[k] = row
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(w, args.workload),
            "timing": {"wall_ms": wall_ms, "flush_ms": flush_ms, "defer_window": dwin,
                       "tile": list(tiling)},
            "roofline": roof, "clocks": clk,
            "kernels": kern,
            "gpu_launches": int(sum(kcnt.values())),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 48 * w.n,
                    "d2h_bytes_per_step": 48 * w.n, "steps": ne}}
    sysm.close()
    if not args.no_extra:
        for key, fn in (("batched", lambda: ensemble_leg(args.ensemble_steps)),
                        ("adjoint", adjoint_leg), ("ejection", eject_leg),
                        ("growth", growth_leg), ("semiactive", semiactive_leg)):
            if key not in args.legs.split(","):
                continue
            try:
                line[key] = fn()
            except Exception as exc:  # reported, not hidden
                line[key] = {"error": str(exc)[:120]}
    if not args.no_cpu_baseline:
        one, _, _ = oracle_rate(w, 3.0, threads=1)
        cb, _, _ = oracle_rate(w, 12.0)
        cb["single_thread"] = one["value"]
        line["cpu_baseline"] = cb
    if world > 1:
        torch.distributed.destroy_process_group()
    print(json.dumps(r4(line), separators=(",", ":")), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_mx(args)


if __name__ == "__main__":
    main()
