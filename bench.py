"""Benchmark of the WCSPH hot path on GB300 (one JSON line on rank 0).

Default workload: the 3-D dam break at dp = 0.004 m (1,000,000 fluid +
479,826 boundary particles, cells of h), stepped with the Symplectic scheme
over the neighbour list kept across steps.  A "step" is one full Symplectic
step: NL (when the list needs a rebuild) -> PI -> dt -> predictor -> PI ->
corrector.  The metric is particle interactions per second (ordered pairs
evaluated by the two PI evaluations of each step, the paper's PIPS); steps/s
is reported beside it.  The default line also carries, measured in the same
run: the roofline of the interaction kernel against the FP32 throughput
measured on this GPU, the case's whole 2,000-step run (its own list-rebuild
rate), the batched execution of the 256 dam breaks against one case at a
time, a scaled serving trace against one request at a time, the end-to-end
figure through the C ABI from pinned host memory, and the FP64 oracle on the
host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload dam_break|dam_break_small|wave_flume|batched|served]

Under torchrun each rank runs its own replica of the workload (independent
cases, no data-path collective): "scaling": "weak".
"""
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

import numpy as np  # noqa: E402

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Algorithmic FLOPs per evaluated pair (each +, -, *, comparison, sqrt and
# reciprocal counts 1; a fused multiply-add counts 2), counted operation by
# operation on the pair formula of Eq 11, 15, 17-18, 21-22 and 35:
F_PAIR_FF = 48   # a in F, b in F: momentum + viscosity + continuity + DDT + Eq 35 max
F_PAIR_FB = 45   # a in F, b in B: as above without density diffusion
F_PAIR_BF = 25   # a in B, b in F: continuity of Eq 36 only
# Eq 19-20 adds, per fluid-fluid pair: g . r_ab (5), P^H / B -> (1 + x)^(1/gamma)
# as log, multiply, exp (3), times rho0 minus rho0 (2), minus from rho_b - rho_a (1)
F_PAIR_FF_HYD = F_PAIR_FF + 11
# Laminar + SPS (Eq 23-27) adds, per pair with a in F: Eq 23 (9), Eq 26 with
# the stored tau (33) and the strain pass of Eq 24-25 (33); Eq 21 drops (4)
F_PAIR_VISC = 9 + 33 + 33 - 4
FP32_LANES, SM_MAX_MHZ = 128, 2070.0  # per SM (Blackwell); the nominal maximum SM clock
# Algorithmic HBM bytes per particle of one Symplectic step: two sorts of
# three 8-bit passes (20 each), two reorders (90), two cell tables (~7),
# predictor (91), corrector (115), two interactions (52)
STEP_BYTES_PER_PARTICLE = 2 * 3 * 20 + 2 * 90 + 2 * 7 + 91 + 115 + 2 * 52


def hbm_peak_gbs():
    try:
        return float(json.load(open(MEASURED_PEAKS))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0  # fallback figure for a GB300 copy


def list_capture(cell_mode, workload_name, variant, pair_once=False):
    """The committed ncu capture of the list kernels for this variant
    (profiles/k_interact_list_traffic.json), or None when it does not match:
    another workload / cell size / variant, or the kernel source or the build
    flags changed since the counters were taken."""
    import hashlib
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "k_interact_list_traffic.json")))
        src = open(os.path.join(ROOT, d["source"]), "rb").read()
        flags = open(os.path.join(ROOT, d["build"]), "rb").read()
        v = d["variants"][str(variant) + ("p" if pair_once else "")]
    except (OSError, ValueError, KeyError):
        return None
    if hashlib.sha256(src).hexdigest() != d["source_sha256"]:
        return None
    if hashlib.sha256(flags).hexdigest() != d.get("build_sha256"):
        return None
    if workload_name != "dam_break" or cell_mode != 1:
        return None
    return v


def measured_traffic(cell_mode, workload_name, variant, builds_per_step=1.0, pair_once=False):
    """DRAM bytes per interaction launch, as bench.py times it, from the
    committed capture (None when it does not match, see list_capture).
    Variant 4: (build + two evaluations) / 2; variant 5: one evaluation plus
    half the build times the builds per step (pair_once: the pair-once walk
    and its finish as the evaluation, the half-list build as the build)."""
    v = list_capture(cell_mode, workload_name, variant, pair_once)
    if v is None:
        return None
    if variant == 4:
        return (v["build_bytes"] + 2 * v["eval_bytes"]) / 2
    return v["eval_bytes"] + builds_per_step * v["build_bytes"] / 2


def measured_limiter(cell_mode, workload_name, variant, pair_once=False):
    """The hardware unit that bounds the list evaluation in the committed
    capture, with its utilisation (None when the capture does not match)."""
    v = list_capture(cell_mode, workload_name, variant, pair_once)
    return None if v is None else v.get("limiter")


def workload(name, rank=0, dp=None, **kw):
    from paper_2104_00537_gb300 import cases
    if name == "wave_flume" and dp:
        c = cases.wave_flume(dp, seed=rank, **kw)
        return [c], "wave flume 25x1x1.2 m dp=%g (%.1fM particles)" % (dp, c.n / 1e6)
    if name == "dam_break":
        return [cases.dam_break(0.004, seed=rank, **kw)], "3-D dam break dp=0.004 (1.48M particles)"
    if name == "dam_break_small":
        return [cases.dam_break(0.02, seed=rank, **kw)], "3-D dam break dp=0.02 (28k particles)"
    if name == "wave_flume":
        return [cases.wave_flume(0.008, seed=rank, **kw)], "wave flume 25x1x1.2 m dp=0.008 (32M particles)"
    if name == "batched":
        return cases.batch_dam_breaks(256, seed=rank, **kw), "256 dam breaks, 5k-200k fluid each"
    raise ValueError(name)


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        if not sm:
            return None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world <= 1:
        return 0, 1, 0, None
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    import torch
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend)
    return rank, world, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(x, dist):
    if dist is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, dist):
    if dist is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def cpu_baseline(case, seconds_budget=15.0):
    """The FP64 oracle timed on the host cores over a bounded sample of the same
    workload: whole Symplectic steps (neighbour list + two interaction
    evaluations + update, as the GPU steps) of the case from rest; one
    calibration step sizes the sample to about `seconds_budget` seconds."""
    import oracle
    s = oracle.OracleState(case)
    t0 = time.perf_counter()
    s.step(1)
    t_cal = time.perf_counter() - t0
    nsteps = max(1, min(200, int(seconds_budget / max(t_cal, 1e-3))))
    t0 = time.perf_counter()
    pairs = s.step(nsteps)
    dt = time.perf_counter() - t0
    return {"value": pairs / dt, "unit": "interactions/s", "cores": os.cpu_count(),
            "kind": "oracle", "steps_per_s": nsteps / dt,
            "sample": "FP64 oracle, OpenMP: Symplectic steps 2-%d of the %d-particle case "
                      "from rest (neighbour list + 2 interaction evaluations + update per "
                      "step; %d pairs, %.1f s)" % (nsteps + 1, case.n, pairs, dt)}


def run_reference(args, rank, world, dist):
    """Reference arm: the FP64 oracle on the host cores, same metric and
    workload: W untimed and K timed whole Symplectic steps of the case from
    rest, as the GPU arm times them (the same window of the run)."""
    import oracle
    if rank != 0:
        return
    cs, desc = workload(args.workload, 0)
    case = cs[0]
    s = oracle.OracleState(case)
    if args.warmup:
        s.step(args.warmup)
    t0 = time.perf_counter()
    pairs = s.step(args.steps)
    dt = time.perf_counter() - t0
    v = pairs / dt
    out = {"metric": "particle_interactions_per_s", "value": v, "unit": "interactions/s",
           "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "steps_per_s": args.steps / dt,
           "config": {"workload": desc, "particles": case.n,
                      "window": "steps %d-%d of the run from rest" % (
                          args.warmup, args.warmup + args.steps)},
           "cpu_baseline": {"value": v, "unit": "interactions/s", "cores": os.cpu_count(),
                            "kind": "oracle",
                            "sample": "FP64 oracle, OpenMP: Symplectic steps %d-%d of the "
                                      "%d-particle case from rest (neighbour list + 2 "
                                      "interaction evaluations + update per step)"
                                      % (args.warmup, args.warmup + args.steps, case.n)},
           "e2e": {"value": v, "unit": "interactions/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def timed_steps(eng, stream, steps):
    """Device time (ms) of `steps` Symplectic steps on the engine's stream."""
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    eng.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def measure_batched(ncases, steps, warmup, tune, clock_index=0, pair_once=0, fixed=None):
    """C3: `ncases` uneven dam breaks in one batched engine (one launch per
    stage for all cases, CUDA-graph replay) against the plain path that steps
    each case alone in its own engine (the list kept across steps, each step
    replayed from a captured graph: the fastest plain way measured).  Both
    time the same steps (warmup .. warmup + steps of every case from rest)
    with CUDA events on the engines' stream.  tune: pick cell size and
    interaction variant and list-walk block size with the autotuner (else
    cells of h, kept list, 128 threads).  pair_once: both paths evaluate each
    pair once (atomic sums: the two paths then agree to rounding, not bit for
    bit, and their pair counts may differ by the pairs at the cut-off)."""
    import torch
    from paper_2104_00537_gb300 import autotune, cases, sph
    stream = torch.cuda.Stream()
    cs = cases.batch_dam_breaks(ncases, seed=0)
    cm, var, block, tune_ms = 1, 5, 128, None
    if fixed:  # (cell_mode, pi_variant, pi_block) of an earlier tuning
        cm, var, block = fixed
    elif tune:
        mk = lambda cc: sph.Engine.batch(cc, stream=stream)
        (cm, var, block), tune_ms = autotune.tune(cs, mk, torch.cuda.get_device_name(0),
                                                  pair_once=pair_once)
    for c in cs:
        c.params["cell_mode"] = cm
    eng = sph.Engine.batch(cs, stream=stream)
    eng.set_options(pi_variant=var, pi_block=block, use_graph=1, pair_once=pair_once)
    eng.step(warmup)
    p0 = sum(eng.stats(i)["interactions"] for i in range(len(cs)))
    clocks = ClockSampler(clock_index)
    ms_b = timed_steps(eng, stream, steps)
    clk = clocks.stop()
    p1 = sum(eng.stats(i)["interactions"] for i in range(len(cs)))
    eng.destroy()
    ms_p, pp = 0.0, 0
    for c in cs:
        e = sph.Engine.create(c, stream=stream)
        e.set_options(pi_variant=var, pi_block=block, use_graph=1, pair_once=pair_once)
        e.step(warmup)
        q0 = e.stats()["interactions"]
        ms_p += timed_steps(e, stream, steps)
        pp += e.stats()["interactions"] - q0
        e.destroy()
    nb = len(cs) * steps
    return {"cases": len(cs), "particles": sum(c.n for c in cs), "steps": steps,
            "warmup": warmup, "cell_mode": cm, "pi_variant": var, "pi_block": block,
            "pair_once": bool(pair_once),
            "batched": {"case_steps_per_s": nb / (ms_b / 1e3), "ms_per_step": ms_b / steps,
                        "interactions_per_s": (p1 - p0) / (ms_b / 1e3)},
            "plain": {"case_steps_per_s": nb / (ms_p / 1e3), "ms_per_round": ms_p / steps,
                      "interactions_per_s": pp / (ms_p / 1e3)},
            "speedup_vs_plain": ms_p / ms_b, "same_pairs": p1 - p0 == pp,
            "autotune_ms_per_step": tune_ms, "clocks": clk}


def measure_served(requests, rate, max_fluid, t_end, chunk, cell_mode=1, pi_variant=-1,
                   list_skin=-1.0, plain=True, max_particles=None, pair_once=0):
    """C4: Poisson arrivals of sloshing-tank requests served by continuous
    batching on one pool engine (64 slots), against the same trace served one
    request at a time (a one-slot pool); wall-clock time-to-result.
    pair_once: both evaluate each pair once."""
    import torch
    from paper_2104_00537_gb300 import cases, serve, sph
    stream = torch.cuda.Stream()
    trace = cases.sloshing_trace(requests, rate=rate, seed=0, n_min=10000, n_max=max_fluid,
                                 t_end=t_end)
    for _, c, _ in trace:
        c.params["cell_mode"] = cell_mode
    free, _ = torch.cuda.mem_get_info()
    # about 200 B of state and 1.5 KB of per-step list per particle slot
    max_p = int(min(free * 0.3 / 1800, max_particles or 16_000_000))
    max_cells = int(min(free * 0.05 / 8, 200_000_000))
    results = {}
    for name, slots in (("served", 64), ("plain", 1)) if plain else (("served", 64),):
        pool = sph.Engine.pool(max_p, max_cells, slots, stream=stream)
        pool.set_options(use_graph=1, pi_variant=pi_variant, list_skin=list_skin,
                         pair_once=pair_once)
        reqs = [serve.Request(i, a, c, te) for i, (a, c, te) in enumerate(trace)]
        srv = serve.Server(pool, chunk=chunk)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        srv.run(reqs)
        wall = time.perf_counter() - t0
        st = serve.summary(reqs, wall)
        st["case_steps_per_s"] = srv.case_steps / wall
        results[name] = st
        pool.destroy()
    out = {"trace": "sloshing tanks 1x0.5x0.6 m, Poisson %.3g req/s, %d requests, fluid "
                    "10k-%d log-uniform, %.3g s simulated each"
                    % (rate, requests, max_fluid, t_end),
           "chunk_steps": chunk, "served": results["served"]}
    if plain:
        out["plain"] = results["plain"]
        out["throughput_ratio"] = (results["served"]["throughput_req_s"] /
                                   results["plain"]["throughput_req_s"])
        out["case_steps_ratio"] = (results["served"]["case_steps_per_s"] /
                                   results["plain"]["case_steps_per_s"])
    return out


def measure_full_run(case, stream, steps=2000, pair_once=0):
    """The case's whole run from rest (C1's 2,000 steps), graph-replayed with
    the list kept across steps: the step time at the run's own rebuild rate.
    pair_once: each pair evaluated once (atomic sums, not bit-reproducible)."""
    import torch
    from paper_2104_00537_gb300 import sph
    e = sph.Engine.create(case, stream=stream)
    e.set_options(use_graph=1, pair_once=pair_once)
    torch.cuda.synchronize()
    ms = timed_steps(e, stream, steps)
    s = e.stats()
    out = {"steps": steps, "ms_per_step": ms / steps, "steps_per_s": steps / (ms / 1e3),
           "interactions_per_s": s["interactions"] / (ms / 1e3),
           "builds_per_step": e.list_info()["builds"] / steps, "t_end_s": s["t"]}
    e.destroy()
    return out


def run_batched(args):
    import torch
    torch.cuda.set_device(0)
    r = measure_batched(args.ncases, args.steps, args.warmup, tune=True,
                        pair_once=args.pair_once)
    out = {"metric": "case_steps_per_s", "value": r["batched"]["case_steps_per_s"],
           "unit": "case-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": r["batched"]["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "%d dam breaks, fluid 5k-200k log-uniform" % r["cases"],
                      "particles": r["particles"], "cell_mode": r["cell_mode"],
                      "pi_variant": r["pi_variant"], "pi_block": r["pi_block"],
                      "pair_once": r["pair_once"]},
           "batched": r["batched"], "plain": r["plain"],
           "speedup_vs_plain": r["speedup_vs_plain"],
           "autotune_ms_per_step": r["autotune_ms_per_step"], "clocks": r["clocks"]}
    print(json.dumps(out), flush=True)


def run_served(args):
    import torch
    torch.cuda.set_device(0)
    r = measure_served(args.requests, args.rate, args.max_fluid, args.t_end, args.chunk,
                       args.cell_mode, args.pi_variant, args.list_skin,
                       pair_once=args.pair_once)
    out = {"metric": "served_p50_time_to_result_s", "value": r["served"]["p50_s"],
           "unit": "s", "n_gpus": 1, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": r["trace"], "chunk_steps": args.chunk,
                      "cell_mode": args.cell_mode,
                      "pi_variant": args.pi_variant if args.pi_variant >= 0 else 5},
           "served": r["served"], "plain": r["plain"],
           "throughput_ratio": r["throughput_ratio"], "case_steps_ratio": r["case_steps_ratio"]}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 2,000 for the dam break, its whole run "
                         "from rest; 100 otherwise and for the reference arm)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="dam_break")
    ap.add_argument("--cell-mode", type=int, default=1)
    ap.add_argument("--ddt-mode", type=int, default=1, choices=[0, 1, 2])
    ap.add_argument("--pi-variant", type=int, default=-1, choices=[-1, 0, 1, 2, 3, 4, 5, 6])
    ap.add_argument("--list-skin", type=float, default=-1.0)
    ap.add_argument("--pi-block", type=int, default=0,
                    help="threads per block of the list walk (0: the engine default)")
    ap.add_argument("--pi-lanes", type=int, default=0, choices=[0, 1, 2, 4, 8],
                    help="threads per target of the list walk (0: the engine default)")
    ap.add_argument("--pair-once", type=int, default=1, choices=[0, 1],
                    help="1 (default): evaluate each pair once (atomic sums, not "
                         "bit-reproducible); 0: every target sums its own pairs (the "
                         "library's default, reproducible bit for bit)")
    ap.add_argument("--integrator", default="symplectic", choices=["symplectic", "verlet"])
    ap.add_argument("--visc-mode", type=int, default=0, choices=[0, 1])
    ap.add_argument("--nu0", type=float, default=1e-6)
    ap.add_argument("--boundary-mode", type=int, default=0, choices=[0, 1])
    ap.add_argument("--mdbc-slip", type=int, default=0, choices=[0, 1, 2])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--dp", type=float, default=None,
                    help="particle spacing of the wave flume (default 0.008 m)")
    ap.add_argument("--no-modes", action="store_true",
                    help="skip the batched / served / full-run sub-measurements of the "
                         "default line")
    ap.add_argument("--ncases", type=int, default=256)
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--max-fluid", type=int, default=200000)
    ap.add_argument("--t-end", type=float, default=0.1)
    ap.add_argument("--chunk", type=int, default=10)
    args = ap.parse_args()
    if args.steps is None:  # the reference arm's steps are whole oracle steps: 20 by default
        args.steps = (2000 if args.workload == "dam_break" else 100) if args.impl == "gb300" \
            else 20
    args.warmup = max(3, args.warmup)
    if args.impl != "reference" and args.workload == "batched":
        return run_batched(args)
    if args.impl != "reference" and args.workload == "served":
        return run_served(args)

    rank, world, local, dist = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, world, dist)
        return

    import torch
    from paper_2104_00537_gb300 import sph
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    cs, desc = workload(args.workload, rank, dp=args.dp, boundary_mode=args.boundary_mode)
    for c in cs:
        c.params["cell_mode"] = args.cell_mode
        c.params["ddt_mode"] = args.ddt_mode
        c.params["integrator"] = 1 if args.integrator == "verlet" else 0
        c.params["visc_mode"] = args.visc_mode
        c.params["nu0"] = args.nu0
        c.params["boundary_mode"] = args.boundary_mode
        c.params["mdbc_slip"] = args.mdbc_slip
    with torch.cuda.stream(stream):
        eng = sph.Engine.batch(cs, stream=stream) if len(cs) > 1 else \
            sph.Engine.create(cs[0], stream=stream)
    eng.set_options(pi_variant=args.pi_variant, list_skin=args.list_skin, pi_block=args.pi_block,
                    pi_lanes=args.pi_lanes, pair_once=args.pair_once)
    n_particles = sum(c.n for c in cs)
    # the pi_variant the engine runs (its default: 5, the list kept across
    # steps; beyond 2^25 particles with wide records, for the default physics)
    default_physics = (args.ddt_mode != 2 and args.visc_mode == 0 and args.boundary_mode == 0)
    list_ok = n_particles < (1 << 25) or default_physics
    default_var = 5
    eff_var = args.pi_variant if args.pi_variant in (0, 1, 2, 3, 4, 5, 6) else (
        default_var if list_ok else 0)
    if eff_var in (3, 4, 5) and not list_ok:
        eff_var = 0
    if args.integrator == "verlet" and eff_var in (3, 4):
        eff_var = 0
    kernel = {3: "k_interact_list", 4: "k_interact_list", 5: "k_interact_list",
              6: "k_interact_tile"}.get(eff_var, "k_interact")
    pair_once_on = bool(args.pair_once) and eff_var in (4, 5) and default_physics
    if pair_once_on:
        kernel = "k_interact_sym + k_sym_finish"

    # the FP32 / FP64 pipe throughput of this GPU (roofline denominators),
    # measured before the warm-up
    peaks = sph.probe_peaks(stream)
    # warm-up
    eng.step(args.warmup)
    eng.set_options(pi_variant=args.pi_variant, list_skin=args.list_skin, timing=1,
                    pi_block=args.pi_block, pi_lanes=args.pi_lanes, pair_once=args.pair_once)
    eng.timing(reset=True)
    builds0 = eng.list_info()["builds"]

    def totals():
        s = [eng.stats(i) for i in range(len(cs))]
        return (sum(x["interactions"] for x in s), sum(x["interactions_fb"] for x in s),
                sum(x["interactions_bf"] for x in s))

    p0 = totals()
    barrier(dist)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    eng.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    p1 = totals()
    # per-step device times of the timed steps (CUDA events on the engine's
    # stream, start of one step's first interaction to the next's)
    st_ms = eng.step_times()
    step_time = None
    if len(st_ms):
        step_time = {"p50": max_over_ranks(float(np.percentile(st_ms, 50)), dist),
                     "p99": max_over_ranks(float(np.percentile(st_ms, 99)), dist),
                     "max": max_over_ranks(float(st_ms.max()), dist), "unit": "ms",
                     "steps": int(len(st_ms))}
    tm = eng.timing(reset=True)
    builds = eng.list_info()["builds"] - builds0
    pairs = p1[0] - p0[0]
    fb = p1[1] - p0[1]
    bf = p1[2] - p0[2]
    ff = pairs - fb - bf
    ms_max = max_over_ranks(ms, dist)
    pairs_all = sum_over_ranks(pairs, dist)
    value = pairs_all / (ms_max / 1000.0)
    steps_per_s = args.steps / (ms_max / 1000.0) * world

    # roofline of the dominant kernel (the interaction): algorithmic FLOPs per
    # launch / average launch duration (CUDA events on the engine's stream)
    f_ff = {0: F_PAIR_FB, 1: F_PAIR_FF, 2: F_PAIR_FF_HYD}[args.ddt_mode]
    f_fb = F_PAIR_FB
    if args.visc_mode == 1:
        f_ff += F_PAIR_VISC
        f_fb += F_PAIR_VISC
    flops = f_ff * ff + f_fb * fb + F_PAIR_BF * bf
    launches = max(1, tm["pi_launches"])
    pi_avg_s = tm["pi_ms"] / 1000.0 / launches
    achieved = flops / launches / pi_avg_s / 1e12
    peak = peaks["fp32_tflops"]
    mhz = clk["sm_mhz"] if clk else SM_MAX_MHZ
    nominal = peaks["sms"] * FP32_LANES * 2 * mhz * 1e6 / 1e12
    # the committed capture is of the default physics and launch shape
    captured = ((args.ddt_mode, args.integrator, args.visc_mode, args.boundary_mode) ==
                (1, "symplectic", 0, 0) and eff_var in (4, 5) and
                args.pi_block in (0, 128) and args.pi_lanes in (0, 1) and args.list_skin < 0)
    roofline = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "flop_basis": "48 / 45 / 25 FLOP per directed fluid-fluid / fluid-boundary / "
                              "boundary-fluid pair" + (
                                  " (the work of the per-target walk; the pair-once walk "
                                  "itself does about 56 FLOP per unordered pair)"
                                  if pair_once_on else ""),
                "peak_basis": "measured in this run: FP32 FMA chains on all %d SMs "
                              "(sph_probe_peaks, best of 3, CUDA events)" % peaks["sms"],
                "peak_nominal": nominal, "frac_nominal": achieved / nominal,
                "peak_nominal_basis": "%d SMs (device) x 128 FP32 lanes x 2 FLOP x %.0f MHz "
                                      "(median SM clock sampled in the timed region)"
                                      % (peaks["sms"], mhz),
                "fp64_measured_tflops": peaks["fp64_tflops"],
                "traffic": measured_traffic(args.cell_mode, args.workload, eff_var,
                                            pair_once=pair_once_on, builds_per_step=
                                            builds / args.steps) if captured else None,
                "limiter": measured_limiter(args.cell_mode, args.workload, eff_var,
                                            pair_once_on) if captured else None,
                "pi_share_of_step": tm["pi_ms"] / max(tm["step_ms"], 1e-9),
                "pi_ms_per_launch": 1000 * pi_avg_s}

    # whole-step bound T = interaction FLOPs / FP32 peak + step bytes / HBM peak
    # (default Symplectic step: two interactions); reported against ms_per_step
    step_bound = None
    if args.integrator == "symplectic" and args.boundary_mode == 0 and args.visc_mode == 0:
        t_alu = flops / args.steps / (peak * 1e12)
        t_hbm = STEP_BYTES_PER_PARTICLE * n_particles / (hbm_peak_gbs() * 1e9)
        step_bound = {"ms": 1000 * (t_alu + t_hbm), "alu_ms": 1000 * t_alu,
                      "hbm_ms": 1000 * t_hbm,
                      "frac": 1000 * (t_alu + t_hbm) / (ms_max / args.steps)}
    out = {"metric": "particle_interactions_per_s", "value": value, "unit": "interactions/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": desc, "particles": n_particles, "cases": len(cs),
                      "cell_mode": ["2h", "h", "2h/3"][args.cell_mode],
                      "density_diffusion": ["none", "Eq 18", "Eq 19-20"][args.ddt_mode],
                      "viscosity": ["artificial, Eq 21", "laminar + SPS, Eq 23-27 (nu0 %g)"
                                    % args.nu0][args.visc_mode],
                      "boundary": ["DBC, Eq 36 (2 wall layers)",
                                   "mDBC, Eq 38-39 (wall layers filling 2h, slip mode %d)"
                                   % args.mdbc_slip][args.boundary_mode],
                      "integrator": {"symplectic": "Symplectic, Eq 33-34 (2 PI per step)",
                                     "verlet": "Verlet, Eq 30-31, N_S = 40 (1 PI per step)"}[
                          args.integrator],
                      "pi_variant": eff_var,
                      "pair_once": bool(args.pair_once),
                      "window": "steps %d-%d of the run from rest" % (
                          args.warmup, args.warmup + args.steps),
                      "neighbour_list": (
                          {"builds_per_step": builds / args.steps,
                           "records": "wide (32-bit index)" if n_particles >= (1 << 25)
                           else "narrow (25-bit index + row code)",
                           "skin": "list_k |v|max + 1e-3 h + %g x 2h" % (
                               args.list_skin if args.list_skin >= 0 else 0.04)}
                          if eff_var == 5 else
                          {"builds_per_step": builds / args.steps} if eff_var in (3, 4)
                          else None),
                      "l2": "state (%.0f MB) larger than L2 (129 MB), no flush" %
                            (n_particles * 177 / 1e6),
                      "parallelism": "replicas" if world > 1 else "single"},
           "steps_per_s": steps_per_s, "interactions_per_step": pairs / args.steps,
           "gpu_launches": tm["kernel_launches"], "roofline": roofline, "clocks": clk,
           "step_bound": step_bound, "step_time": step_time}

    if rank == 0 and not args.no_e2e and len(cs) == 1:
        # end to end through the public API: the case's arrays and the result
        # buffers sit in pinned host memory before the clock starts; timed:
        # create (the H2D copy of the case and its first sort), K steps and
        # the read-back of the state (D2H)
        hp = sph.HostParticles(cs[0], pinned=True)
        outbuf = sph.state_buffers(cs[0].n, pinned=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2 = sph.Engine.create(cs[0], stream=stream, host=hp)
        e2.set_options(pi_variant=args.pi_variant, list_skin=args.list_skin,
                       pi_block=args.pi_block, pi_lanes=args.pi_lanes, pair_once=args.pair_once)
        e2.step(args.steps)
        st = [e2.get_state(0, out=outbuf)]
        e2pairs = e2.stats(0)["interactions"]
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        h2d = sum(c.n * (24 + 12 + 4 + 1 + 4) for c in cs)
        d2h = sum(c.n * (24 + 12 + 4 + 4) for c in cs)
        out["e2e"] = {"value": e2pairs / t_e2e, "unit": "interactions/s",
                      "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                      "note": "create from pinned host arrays + %d steps + get_state into "
                              "pinned arrays, wall clock" % args.steps}
        e2.destroy()
        del st
    eng.destroy()
    if rank == 0 and world == 1 and not args.no_modes and args.workload == "dam_break" and \
            (args.ddt_mode, args.integrator, args.visc_mode, args.boundary_mode) == \
            (1, "symplectic", 0, 0) and args.pi_variant in (-1, 5):
        # the rest of the metric, measured in the same run: the whole 2,000-step
        # run of this case, batched vs plain (C3), served vs plain (C4, scaled),
        # each in the mode of the line (pair_once as given) and in the other
        po = args.pair_once
        other = "reproducible" if po else "pair_once"
        out["full_run"] = measure_full_run(cs[0], stream, pair_once=po)
        out["full_run_" + other] = measure_full_run(cs[0], stream, pair_once=1 - po)
        out["batched"] = measure_batched(256, 500, 3, tune=True, clock_index=local,
                                         pair_once=po)
        out["batched"]["note"] = ("C3 as configured (256 cases, 26.6M particles, 500 timed "
                                  "steps after 3 from rest); cell size, pair loop and block "
                                  "size from the autotuner (3 timed steps per candidate), the "
                                  "same for both paths" + (
                                      "; each pair evaluated once on both paths (atomic "
                                      "sums: the paths agree to rounding, and their pair "
                                      "counts differ by pairs at the cut-off)" if po else
                                      "; each path's state equals the other's (same pairs)"))
        b = out["batched"]
        out["batched_" + other] = measure_batched(
            256, 500, 3, tune=False, clock_index=local, pair_once=1 - po,
            fixed=(b["cell_mode"], b["pi_variant"], b["pi_block"]))
        out["batched_" + other]["note"] = "as batched, both paths with pair_once = %d" % (1 - po)
        out["served"] = measure_served(48, 20.0, 200000, 0.1, 10, pair_once=po)
        out["served"]["note"] = ("C4 scaled to fit the run: 48 requests, fluid <= 200k, "
                                 "0.1 s simulated (C4: 100+ requests, <= 2M, 1 s; run with "
                                 "--workload served)")
        out["served_" + other] = measure_served(48, 20.0, 200000, 0.1, 10, pair_once=1 - po)
        out["served_" + other]["note"] = "as served, both modes with pair_once = %d" % (1 - po)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(cs[0])
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
