#!/usr/bin/env python3
"""SPH time-step benchmark (arXiv 1809.08013, Algorithm 1) on one GB300.

Default workload: rotating square patch, 100^3 = 1,000,000 particles, FP64
accuracy (the double-float pair kernels), 20 leapfrog steps from the initial
conditions (neighbour lists rebuilt and h iterated to 100 +- 5 every step).
One benchmark "step" is one full SPH time step through the C ABI (sph_step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                  [--workload patch|evrard] [--precision fp64|mixed|fp64-pipe]

--workload evrard --precision mixed is the Evrard collapse (Section 5.1.2,
hydrodynamics only) of 10^6 particles with the mixed-precision pair kernels;
--precision fp64-pipe runs the pair sums in native FP64 arithmetic.

N > 1 runs under torchrun as independent replicas (one instance per GPU, no
collective on the data path; the barrier and max-over-ranks timing only).
--impl reference times the CPU oracle on the host cores instead.

Output, three JSON lines on rank 0, the headline last:
  {"detail": ...}   every record in full (phases, the ensemble with its
                    autotuner trials, the serving stream, the Table 1 variants);
  {"summary": ...}  the same records in a few numbers each: steady state, the
                    27k small case, the Evrard 10^6 mixed-precision run, the 1M
                    patch with FP64-pipe pair sums, the 256-instance ensemble
                    (FP64 and mixed), the 2,000-request serving stream (batched
                    FP64, batched mixed, one at a time FP64, latency split),
                    the variants;
  headline          metric, value, e2e (through sph_step_host on pinned host
                    arrays), roofline of the dominant kernel, cpu_baseline,
                    clocks, gpu_launches.
--no-ensemble, --no-serving, --no-variants, --no-extra-workloads skip legs.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SPH particle-updates/s at 1M on 1 GB300 (% roofline); ensemble p50/p99 latency"
UNIT = "particle-updates/s"

# Counted FP64 work of one pair term of the force kernel, from the operations
# the definition writes out (each +, -, *, / and sqrt = 1): pair vector 3,
# r^2 5, r 1, q_i and q_j 2, two cubic-spline derivatives 2 x 5 plus their
# 1/(pi h^4) factors 2, Fbar 3, v_ij 3, v.r 5, (A_i + A_j + Pi) m_j Fbar 4,
# acceleration 6, energy sums 7  -> 51; the viscosity branch (v.r < 0) adds
# hb, cb, rhob 6, mu 5, Pi 6 -> 17 more.
FLOPS_PAIR_BASE = 51
FLOPS_PAIR_AV = 17


def variant_flops(kernel, gradients, sinc_n):
    """Counted FP64 work of the Table 1 variants, by the same rule (each +, -,
    *, / and sqrt = 1; sin and cos not counted). Shapes: the derivative f of
    M4 and Wendland C2 takes 5 operations and the sinc one n + 6 (x, S = sin
    x / x, S^(n-1), (x cos x - sin x) / x^2, n S^(n-1) S'); the value g takes 6
    (M4), 7 (Wendland) or n + 1 (sinc). Returns (per pair of S_i in the force
    pass, its viscosity extra, per pair of N_i in the IAD matrix pass).
    Kernel derivatives: FLOPS_PAIR_BASE with the two derivative shapes
    swapped. IAD force pair: pair vector 3, r^2 5, r 1, q_i and q_j 2, two
    values g, their h^-3 wnorm factors 4, C_i r and C_j r 30, G 12, v_ij 3,
    v.r 5, G.v 5, (A_i + A_j + Pi) m_j 3, times G 3, acceleration 3, energy
    sums 4 -> 83 + 2 g. IAD matrix pair: pair vector 3, r^2 5, r 1, q 1, g,
    m_j / rho_j 1, the weight 1, the six products and sums 15 -> 27 + g."""
    f = {0: 5, 1: 5, 2: sinc_n + 6}[kernel]
    g = {0: 6, 1: 7, 2: sinc_n + 1}[kernel]
    if gradients == 1:
        return 83 + 2 * g, FLOPS_PAIR_AV, 27 + g
    return FLOPS_PAIR_BASE - 2 * 5 + 2 * f, FLOPS_PAIR_AV, 0

# Counted work of one pair term by the per-pair figure of the scope table
# (about 75 operations per pair of S_i with the viscosity branch folded in),
# reported next to the count above.
FLOPS_PAIR_TABLE = 75

# ncu evidence for the dominant kernel of each precision, from one capture of
# that kernel at the benchmark size (profiles/<kernel>_patch1m.md or
# _evrard1m.md): DRAM bytes read + written per launch, warp instructions per
# launch, and the share of cycles with an instruction issued. Each entry is
# used only while the kernel's sources hash to the captured version (sha1 of
# the files listed, in order); otherwise the bench reports null.
NCU_EVIDENCE = {
    # k_forces_df<2, M4>, the 1M patch, second step of the timed call
    "df": {"sources": ("physics_df.cu", "df.cuh"), "sha1": "f8d02101d48d3d37cc808df61a0e0cc2ec302d17",
           "dram_bytes": (697.33 + 44.48) * 1e6, "warp_inst": 1708627293,
           "issue_active": 73.42, "pairs": 100727656,
           "profile": "profiles/forces_patch1m_evrard1m.md"},
    # k_forces_mx<2>, the 1M Evrard sphere, mixed precision
    "mixed": {"sources": ("physics_mixed.cu", "df.cuh"), "sha1": "342c531574d34f46723d3a8d907325d05aed3aee",
              "dram_bytes": (650.91 + 37.92) * 1e6, "warp_inst": 583622306,
              "issue_active": 47.63, "pairs": 105700202,
              "profile": "profiles/forces_patch1m_evrard1m.md"},
    # k_forces<M4>, the 1M patch, native FP64 pair sums
    "fp64": {"sources": ("physics.cu",), "sha1": "6247f00dbf82cc04d06456dd9af9a433de9cf7fe",
             "dram_bytes": (654.77 + 37.64) * 1e6, "warp_inst": 1248076044,
             "issue_active": 7.48, "pairs": 100727656,
             "profile": "profiles/forces_patch1m_evrard1m.md"},
}


def ncu_evidence(kind):
    import hashlib
    ref = NCU_EVIDENCE.get(kind)
    if ref is None:
        return None
    h = hashlib.sha1()
    src = os.path.join(ROOT, "paper_1809_08013_gb300", "csrc")
    for f in ref["sources"]:
        with open(os.path.join(src, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != ref["sha1"]:
        return None
    return ref


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--side", type=int, default=100, help="lattice side (100 -> 1M particles)")
    ap.add_argument("--seed", type=int, default=None, help="default 2 (patch), 3 (evrard)")
    ap.add_argument("--workload", choices=("patch", "evrard"), default="patch")
    ap.add_argument("--n", type=int, default=1_000_000, help="Evrard particle count")
    ap.add_argument("--precision", choices=("fp64", "mixed", "fp64-pipe"), default="fp64")
    ap.add_argument("--cell-scale", type=float, default=0.0,
                    help="neighbour-search cell width / (2 <h>); 0 = library default")
    ap.add_argument("--pair-threads", type=int, default=0,
                    help="lanes per particle in the pair sums (0 = library default)")
    ap.add_argument("--defer-lanes", type=int, default=0,
                    help="h-search hand-over threshold (0 = library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the batched-ensemble measurement")
    ap.add_argument("--ensemble-steps", type=int, default=50)
    ap.add_argument("--ensemble-count", type=int, default=256)
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the Table 1 variants (Wendland, sinc, IAD) at the bench size")
    ap.add_argument("--variant-steps", type=int, default=5)
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving stream (the configuration's 2000)")
    ap.add_argument("--serve-tick-s", type=float, default=0.25,
                    help="target seconds per serving tick (steps per tick adapt to it)")
    ap.add_argument("--no-extra-workloads", action="store_true",
                    help="skip the Evrard mixed-precision and FP64-pipe runs")
    ap.add_argument("--serve-rate", type=float, default=20.0, help="mean arrivals per second")
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-quantum", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms, world, device):
    """The slowest rank's time: replicas run the same work, so the job ends
    when the last one does (an all-reduce of one number, outside the timed
    region; nothing of the SPH data is exchanged)."""
    if world == 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, n, steps, ms_max):
    """Particle updates per second of the whole job: every rank advances its
    own n-particle replica `steps` steps, all within ms_max milliseconds."""
    return world * n * steps / (ms_max * 1e-3)


PRECISION = {"fp64": 0, "mixed": 1, "fp64-pipe": 2}
# The arithmetic of the pair sums; state, h, neighbour sets, dt and the
# integration are FP64 in all three.
DTYPE = {"fp64": "df64: float-float pair sums on the FP32 pipes (~48-bit significand, FP64 "
                 "state; held to the 1e-12 FP64 tolerance)",
         "mixed": "mixed: f32 pair terms, float-float sums, f64 state",
         "fp64-pipe": "f64"}


def workload_name(args, n=None):
    prec = {"fp64": "FP64 accuracy (double-float pair sums)",
            "fp64-pipe": "FP64 (native FP64 pair sums)",
            "mixed": "mixed precision (FP32 relative-coordinate pair terms, double-float sums, "
                     "FP64 positions, h, neighbour sets and integration)"}[args.precision]
    if args.workload == "evrard":
        n = n or args.n
        return (f"Evrard collapse, hydrodynamics only, {n:,} particles (Section 5.1.2: R=M=1, "
                f"rho ~ 1/r sampled r=R sqrt(U), u=0.05, ideal gas gamma=5/3, v=0), {prec}, "
                f"cubic spline, h iterated to 100+-5 neighbours every step, Monaghan AV alpha=1 "
                f"beta=2, CFL 0.3, kick-drift leapfrog from the initial conditions")
    side = args.side if n is None else round(n ** (1 / 3))
    n = side ** 3
    return (f"rotating square patch {side}^3 = {n:,} particles (Section 5.1.1: lattice dx=1/{side}, "
            f"jitter 0.01 dx, omega=5, rho0=1000, Tait c0=50, periodic z), {prec}, cubic spline, "
            f"h iterated to 100+-5 neighbours every step, Monaghan AV alpha=1 beta=2, CFL 0.3, "
            f"kick-drift leapfrog from the initial conditions")


def make_workload(args, n=None):
    """Seeded initial conditions of the selected workload (n overrides the size)."""
    from paper_1809_08013_gb300 import ics
    if args.workload == "evrard":
        seed = 3 if args.seed is None else args.seed
        s, prm = ics.evrard(n or args.n, seed=seed)
    else:
        seed = 2 if args.seed is None else args.seed
        side = args.side if n is None else round(n ** (1 / 3))
        s, prm = ics.square_patch(side, seed=seed)
    prm.precision = PRECISION[args.precision]
    prm.cell_scale = args.cell_scale
    prm.pair_threads = args.pair_threads
    prm.defer_lanes = args.defer_lanes
    return s, prm


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons (read-only)."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.proc = None
        self.lines = []
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self, t0, t1):
        import datetime
        rows = []
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        inside = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05]
        if not inside:  # region shorter than the sampling period: nearest samples
            inside = sorted(rows, key=lambda r: abs(r[0] - 0.5 * (t0 + t1)))[:3]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in inside for k in range(4) if r[3][k].lower() == "active"})
        mhz = sorted(r[1] for r in inside)
        return {"sm_mhz": mhz[len(mhz) // 2], "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside)}


# --------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    # bounded sample of the workload: the same recipe at about 50k particles
    s, prm = make_workload(args, n=50_653)
    n = len(s["x"])
    for _ in range(args.warmup):
        oracle.step(prm, s, nsteps=1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.step(prm, s, nsteps=1)  # every step starts from the initial conditions
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    sample = (f"oracle (plain C FP64, OpenMP) step of the same {args.workload} recipe at {n:,} "
              f"particles from its initial conditions, {args.steps} steps")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "sample_particles": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- native arm
def av_fraction(B, ctx, arr, periodic_z, sample_rows=4000):
    """Share of interaction pairs with v_ij . r_ij < 0 (viscosity branch) on a
    sample of rows of the last step's neighbour list (host-side estimate used
    only for the counted-flop figure)."""
    import numpy as np
    off, idx, ng, order = ctx.neighbors_to_host()
    n = len(order)
    if n == 0 or off[-1] == 0:
        return 0.0, 0
    rng = np.random.Generator(np.random.PCG64(0))
    rows = rng.choice(n, size=min(sample_rows, n), replace=False)
    x = {k: arr[k].cpu().numpy() for k in ("x", "y", "z", "vx", "vy", "vz")}
    tot = neg = 0
    for k in rows:
        js = order[idx[off[k]:off[k + 1]]]
        i = order[k]
        d = np.stack([x["x"][i] - x["x"][js], x["y"][i] - x["y"][js], x["z"][i] - x["z"][js]])
        if periodic_z:
            d[2] -= np.round(d[2])
        w = np.stack([x["vx"][i] - x["vx"][js], x["vy"][i] - x["vy"][js], x["vz"][i] - x["vz"][js]])
        vr = (w * d).sum(0)
        neg += int(np.count_nonzero(vr < 0))
        tot += len(js)
    return neg / max(tot, 1), int(off[-1])


def ensemble_instances(count, precision, seed=1000):
    """Configuration 4: `count` rotating patches, N log-uniform in [4096,
    262144] rounded to cubes, omega ~ U[2, 8], seeds seed + k."""
    from paper_1809_08013_gb300 import ics
    out = []
    for k, (side, omega) in enumerate(ics.ensemble_sizes(count, seed)):
        s, p = ics.square_patch(side, seed=seed + k, omega=omega)
        p.precision = PRECISION[precision]
        out.append((s, p))
    return out


def run_ensemble(args, B, dev, precision):
    """Batched ensemble (one CUDA graph of sph_batch_step over all instances)
    against the single-instance path run one instance after another.
    Latency of an instance = time from submission to its result: in the
    batch every instance is submitted together and completes with the graph;
    one at a time, instance k completes after all earlier ones."""
    import numpy as np
    import torch
    stream = torch.cuda.Stream(device=dev)  # graphs are captured on a non-default stream
    with torch.cuda.stream(stream):
        out = _run_ensemble(args, B, dev, stream, precision)
    torch.cuda.empty_cache()
    return out


def _run_ensemble(args, B, dev, stream, precision):
    import numpy as np
    import torch
    K = args.ensemble_steps
    insts = ensemble_instances(args.ensemble_count, precision)
    counts = [len(s["x"]) for s, _ in insts]
    ntot = sum(counts)
    state = {k: np.concatenate([s[k] for s, _ in insts]) for k in B.STATE_FIELDS}
    ctx = B.Context(ntot, max_instances=len(insts), device=dev.index)
    ctx.batch_set(counts, [p for _, p in insts], stream=stream)
    arr = B.alloc_arrays(state, device=dev, ninst=len(insts))
    ic = {k: arr[k].clone() for k in B.STATE_FIELDS}

    def reset():
        for k in B.STATE_FIELDS:
            arr[k].copy_(ic[k])
        arr["time"].zero_()

    ctx.batch_step(arr, nsteps=1, stream=stream)  # warm-up
    ctx.sync(stream)
    reset()
    tune = ctx.autotune(arr, nsteps=2, stream=stream)  # knobs of the whole batch
    ctx.sync(stream)
    tuned = {"cell_scale": tune["cell_scale"], "pair_threads": tune["pair_threads"],
             "defer_lanes": tune["defer_lanes"]}
    torch.cuda.synchronize(dev)
    g = torch.cuda.CUDAGraph()
    l0 = ctx.launch_count()
    with torch.cuda.graph(g, stream=stream):
        ctx.batch_step(arr, nsteps=K, stream=stream)
    graph_kernels = ctx.launch_count() - l0
    g.replay()  # warm replay
    torch.cuda.synchronize(dev)
    reset()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_batch = e0.elapsed_time(e1)
    st = ctx.sync(stream)
    batched = {k: arr[k].cpu().numpy() for k in ("x", "y", "z", "vx", "vy", "vz", "h", "u")}
    del g

    staged = _run_staged(B, dev, stream, insts, counts, tuned, K, batched)

    # the plain single-instance path, one instance after another on one context
    one = B.Context(max(counts), device=dev.index)
    t_alone = []
    same = True
    off = np.concatenate([[0], np.cumsum(counts)])
    from paper_1809_08013_gb300 import ics
    for k, (s, p) in enumerate(insts):
        p = ics.SphParams(**{**p.as_dict(), **tuned})  # the same knobs as the batch
        a = B.alloc_arrays(s, device=dev)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        one.step(p, a, nsteps=K, stream=stream)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        t_alone.append(f0.elapsed_time(f1))
        for f in batched:
            same = same and np.array_equal(a[f].cpu().numpy().view(np.uint8),
                                           batched[f][off[k]:off[k + 1]].view(np.uint8))
    one.sync(stream)
    t_alone = np.array(t_alone)
    done_seq = np.cumsum(t_alone)
    upd = ntot * K
    return {
        "workload": f"{len(insts)} rotating patches, N log-uniform in [4096, 262144] rounded to "
                    f"cubes (sum {ntot:,}), omega ~ U[2,8], seeds 1000+k, {K} steps each, "
                    f"{precision}",
        "instances": len(insts), "particles": ntot, "steps": K,
        "batched": {"ms": t_batch, "updates_per_s": upd / (t_batch * 1e-3),
                    "latency_ms_p50": t_batch, "latency_ms_p99": t_batch,
                    "launch": "one CUDA graph of sph_batch_step",
                    "kernels_in_graph": graph_kernels,
                    "status": B.STATUS_NAMES.get(st)},
        "single_instance_path": {"ms": float(done_seq[-1]),
                                 "updates_per_s": upd / (done_seq[-1] * 1e-3),
                                 "latency_ms_p50": float(np.percentile(done_seq, 50)),
                                 "latency_ms_p99": float(np.percentile(done_seq, 99)),
                                 "own_time_ms_p50": float(np.percentile(t_alone, 50)),
                                 "own_time_ms_p99": float(np.percentile(t_alone, 99)),
                                 "launch": "sph_step per instance, one after another"},
        "staged": staged,
        "batched_equals_single_bitwise": bool(same),
        "autotune": {"chosen": tuned, "trials": tune["trials"],
                     "method": "sph_autotune: one coordinate-descent pass over pair_threads "
                               "{1,2,4}, cell_scale {0.875,1,1.25}, defer_lanes {8,16}; 2 timed "
                               "steps per trial"},
    }


def stage_groups(counts, stages):
    """Instance indices in order of size (stable), cut into at most `stages`
    consecutive groups, a group closing once the running particle count
    reaches the next multiple of total / stages."""
    import numpy as np
    order = np.argsort(np.array(counts), kind="stable")
    tot = int(sum(counts))
    groups, cur, acc = [], [], 0
    for k in order:
        cur.append(int(k))
        acc += counts[k]
        if len(groups) < stages - 1 and acc >= tot * (len(groups) + 1) / stages:
            groups.append(cur)
            cur = []
    if cur:
        groups.append(cur)
    return groups


def _run_staged(B, dev, stream, insts, counts, tuned, K, batched, stages=4):
    """The ensemble as `stages` batches run back to back, the instances taken
    in order of size and cut into groups of about equal particle count, each
    group its own context and captured graph of sph_batch_step(K). An
    instance's latency is the end of its group's replay, so the small
    instances finish early; the results equal the one-graph batch's bitwise."""
    import numpy as np
    import torch
    from paper_1809_08013_gb300 import ics
    tot = int(sum(counts))
    groups = stage_groups(counts, stages)
    runs = []
    for gi in groups:
        sub = [insts[k] for k in gi]
        cnt = [counts[k] for k in gi]
        state = {f: np.concatenate([s[f] for s, _ in sub]) for f in B.STATE_FIELDS}
        ctx = B.Context(sum(cnt), max_instances=len(sub), device=dev.index)
        ctx.batch_set(cnt, [ics.SphParams(**{**p.as_dict(), **tuned}) for _, p in sub],
                      stream=stream)
        arr = B.alloc_arrays(state, device=dev, ninst=len(sub))
        ic = {f: arr[f].clone() for f in B.STATE_FIELDS}

        def reset(arr=arr, ic=ic):
            for f in B.STATE_FIELDS:
                arr[f].copy_(ic[f])
            arr["time"].zero_()

        ctx.batch_step(arr, nsteps=1, stream=stream)  # untimed
        ctx.sync(stream)
        reset()
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            ctx.batch_step(arr, nsteps=K, stream=stream)
        g.replay()  # warm replay
        torch.cuda.synchronize(dev)
        reset()
        torch.cuda.synchronize(dev)
        runs.append((ctx, arr, g))
    e0 = torch.cuda.Event(enable_timing=True)
    ends = [torch.cuda.Event(enable_timing=True) for _ in runs]
    e0.record(stream)
    for (_, _, g), e in zip(runs, ends):
        g.replay()
        e.record(stream)
    torch.cuda.synchronize(dev)
    t_end = [e0.elapsed_time(e) for e in ends]
    st = max(ctx.sync(stream) for ctx, _, _ in runs)
    lat = np.concatenate([[t_end[q]] * len(gi) for q, gi in enumerate(groups)])
    off = np.concatenate([[0], np.cumsum(counts)])
    same = True
    for (ctx, arr, _), gi in zip(runs, groups):
        host = {f: arr[f].cpu().numpy() for f in batched}
        pos = 0
        for k in gi:
            for f in batched:
                same = same and np.array_equal(host[f][pos:pos + counts[k]].view(np.uint8),
                                               batched[f][off[k]:off[k + 1]].view(np.uint8))
            pos += counts[k]
    for ctx, arr, g in runs:
        del g
    del runs
    torch.cuda.empty_cache()
    return {"stages": len(groups), "instances_per_stage": [len(gi) for gi in groups],
            "particles_per_stage": [int(sum(counts[k] for k in gi)) for gi in groups],
            "stage_end_ms": t_end, "ms": t_end[-1],
            "updates_per_s": tot * K / (t_end[-1] * 1e-3),
            "latency_ms_p50": float(np.percentile(lat, 50)),
            "latency_ms_p99": float(np.percentile(lat, 99)),
            "launch": f"{len(groups)} CUDA graphs of sph_batch_step, smallest instances first",
            "equals_batched_bitwise": bool(same), "status": B.STATUS_NAMES.get(st)}


# (name, kernel, gradients, sinc_n, precision): every kernel and gradient
# variant runs in double-float at precision 0 and on the FP64 pipe at precision 2.
VARIANTS = (("M4, kernel derivatives, FP64 pipe (precision 2)", 0, 0, 5, 2),
            ("Wendland C2, kernel derivatives, double-float (precision 0)", 1, 0, 5, 0),
            ("Wendland C2, kernel derivatives, FP64 pipe (precision 2)", 1, 0, 5, 2),
            ("sinc n=5, kernel derivatives, double-float (precision 0)", 2, 0, 5, 0),
            ("sinc n=5, kernel derivatives, FP64 pipe (precision 2)", 2, 0, 5, 2),
            ("M4, IAD gradients, double-float (precision 0)", 0, 1, 5, 0),
            ("Wendland C2, IAD gradients, double-float (precision 0)", 1, 1, 5, 0),
            ("sinc n=5, IAD gradients, double-float (precision 0)", 2, 1, 5, 0),
            ("M4, IAD gradients, FP64 pipe (precision 2)", 0, 1, 5, 2))


def run_variants(args, B, dev, fp64_peak, fp32_peak):
    """The Table 1 variants on the benchmark workload: each a separate run of
    --variant-steps steps from the initial conditions (after one untimed
    step), with the pair kernels VARIANTS names. Roofline of the force phase
    (the force kernel, with k_volume + k_iad for IAD and k_dt_finish) from
    the counted flops of variant_flops, against the FMA-chain probe of the
    pipe the pair arithmetic runs on: FP32 for double-float (precision 0),
    FP64 for precision 2."""
    import numpy as np
    import torch
    s, base = make_workload(args)
    n = len(s["x"])
    ctx = B.Context(n, device=dev.index)
    arr = B.alloc_arrays(s, device=dev)
    ic = {k: arr[k].clone() for k in B.STATE_FIELDS}
    stream = torch.cuda.current_stream(dev)
    out = []
    for name, kernel, grads, sn, prec in VARIANTS:
        prm = ics_params_copy(base)
        prm.precision = prec
        prm.kernel, prm.gradients, prm.sinc_n = kernel, grads, sn

        def reset():
            for k in B.STATE_FIELDS:
                arr[k].copy_(ic[k])
            arr["time"].zero_()

        reset()
        ctx.step(prm, arr, nsteps=1, stream=stream)
        ctx.sync(stream)
        reset()
        torch.cuda.synchronize(dev)
        ctx.timing_enable(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.step(prm, arr, nsteps=args.variant_steps, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        phase_ms, _, tsteps = ctx.timing_read()
        ctx.timing_enable(False)
        st = ctx.sync(stream)
        f_av, nnz = av_fraction(B, ctx, arr, prm.periodic_z)
        ngather = int(arr["nnb"].sum().item())
        base_f, av_f, iad_f = variant_flops(kernel, grads, sn)
        flops = nnz * (base_f + av_f * f_av) + ngather * iad_f
        forces_s = phase_ms["forces"] * 1e-3 / max(tsteps, 1)
        ach = flops / forces_s / 1e12
        peak = (fp64_peak if prec == 2 else fp32_peak) / 1e12
        out.append({"variant": name, "kernel": kernel, "gradients": grads,
                    "sinc_n": sn if kernel == 2 else None,
                    "ms_per_step": ms / args.variant_steps,
                    "value": n * args.variant_steps / (ms * 1e-3), "unit": UNIT,
                    "phases_ms_per_step": {k: v / max(tsteps, 1) for k, v in phase_ms.items()},
                    "status": B.STATUS_NAMES.get(st),
                    "precision": prec,
                    "roofline": {"bound": "alu", "kernel": kernel_names(kernel, grads, prec),
                                 "achieved": ach, "peak": peak,
                                 "unit": "TFLOP/s", "frac": ach / peak,
                                 "flops_per_launch": flops,
                                 "counted": {"pair": base_f, "pair_av": av_f,
                                             "iad_pair": iad_f},
                                 "peak_source": ("FP64" if prec == 2 else "FP32") +
                                                " FMA-chain probe, this run"}})
    del ctx
    torch.cuda.empty_cache()
    return {"workload": workload_name(args).split(", FP64 accuracy")[0], "steps": args.variant_steps,
            "runs": out}


def kernel_names(kernel, grads, prec):
    """The force phase's kernels of a variant run."""
    df = prec == 0
    if grads:
        return "k_volume_df + k_iad_df + k_forces_iad_df" if df else "k_volume + k_iad + k_forces_iad"
    return "k_forces_df" if df else "k_forces"


def ics_params_copy(p):
    import dataclasses
    return dataclasses.replace(p)


def run_serving(args, B, dev):
    """Configuration 5: a Poisson stream of patch / Evrard requests served by
    continuous batching (paper_1809_08013_gb300.serve) in FP64 and in mixed
    precision, against the plain single-instance FP64 path taking the same
    requests one at a time in arrival order."""
    import numpy as np
    import torch

    from paper_1809_08013_gb300 import serve
    torch.cuda.empty_cache()
    stream = torch.cuda.Stream(device=dev)
    out = {"workload": f"{args.serve_requests} requests, Poisson arrivals at {args.serve_rate}/s, "
                       f"patch (omega ~ U[2,8]) or Evrard 50/50, N log-uniform in [8000, 1e6], "
                       f"steps ~ U{{10..100}}, device budget {args.serve_budget_gb} GB, "
                       f"ticks of about {args.serve_tick_s} s (at most {args.serve_quantum} "
                       f"steps), admission in arrival order",
           "latency_unit": "s"}
    base = serve.make_stream(args.serve_requests, args.serve_rate, seed=5)
    with torch.cuda.stream(stream):
        # the single-instance FP64 path, one request at a time (time alone per request)
        one = B.Context(max(r.n for r in base), device=dev.index)
        run_time, alone = {}, {}
        for r in base:
            st, p = serve.initial_state(r, 0)
            a = B.alloc_arrays(st, device=dev)
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            one.step(p, a, nsteps=r.steps, stream=stream)
            f1.record(stream)
            torch.cuda.synchronize(dev)
            run_time[r.rid] = f0.elapsed_time(f1) * 1e-3
            if r.rid < 16:
                alone[r.rid] = {f: a[f].cpu().numpy() for f in ("x", "vx", "h", "u", "rho")}
        one.sync(stream)
        del one
        out["single_instance_fp64"] = serve.fifo_single(
            [dataclasses_replace(r) for r in base], run_time)
        bpp = serve.Server.bytes_per_particle()
        cap = int(args.serve_budget_gb * 1e9 / bpp)
        for prec, name in ((0, "batched_fp64"), (1, "batched_mixed")):
            reqs = serve.make_stream(args.serve_requests, args.serve_rate, seed=5)
            states = {r.rid: serve.initial_state(r, prec) for r in reqs}
            srv = serve.Server(cap, max_instances=256, quantum=args.serve_quantum,
                               device=dev.index, stream=stream, tick_s=args.serve_tick_s,
                               result_fields=("x", "vx", "h", "u", "rho"),
                               keep_result=lambda r: r.rid < 16)
            summ = serve.serve(srv, reqs, states, clock="real")
            summ["capacity_particles"] = cap
            summ["device_bytes_per_particle"] = bpp
            summ["ticks"] = srv.ticks
            summ["status"] = B.STATUS_NAMES.get(srv.status)
            if prec == 0:
                summ["results_equal_single_instance_bitwise"] = bool(all(
                    np.array_equal(reqs[k].result[f].view(np.uint8), v.view(np.uint8))
                    for k, ref in alone.items() for f, v in ref.items()))
                summ["compared_requests"] = len(alone)
            out[name] = summ
            del srv
            torch.cuda.empty_cache()
    return out


def dataclasses_replace(r):
    import dataclasses
    return dataclasses.replace(r)


def gpu_small_case(args, B, dev, steps=20):
    """The 30^3 = 27,000-particle patch (seed 1, the small configuration) on
    the GPU: one sph_step(steps) call from the initial conditions, after one
    untimed call. It fits in L2; a latency figure, not a roofline case."""
    import torch
    from paper_1809_08013_gb300 import ics
    s, prm = ics.square_patch(30, seed=1)
    prm.precision = PRECISION[args.precision]
    n = len(s["x"])
    ctx = B.Context(n, device=dev.index)
    arr = B.alloc_arrays(s, device=dev)
    ic = {k: arr[k].clone() for k in B.STATE_FIELDS}
    stream = torch.cuda.current_stream(dev)
    ctx.step(prm, arr, nsteps=steps, stream=stream)
    ctx.sync(stream)
    for k in B.STATE_FIELDS:
        arr[k].copy_(ic[k])
    arr["time"].zero_()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    ctx.step(prm, arr, nsteps=steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    st = ctx.sync(stream)
    return {"workload": f"rotating patch 30^3 = {n:,} particles, {steps} steps from the initial "
                        f"conditions", "ms_per_step": ms / steps,
            "value": n * steps / (ms * 1e-3), "unit": UNIT, "status": B.STATUS_NAMES.get(st)}


def oracle_small_case(oracle, args):
    """The oracle on the 30^3 = 27,000-particle patch (seed 1, the small
    configuration), one step from the initial conditions, on all host cores
    and on one."""
    from paper_1809_08013_gb300 import ics
    s, prm = ics.square_patch(30, seed=1)
    prm.precision = PRECISION[args.precision]
    n = len(s["x"])
    out = {"workload": f"rotating patch 30^3 = {n:,} particles, one step"}
    cores = oracle.get_threads()
    for label, k in (("all_cores", cores), ("one_core", 1)):
        oracle.set_threads(k)
        t0 = time.perf_counter()
        oracle.step(prm, s, nsteps=1)
        t = time.perf_counter() - t0
        out[label] = {"cores": k, "seconds": t, "value": n / t, "unit": UNIT}
    oracle.set_threads(cores)
    return out


def forces_roofline(B, ctx, arr, prm, phase_ms, tsteps, fp64_peak, fp32_peak):
    """Roofline of the force phase, the dominant kernel of a step: counted
    flops per launch (pairs of S_i x the per-pair count, with the viscosity
    branch weighted by its measured share) over the phase's CUDA-event time,
    against the FMA probe of the pipe the arithmetic runs on -- the FP32 pipe
    for the double-float and mixed kernels, the FP64 pipe for native FP64."""
    f_av, nnz = av_fraction(B, ctx, arr, prm.periodic_z)
    flops = nnz * (FLOPS_PAIR_BASE + FLOPS_PAIR_AV * f_av)
    sec = phase_ms["forces"] * 1e-3 / max(tsteps, 1)
    achieved = flops / sec / 1e12
    kind = {0: "df", 1: "mixed", 2: "fp64"}[prm.precision]
    kernel = {"df": "k_forces_df", "mixed": "k_forces_mx", "fp64": "k_forces"}[kind]
    peak = (fp64_peak if kind == "fp64" else fp32_peak) / 1e12
    ev = ncu_evidence(kind)
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak,
           "traffic": ev["dram_bytes"] * nnz / ev["pairs"] if ev else None,
           "kernel": kernel + " (+ k_dt_finish)",
           "peak_source": ("FP64" if kind == "fp64" else "FP32") +
                          " FMA-chain probe of this GPU in this run (sph_probe_fma_peak), 2 flops "
                          "per FMA: the pipe the pair arithmetic runs on",
           "counted_flops_per_pair": f"{FLOPS_PAIR_BASE} + {FLOPS_PAIR_AV} when v.r < 0",
           "flops_per_launch": flops, "pairs_per_launch": nnz, "av_pair_fraction": f_av,
           "achieved_at_75_per_pair": nnz * FLOPS_PAIR_TABLE / sec / 1e12,
           "fp64_probe_tflops": fp64_peak / 1e12, "fp32_probe_tflops": fp32_peak / 1e12,
           "ms_per_launch": sec * 1e3}
    if ev:
        out["issue"] = {"warp_inst_per_pair": ev["warp_inst"] / ev["pairs"],
                        "lane_inst_per_pair": 32 * ev["warp_inst"] / ev["pairs"],
                        "issue_active": ev["issue_active"], "source": ev["profile"]}
    return out


def measure_workload(args, B, dev, fp64_peak, fp32_peak, e2e=True, sampler=None):
    """One workload through sph_step: W untimed warm-up steps, the state reset
    to the initial conditions, then K timed steps in one call (CUDA events on
    the launching stream, per-phase events inside the library), step 0 alone
    (steady state = the rest), the end-to-end rate through sph_step_host on
    pinned host arrays, and the force phase's roofline."""
    import numpy as np
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    s, prm = make_workload(args)
    n = len(s["x"])
    ctx = B.Context(n, device=dev.index)
    arr = B.alloc_arrays(s, device=dev)
    ic = {k: arr[k].clone() for k in B.STATE_FIELDS}
    stream = torch.cuda.current_stream(dev)

    def reset():
        for k in B.STATE_FIELDS:
            arr[k].copy_(ic[k])
        arr["time"].zero_()

    ctx.step(prm, arr, nsteps=args.warmup, stream=stream)
    st = ctx.sync(stream)
    if st not in (B.SPH_OK, B.SPH_E_HNOCONV):
        raise RuntimeError(f"warm-up status {B.STATUS_NAMES.get(st)}: {ctx.error()}")
    reset()
    torch.cuda.synchronize(dev)
    if sampler is not None:
        time.sleep(1.0)
    # the timed region: one sph_step(K) call as a user makes it (each step
    # replays the library's captured step graph)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    l0 = ctx.launch_count()
    w0 = time.time()
    e0.record(stream)
    ctx.step(prm, arr, nsteps=args.steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    w1 = time.time()
    if world > 1:
        dist.barrier()
    launches = ctx.launch_count() - l0
    ms = e0.elapsed_time(e1)
    status = ctx.sync(stream)
    if status not in (B.SPH_OK, B.SPH_E_HNOCONV):
        raise RuntimeError(f"timed status {B.STATUS_NAMES.get(status)}: {ctx.error()}")
    ms_max = max_over_ranks(ms, world, dev)
    # the same K steps again with per-phase CUDA events inside the library
    # (the kernels launched one by one between the events): the phase split
    # and the force phase's time per launch for the roofline
    reset()
    ctx.timing_enable(True)
    ctx.step(prm, arr, nsteps=args.steps, stream=stream)
    phase_ms, phase_launches, tsteps = ctx.timing_read()
    ctx.timing_enable(False)
    ctx.sync(stream)
    out = {"n": n, "prm": prm, "state": s, "ms": ms_max, "ms_per_step": ms_max / args.steps,
           "value": whole_job_rate(world, n, args.steps, ms_max), "launches": launches,
           "status": B.STATUS_NAMES.get(status), "wall": (w0, w1),
           "phases_ms_per_step": {k: v / max(tsteps, 1) for k, v in phase_ms.items()},
           "launches_per_phase": phase_launches}

    # step 0 alone from the initial conditions (the longest h search): the timed
    # run's first step is this same work, so the rest gives the steady state
    reset()
    torch.cuda.synchronize(dev)
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    ctx.step(prm, arr, nsteps=1, stream=stream)
    g1.record(stream)
    torch.cuda.synchronize(dev)
    step0_ms = g0.elapsed_time(g1)
    ctx.sync(stream)
    out["steady_state"] = None
    if args.steps > 1 and ms > step0_ms:
        sms = (ms - step0_ms) / (args.steps - 1)
        out["steady_state"] = {"ms_per_step": sms, "value": world * n / (sms * 1e-3),
                               "step0_ms": step0_ms,
                               "steps": f"2-{args.steps} of the timed run (total minus a separate "
                                        f"step 0)"}

    out["e2e"] = None
    if e2e:
        # through the C ABI on HOST buffers (sph_step_host): every step reads
        # the state from pinned host memory, steps, and writes it back (all
        # but m, which the step only reads)
        ic_host = {k: torch.from_numpy(np.ascontiguousarray(s[k])) for k in B.STATE_FIELDS}
        host = {k: v.clone().pin_memory() for k, v in ic_host.items()}
        host["time"] = torch.zeros(1, dtype=torch.float64).pin_memory()
        host["dt"] = torch.zeros(1, dtype=torch.float64).pin_memory()
        ctx.step_host(prm, host, nsteps=1, stream=stream)  # untimed: allocates the staging
        torch.cuda.synchronize(dev)
        for k in B.STATE_FIELDS:
            host[k].copy_(ic_host[k])
        host["time"].zero_()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        f0.record(stream)
        for _ in range(args.steps):
            ctx.step_host(prm, host, nsteps=1, stream=stream)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        ems = max_over_ranks(f0.elapsed_time(f1), world, dev)
        ctx.sync(stream)
        out["e2e"] = {"value": whole_job_rate(world, n, args.steps, ems), "unit": UNIT,
                      "h2d_bytes_per_step": 8 * len(B.STATE_FIELDS) * n + 8,
                      "d2h_bytes_per_step": 8 * (len(B.STATE_FIELDS) - 1) * n + 16,
                      "api": "sph_step_host (C ABI, pinned host arrays: read in place by the "
                             "first kernel, results streamed back by a copy kernel)"}
    out["roofline"] = None
    if rank == 0:
        # the last step of the timed configuration again, for its neighbour list
        reset()
        ctx.step(prm, arr, nsteps=args.steps, stream=stream)
        ctx.sync(stream)
        out["phase_timed_total_ms_per_step"] = sum(phase_ms.values()) / max(tsteps, 1)
        out["roofline"] = forces_roofline(B, ctx, arr, prm, phase_ms, tsteps, fp64_peak,
                                          fp32_peak)
    del ctx, arr, ic
    torch.cuda.empty_cache()
    return out


def _r(x, nd=4):
    """Round for the compact summary line (None passes through)."""
    if x is None:
        return None
    return float(f"{x:.{nd}g}")


def summary_of(main, extra, small, ensembles, serving, variants):
    """A few numbers per record, short enough to stay in a log's tail."""
    sm = {}
    if main.get("steady_state"):
        sm["steady_ms_per_step"] = _r(main["steady_state"]["ms_per_step"])
        sm["step0_ms"] = _r(main["steady_state"]["step0_ms"])
    sm["phases_ms"] = {k: _r(v, 3) for k, v in main["phases_ms_per_step"].items()}
    if small:
        sm["patch27k_ms_per_step"] = _r(small["ms_per_step"])
    for name, r in extra.items():
        sm[name] = {"value": _r(r["value"]), "ms_per_step": _r(r["ms_per_step"]),
                    "e2e": _r(r["e2e"]["value"]) if r.get("e2e") else None,
                    "roofline_frac": _r(r["roofline"]["frac"], 3) if r.get("roofline") else None,
                    "forces_ms": _r(r["phases_ms_per_step"]["forces"], 3)}
    for prec, e in ensembles.items():
        sm[f"ensemble_{prec}"] = {
            "batched_ups": _r(e["batched"]["updates_per_s"]),
            "staged_p50_p99_s": [_r(e["staged"]["latency_ms_p50"] / 1e3, 3),
                                 _r(e["staged"]["latency_ms_p99"] / 1e3, 3)],
            "single_ups": _r(e["single_instance_path"]["updates_per_s"]),
            "single_p50_p99_s": [_r(e["single_instance_path"]["latency_ms_p50"] / 1e3, 3),
                                 _r(e["single_instance_path"]["latency_ms_p99"] / 1e3, 3)],
            "bitwise": e["batched_equals_single_bitwise"]}
    if serving:
        sv = {"requests": (serving.get("batched_fp64") or {}).get("requests")}
        for k in ("batched_fp64", "batched_mixed", "single_instance_fp64"):
            r = serving.get(k)
            if not r:
                continue
            d = {"p50_p99_s": [_r(r["latency_p50"], 3), _r(r["latency_p99"], 3)],
                 "served_ups": _r(r["served_updates_per_s"])}
            if "split" in r:
                d["p99_tickwait_queue_run_s"] = [_r(r["split"][q]["p99"], 3)
                                                 for q in ("tick_wait", "queueing", "run")]
            sv[k] = d
        sv["offered_ups"] = _r(serving["batched_fp64"]["offered_updates_per_s"]) \
            if "batched_fp64" in serving else None
        sm["serving"] = sv
    if variants:
        sm["variants_ms_frac"] = [[v["kernel"], v["gradients"], v["precision"],
                                   _r(v["ms_per_step"], 3), _r(v["roofline"]["frac"], 3)]
                                  for v in variants["runs"]]
    return sm


def run_native(args):
    import torch
    import torch.distributed as dist

    from paper_1809_08013_gb300 import binding as B

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo",
                                init_method="env://")
    if not torch.cuda.is_available():
        raise RuntimeError("the native arm needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.load()
    stream = torch.cuda.current_stream(dev)
    fp64_peak = B.probe_fma_peak(local, fp64=True, stream=stream)
    fp32_peak = B.probe_fma_peak(local, fp64=False, stream=stream)

    uuid = None
    try:
        u = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
        if u is not None:
            us = str(u)
            uuid = us if us.startswith("GPU-") else "GPU-" + us
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid) if rank == 0 else None
    main = measure_workload(args, B, dev, fp64_peak, fp32_peak, e2e=not args.no_e2e,
                            sampler=sampler)
    if sampler:
        time.sleep(0.3)
        sampler.stop()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    s, prm, n = main["state"], main["prm"], main["n"]
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        oracle.step(prm, s, nsteps=1)
        tc = time.perf_counter() - t0
        cpu = {"value": n / tc, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
               "sample": f"one oracle step (plain C FP64, OpenMP) of the same {n:,}-particle "
                         f"{args.workload} from its initial conditions: {tc:.1f} s",
               "gpu_speedup": main["value"] / (n / tc)}
        if args.workload == "patch":
            cpu["small_case"] = oracle_small_case(oracle, args)

    solo = world == 1 and args.workload == "patch" and args.precision == "fp64"
    small = gpu_small_case(args, B, dev) if args.workload == "patch" and world == 1 else None
    extra = {}
    if solo and not args.no_extra_workloads:
        # configuration 3 (Evrard 10^6, mixed precision) and the benchmark patch
        # with native FP64 pair sums, each the same K steps from its initial
        # conditions
        for name, wl, prec in (("evrard_mixed", "evrard", "mixed"),
                               ("fp64_pipe", "patch", "fp64-pipe")):
            a2 = argparse.Namespace(**{**vars(args), "workload": wl, "precision": prec,
                                       "seed": None})
            r = measure_workload(a2, B, dev, fp64_peak, fp32_peak, e2e=not args.no_e2e)
            r["workload"] = workload_name(a2, r["n"])
            extra[name] = r
    ensembles = {}
    if solo and not args.no_ensemble:
        for prec in ("fp64", "mixed"):
            ensembles[prec] = run_ensemble(args, B, dev, prec)
    serving = run_serving(args, B, dev) if solo and not args.no_serving else None
    variants = (run_variants(args, B, dev, fp64_peak, fp32_peak)
                if solo and not args.no_variants else None)

    clocks = sampler.summary(*main["wall"]) if sampler else None

    def public(r):
        return {k: v for k, v in r.items() if k not in ("prm", "state", "wall")}

    detail = {"main": public(main), "extra_workloads": {k: public(v) for k, v in extra.items()},
              "small_case": small, "ensemble": ensembles, "serving": serving,
              "variants": variants}
    print(json.dumps({"detail": detail}), flush=True)
    print(json.dumps({"summary": summary_of(main, extra, small, ensembles, serving, variants)}),
          flush=True)
    rl = dict(main["roofline"])
    for k in ("fp64_probe_tflops", "fp32_probe_tflops", "achieved_at_75_per_pair",
              "counted_flops_per_pair", "av_pair_fraction", "pairs_per_launch", "peak_source"):
        rl.pop(k, None)
    cpu_short = {k: v for k, v in (cpu or {}).items() if k != "small_case"} or None
    line = {"metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": main["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": workload_name(args), "n_particles": n,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (state ~0.2 GB + neighbour rows ~0.9 GB)"},
            "roofline": rl, "cpu_baseline": cpu_short, "e2e": main["e2e"],
            "gpu_launches": main["launches"], "clocks": clocks, "status": main["status"]}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
