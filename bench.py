#!/usr/bin/env python
"""Benchmark of the MAS-PNCG timestep on one B300 (or N replicas).

Workload: the 64-sphere pile (46,656 vertices, 196,608 tets, seeded random
non-overlapping centres in a 1 m box, E log-uniform in [1e4, 1e6] Pa,
dt = 1/60 s, tol 1e-3), FP32 bulk arithmetic with FP64 for positions,
barrier distances, CCD, the 2x2 and capacitance solves and the energy
checks.  One bench step is one implicit-Euler timestep (Algorithm 1 to
convergence).  Inputs are synthetic and resident in HBM when the timed region
starts; L2 is flushed (256 MB write) before every timed step.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead,
on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PNCG iters/s & steps/s vs plain form at fixed grad tol; p50/p99 step latency"
WORKLOAD = ("64-sphere pile: 46,656 verts, 196,608 tets, 1 m box, E log-uniform [1e4,1e6] Pa, dt 1/60 s, "
            "gradient-norm tol 1e-3, FP32 bulk with FP64 barrier/CCD/2x2/energy")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--plain-steps", type=int, default=12,
                    help="timesteps of the plain FP64 form timed for the comparison (0 = skip)")
    ap.add_argument("--replays", type=int, default=30, help="L2-flushed replays per stage for the roofline")
    ap.add_argument("--profile-replays", action="store_true",
                    help="call cudaProfilerStart/Stop around the roofline replays (ncu --profile-from-start off)")
    ap.add_argument("--serve", type=int, default=16,
                    help="scenes in the serving measurement (ipc_server, 0 = skip)")
    ap.add_argument("--ablation", type=int, default=0,
                    help="timesteps of the ablation runs (MAS maintenance, CCD step; 0 = skip)")
    ap.add_argument("--scale", type=int, default=5,
                    help="timesteps of the large-scene run (512 spheres in a 2.5 x 2 x 2.5 m box; 0 = skip)")
    ap.add_argument("--profile-from-step", type=int, default=-1,
                    help="call cudaProfilerStart before this timed step (for ncu --profile-from-start off)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(v, world):
    """The largest v over the ranks of the process group (v itself alone):
    the whole job takes as long as its slowest replica. The tensor lives on
    the device the group's backend reduces on (GPU for NCCL, host for gloo)."""
    if world <= 1:
        return float(v)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rates(total_ms, world, steps, iters):
    """Timesteps/s and PNCG iterations/s of the whole job: every rank steps
    its own replica, so the work is world x (steps, iters) in the slowest
    rank's time (iters taken from this rank's replica: the replicas are
    the same scene)."""
    secs = total_ms / 1e3
    return world * steps / secs, world * iters / secs


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return pk.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def stage_bytes(nv, nt, nblocks, rsize):
    """Algorithmic bytes per launch of the two per-iteration HBM-bound stages.

    mas_blocks: every 96x96 inverse block once (all levels) + g read + z write.
    forms: per tet the packed Hessian (45), rest inverse (9) and 4 indices;
    per vertex z and p read once.
    """
    mas = nblocks * 96 * 96 * rsize + 2 * 3 * nv * rsize
    forms = nt * (54 * rsize + 16) + 2 * 3 * nv * rsize + nv * 8
    return {"mas_blocks": mas, "forms": forms}


# DRAM bytes per launch from ncu captures of the same kernels (unchanged
# since), scaled by the units a launch processes: profiles/ holds the
# summaries and commands
TRAFFIC = {
    ("mas_blocks", "fp32"): {"bytes_per_block": (56.330496e6 + 0.015872e6) / 1507},
    ("forms", "fp32"): {"bytes_per_tet": (49.594880e6 + 0.052736e6) / 196608},
}


def run_cpu_baseline(sc, gpu_iters_per_step):
    """The oracle as it stands, one PNCG iteration of timestep 0 (bounded sample)."""
    import oracle as O
    o = O.Scene(sc, params={"iter_max": 1})
    t0 = time.perf_counter()
    o.step(sc["x0"], sc["v0"])
    dt = time.perf_counter() - t0
    iters_per_s = 1.0 / dt
    return {
        "value": iters_per_s / max(gpu_iters_per_step, 1e-9),
        "unit": "timesteps/s",
        "cores": 1,
        "kind": "oracle",
        "sample": (f"1 PNCG iteration of timestep 0 of the same workload ({dt:.2f} s, single thread); "
                   f"timesteps/s = oracle iters/s / GPU mean iters per timestep ({gpu_iters_per_step:.1f})"),
        "iters_per_s": iters_per_s,
    }


def run_reference(args):
    """--impl reference: the FP64 CPU oracle timed on host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2604_19892_b300 import scenes as S
    import oracle as O
    sc = S.sphere_pile()
    # each reference step: one PNCG iteration of the timestep, iterations chained
    o = O.Scene(sc, params={"iter_max": 1})
    x, v = sc["x0"].copy(), sc["v0"].copy()
    for _ in range(args.warmup):
        o.step(x, v)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.step(x, v)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    iters_per_s = args.steps / total
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": iters_per_s,
        "unit": "PNCG iters/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "each step = 1 PNCG iteration of timestep 0 (FP64 oracle)"},
        "cpu_baseline": {"value": iters_per_s, "unit": "PNCG iters/s", "cores": 1, "kind": "oracle",
                         "sample": "1 PNCG iteration of timestep 0 per step, single thread"},
        "e2e": {"value": iters_per_s, "unit": "PNCG iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ablation(args, ipc, S, prec):
    """The paper's ablations on the same kernels: MAS maintenance (Woodbury
    updates, full rebuild every iteration, frozen between restarts) and the
    CCD step (per subdomain, global), `args.ablation` timesteps of the
    workload each."""
    import torch
    sc = S.sphere_pile()
    out = {}
    for name, prm in (("woodbury_per_subdomain", {}), ("full_rebuild", {"mas_mode": 1}), ("freeze", {"mas_mode": 2}),
                      ("global_alpha", {"ccd_mode": 1})):
        g = ipc.Scene(sc, params=prm, precision=prec)
        g.step(1)  # one-time setup and graph captures
        g.set_state(sc["x0"], sc["v0"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = g.step(args.ablation)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[name] = {"timesteps": args.ablation, "iters_per_step": st["iters"] / args.ablation,
                     "rebuilds_per_step": st["restarts"] / args.ablation, "ms_per_step": 1e3 * dt / args.ablation,
                     "converged": st["converged"]}
        g.close()
    return out


def run_scale(args, ipc, S, prec, rsize, flush, stream, peak):
    """The same method on a scene 8x the workload's: 512 spheres in a
    2.5 x 2 x 2.5 m box, `args.scale` timesteps, plus the roofline replays of
    the MAS apply and the forms at that size."""
    import torch
    sc = S.sphere_pile(n_balls=512, box=(2.5, 2.0, 2.5))
    t0 = time.perf_counter()
    g = ipc.Scene(sc, precision=prec)
    setup_s = time.perf_counter() - t0
    nv, nt = sc["x0"].shape[0], sc["tets"].shape[0]
    nblocks = sum(int(q.max()) + 1 for q, _ in g.levels())
    g.step(1)
    g.set_state(sc["x0"], sc["v0"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = g.step(args.scale)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    by = stage_bytes(nv, nt, nblocks, rsize)
    roof = {}
    for stg, sid in (("mas_blocks", 2), ("forms", 3)):
        ms = statistics.median(g.profile_replay(sid, 1, flush=flush, stream=stream) for _ in range(args.replays))
        roof[stg] = {"avg_us": ms * 1e3, "achieved_GBs": by[stg] / (ms / 1e3) / 1e9,
                     "frac": by[stg] / (ms / 1e3) / 1e9 / peak, "bytes_per_launch": by[stg]}
    g.close()
    return {"scene": "sphere_pile(n_balls=512, box=(2.5, 2, 2.5))", "vertices": int(nv), "tets": int(nt),
            "blocks": nblocks, "timesteps": args.scale, "timesteps_per_s": args.scale / dt,
            "iters_per_s": st["iters"] / dt, "iters_per_step": st["iters"] / args.scale,
            "converged": st["converged"], "setup_s": setup_s, "roofline": roof}


def run_serving(args, ipc, S, steps_per_scene=6, slots=8):
    """Continuous batching through ipc_server: one closed-loop client per
    scene (it submits one timestep, and the next when that one returns), for
    `args.serve` scenes of 500-20k vertices (log-uniform), FP32 bulk. Against
    it, the same timesteps with each scene stepped alone one after another,
    in the plain FP64 form and in FP32."""
    import torch
    scs = S.batched_scenes(n_scenes=args.serve, seed=2)
    nv = [int(sc["x0"].shape[0]) for sc in scs]

    def make(prec):
        return [ipc.Scene(sc, precision=prec, use_torch_allocator=False) for sc in scs]

    def sequential(scenes):
        for g, sc in zip(scenes, scs):  # warm-up: one-time setup and graph captures
            g.set_state(sc["x0"], sc["v0"])
            g.step(2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for g, sc in zip(scenes, scs):
            g.set_state(sc["x0"], sc["v0"])
            g.step(steps_per_scene)
        torch.cuda.synchronize()
        return len(scs) * steps_per_scene / (time.perf_counter() - t0)

    plain = make(ipc.IPC_PREC_FP64)
    seq64 = sequential(plain)
    for g in plain:
        g.close()
    mixed = make(ipc.IPC_PREC_FP32)
    seq32 = sequential(mixed)
    for g, sc in zip(mixed, scs):
        g.set_state(sc["x0"], sc["v0"])
    srv = ipc.Server(slots=slots)
    left = [steps_per_scene] * len(scs)
    lat = []
    t0 = time.perf_counter()
    live = {srv.submit(g, 1): i for i, g in enumerate(mixed)}
    while live:
        done = []
        for tk, i in live.items():
            r = srv.poll(tk)
            if r is not None:
                lat.append(r["latency_ms"])
                done.append((tk, i))
        for tk, i in done:
            del live[tk]
            left[i] -= 1
            if left[i] > 0:
                live[srv.submit(mixed[i], 1)] = i
        if not done:
            time.sleep(2e-4)
    wall = time.perf_counter() - t0
    srv.close()
    for g in mixed:
        g.close()
    served = len(scs) * steps_per_scene / wall
    lat.sort()
    return {"scenes": len(scs), "vertices": f"{min(nv)}..{max(nv)} (total {sum(nv)})",
            "timesteps_per_scene": steps_per_scene, "slots": slots, "unit": "timesteps/s",
            "served_fp32": served, "sequential_fp32": seq32, "sequential_plain_fp64": seq64,
            "speedup_vs_plain": served / seq64, "latency_ms_p50": lat[len(lat) // 2],
            "latency_ms_p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2604_19892_b300 import build, ipc
    from paper_2604_19892_b300 import scenes as S
    build.build()
    ipc.load()
    prec = ipc.IPC_PREC_FP32 if args.precision == "fp32" else ipc.IPC_PREC_FP64
    rsize = 4 if prec == ipc.IPC_PREC_FP32 else 8
    sc = S.sphere_pile()
    scene = ipc.Scene(sc, precision=prec)
    nv, nt = sc["x0"].shape[0], sc["tets"].shape[0]
    nblocks = sum(int(g.max()) + 1 for g, _ in scene.levels())
    stream = torch.cuda.current_stream()

    # warm-up steps from the initial state, then reset so the timed steps are
    # timesteps 0..K-1 of the workload
    for _ in range(args.warmup):
        scene.step(1)
    scene.set_state(sc["x0"], sc["v0"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ipc.kernel_launches()
    iters = 0
    status = []
    for k in range(args.steps):
        if k == args.profile_from_step:
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
        flush.fill_(float(k))
        ev0[k].record(stream)
        st = scene.step(1)
        ev1[k].record(stream)
        iters += st["iters"]
        status.append(st)
    torch.cuda.synchronize()
    if args.profile_from_step >= 0:
        torch.cuda.profiler.stop()
    launches = ipc.kernel_launches() - launches0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    total_ms = max_over_ranks(sum(step_ms), world)
    steps_per_s, iters_per_s = whole_job_rates(total_ms, world, args.steps, iters)

    # roofline of the two per-iteration HBM-bound stages (MAS block apply,
    # H~ quadratic forms): their kernels replayed on the final state of the
    # timed run, 256 MB written before each replay to evict L2, a CUDA event
    # pair on the launch stream around the stage's launches only (the
    # in-loop stage events also catch host launch gaps; reported beside)
    peak, peak_kind = load_peaks()
    by = stage_bytes(nv, nt, nblocks, rsize)
    roof = {}
    if args.profile_replays:
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
    for stg, sid in (("mas_blocks", 2), ("forms", 3)):
        # median of single-launch replays (robust to the odd slow launch)
        avg_ms = statistics.median(scene.profile_replay(sid, 1, flush=flush, stream=stream)
                                   for _ in range(args.replays))
        ach = by[stg] / (avg_ms / 1e3) / 1e9
        tr = TRAFFIC.get((stg, args.precision))
        traffic = tr["bytes_per_block"] * nblocks if tr and stg == "mas_blocks" else (
            tr["bytes_per_tet"] * nt if tr else None)
        roof[stg] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                     "traffic": traffic, "bytes_per_launch": by[stg], "avg_us": avg_ms * 1e3,
                     "timing": f"median of {args.replays} replays on the final state, 256 MB read before each (L2 evicted), CUDA events",
                     "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}
    if args.profile_replays:
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    dominant = "mas_blocks"

    # stage breakdown: a separate profiled pass over the first timesteps (the
    # per-stage events need the kernels launched one by one, so the timed
    # loop above runs without them and with its CUDA graphs)
    n_prof = min(args.steps, 8)
    scene.set_state(sc["x0"], sc["v0"])
    scene.profile(True)
    for _ in range(n_prof):
        scene.step(1)
    prof = scene.profile_read()
    scene.profile(False)
    for stg in roof:
        n = prof[stg]["launches"]
        roof[stg]["in_loop_avg_us"] = 1e3 * prof[stg]["ms"] / n if n else None
        roof[stg]["in_loop_launches"] = n

    serving = run_serving(args, ipc, S) if args.serve > 0 and world == 1 else None
    ablation = run_ablation(args, ipc, S, prec) if args.ablation > 0 and world == 1 else None
    scale = run_scale(args, ipc, S, prec, rsize, flush, stream, peak) if args.scale > 0 and world == 1 else None

    # end-to-end through the C ABI with host buffers: per step the state goes
    # host -> device, the step runs, positions come back device -> host
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(np.ascontiguousarray(sc["x0"])).pin_memory()
        vh = torch.from_numpy(np.ascontiguousarray(sc["v0"])).pin_memory()
        xo = torch.empty_like(xh).pin_memory()
        n_e2e = args.steps  # the same timesteps as the device-timed loop
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(n_e2e):
            scene.set_state(xh.numpy(), vh.numpy())
            scene.step(1)
            xo.copy_(torch.from_numpy(scene.positions()))
            vh.copy_(torch.from_numpy(scene.velocities()))
            xh.copy_(xo)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": world * n_e2e / dt, "unit": "timesteps/s", "h2d_bytes_per_step": 2 * 3 * nv * 8,
               "d2h_bytes_per_step": 2 * 3 * nv * 8, "steps": n_e2e}

    # plain form: the same timesteps in FP64 on the GPU (the method without
    # mixed precision), compared over the first plain_steps timesteps
    plain = None
    if args.plain_steps > 0 and prec == ipc.IPC_PREC_FP32:
        m = min(args.plain_steps, args.steps)
        s64 = ipc.Scene(sc, precision=ipc.IPC_PREC_FP64)
        for _ in range(args.warmup):
            s64.step(1)
        s64.set_state(sc["x0"], sc["v0"])
        q0 = [torch.cuda.Event(enable_timing=True) for _ in range(m)]
        q1 = [torch.cuda.Event(enable_timing=True) for _ in range(m)]
        it64 = 0
        torch.cuda.synchronize()
        for k in range(m):
            flush.fill_(float(k))
            q0[k].record(stream)
            it64 += s64.step(1)["iters"]
            q1[k].record(stream)
        torch.cuda.synchronize()
        ms64 = sum(a.elapsed_time(b) for a, b in zip(q0, q1))
        ms32 = sum(step_ms[:m])
        it32 = sum(st["iters"] for st in status[:m])
        plain = {"precision": "fp64", "timesteps": f"0..{m - 1}",
                 "timesteps_per_s": m / (ms64 / 1e3), "iters_per_s": it64 / (ms64 / 1e3), "iters": it64,
                 "mixed_timesteps_per_s": m / (ms32 / 1e3), "mixed_iters_per_s": it32 / (ms32 / 1e3),
                 "mixed_iters": it32, "speedup_timesteps": (m / (ms32 / 1e3)) / (m / (ms64 / 1e3))}
        del s64

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(sc, iters / max(args.steps, 1))

    if rank != 0:
        return
    sorted_ms = sorted(step_ms)
    p50 = statistics.median(sorted_ms)
    p99 = sorted_ms[min(len(sorted_ms) - 1, int(math.ceil(0.99 * len(sorted_ms))) - 1)]
    line = {
        "metric": METRIC,
        "value": steps_per_s,
        "unit": "timesteps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == ipc.IPC_PREC_FP32 else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "scene": "sphere_pile(n_balls=64, cells=8, seed=1)",
                   "precision": args.precision, "timesteps": f"0..{args.steps - 1}",
                   "l2": "flushed before every timed step (256 MB write)", "parallelism": "replicas" if world > 1 else "single"},
        "iters_per_s": iters_per_s,
        "mean_iters_per_step": iters / args.steps,
        "p50_ms": p50,
        "p99_ms": p99,
        "converged_steps": sum(s["converged"] for s in status),
        "vs_plain_fp64": plain,
        "roofline": roof.get(dominant) if dominant else None,
        "roofline_stages": roof,
        "stage_ms": {k: v["ms"] for k, v in prof.items()},
        "stage_ms_timesteps": f"0..{n_prof - 1}, a separate profiled pass (kernels launched one by one)",
        "serving": serving,
        "ablation": ablation,
        "scale": scale,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    if dominant:
        line["roofline"]["kernel"] = dominant
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
