#!/usr/bin/env python
"""Benchmark of the MAS-PNCG timestep on one B300 (or N replicas).

Workload: the 64-sphere pile (46,656 vertices, 196,608 tets, seeded random
non-overlapping centres in a 1 m box, E log-uniform in [1e4, 1e6] Pa,
dt = 1/60 s, tol 1e-3), FP32 bulk arithmetic with FP64 for positions,
barrier distances, CCD, the 2x2 and capacitance solves and the energy
checks.  One bench step is one implicit-Euler timestep (Algorithm 1 to
convergence).  Inputs are synthetic and resident in HBM when the timed region
starts; L2 is flushed (256 MB write) before every timed step.

Prints one JSON line whose `value` is PNCG iterations per second over the
timed timesteps (timesteps/s beside it).  `--impl reference` times the FP64
CPU oracle instead, on bounded samples of the same workload, in the same
unit.
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
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16"])
    ap.add_argument("--bf16-steps", type=int, default=-1,
                    help="timesteps of the BF16-factor form (IPC_PREC_BF16_MAS) beside the main one (-1 = --steps, 0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--plain-steps", type=int, default=-1,
                    help="timesteps of the plain FP64 form timed for the comparison (-1 = as many as --steps, 0 = skip)")
    ap.add_argument("--cpu-iters", type=int, default=4,
                    help="PNCG iterations of timestep 0 in the oracle's cpu_baseline sample")
    ap.add_argument("--replays", type=int, default=30, help="L2-flushed replays per stage for the roofline")
    ap.add_argument("--profile-replays", action="store_true",
                    help="call cudaProfilerStart/Stop around the roofline replays (ncu --profile-from-start off)")
    ap.add_argument("--serve", type=int, default=16,
                    help="scenes in the serving measurement (ipc_server, 0 = skip)")
    ap.add_argument("--ablation", type=int, default=0,
                    help="timesteps of the ablation runs (MAS maintenance, CCD step; 0 = skip)")
    ap.add_argument("--stiffness-sweep", type=int, default=0,
                    help="timesteps per case of the stiffness sweep, MAS vs 3x3 block-Jacobi (0 = skip)")
    ap.add_argument("--serve-stream", type=int, default=0,
                    help="requests of the serving stream (Poisson arrivals at 200 timesteps/s over a pool of "
                         "scenes; 0 = skip)")
    ap.add_argument("--pool", type=int, default=200, help="config-3-sized scenes in the serving pool")
    ap.add_argument("--torus", type=int, default=10,
                    help="distinct torus-chain scenes of the serving stream (created on first request, "
                         "evicted least recently used when free device memory runs low)")
    ap.add_argument("--large", type=int, default=0,
                    help="timesteps of the large spiky-ball scene (8 balls, 1.13M vertices, 2.84M tets; 0 = skip)")
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


def fp32_alu_peak_tflops(sm_count, sm_mhz):
    """FP32 FMA peak of the GPU from its unit counts and clock: 128 FP32
    lanes per SM, 2 flops per FMA."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12


def invert_flops(nblocks):
    """Algorithmic flops of the batched block inversion: per 96 x 96 block a
    Cholesky factorisation (n^3 / 3) and the triangular inverse W = L^-1
    (n^3 / 3)."""
    n = 96
    return nblocks * 2 * n ** 3 / 3


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

    mas_blocks: every block factor once (all levels; packed lower triangle,
    96 x 97 / 2 values) + g read + z write.
    forms: per tet the packed Hessian (45), rest inverse (9) and 4 indices;
    per vertex z and p read once.
    """
    mas = nblocks * (96 * 97 // 2) * rsize + 2 * 3 * nv * rsize
    forms = nt * (54 * rsize + 16) + 2 * 3 * nv * rsize + nv * 8
    return {"mas_blocks": mas, "forms": forms}


# DRAM bytes per launch (read + write) from one ncu capture of each kernel in
# its current form on the same workload (profiles/ holds the summaries and
# commands); None where the kernel changed since its last capture
TRAFFIC = {
    # DRAM bytes per launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum)
    # on the 64-sphere pile, replayed after an L2-evicting read.
    # k_invert_tiled (FP32 first pass of the block inversion), 1,507 blocks:
    ("invert", "fp32"): 65064704 + 2966016,
    # k_block_apply_plain (FP32 factors, all 1,507 blocks, no Woodbury patch):
    ("mas_blocks", "fp32"): 29716480 + 0,
    # k_forms_all (FP32 bulk):
    ("forms", "fp32"): 49571584 + 99584,
}


def host_cpu():
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return os.cpu_count() or 1, model


def oracle_iters_per_s(sc, iters, threads):
    """Wall time of the oracle's first `iters` PNCG iterations of timestep 0
    (iter_max = iters), on `threads` host threads (its independent loops run
    in parallel; results do not depend on the count)."""
    import oracle as O
    used = O.set_threads(threads)
    o = O.Scene(sc, params={"iter_max": iters})
    t0 = time.perf_counter()
    _, _, st = o.step(sc["x0"], sc["v0"])
    dt = time.perf_counter() - t0
    return st["iters"] / dt, dt, used, st["iters"]


def run_cpu_baseline(sc, iters):
    """The oracle as it stands on a bounded sample of the workload: the first
    `iters` PNCG iterations of timestep 0, single thread and all host cores."""
    ncpu, model = host_cpu()
    v1, dt1, _, n1 = oracle_iters_per_s(sc, iters, 1)
    vn, dtn, used, nn = oracle_iters_per_s(sc, iters, ncpu)
    return {
        "value": vn,
        "unit": "PNCG iters/s",
        "cores": used,
        "kind": "oracle",
        "sample": (f"first {nn} PNCG iterations of timestep 0 of the same workload (FP64 oracle: level-0 "
                   f"inverses rebuilt every iteration): {dtn:.1f} s on {used} threads, {dt1:.1f} s on 1 thread"),
        "single_thread": {"value": v1, "unit": "PNCG iters/s", "cores": 1},
        "nproc": ncpu,
        "cpu_model": model,
    }


def run_reference(args):
    """--impl reference: the FP64 CPU oracle timed on host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2604_19892_b300 import scenes as S
    import oracle as O
    sc = S.sphere_pile()
    ncpu, model = host_cpu()
    used = O.set_threads(ncpu)
    # each reference step: the first two PNCG iterations of timestep 0 (a
    # restart and a Woodbury iteration), from the workload's initial state
    o = O.Scene(sc, params={"iter_max": 2})
    for _ in range(args.warmup):
        o.step(sc["x0"], sc["v0"])
    times, iters = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, _, st = o.step(sc["x0"], sc["v0"])
        times.append(time.perf_counter() - t0)
        iters += st["iters"]
    total = sum(times)
    iters_per_s = iters / total
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
        "config": {"workload": WORKLOAD, "sample": "each step = the first 2 PNCG iterations of timestep 0 (FP64 oracle)"},
        "cpu_baseline": {"value": iters_per_s, "unit": "PNCG iters/s", "cores": used, "kind": "oracle",
                         "sample": f"first 2 PNCG iterations of timestep 0 per step, {used} host threads",
                         "nproc": ncpu, "cpu_model": model},
        "e2e": {"value": iters_per_s, "unit": "PNCG iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_bf16(args, ipc, S, m, flush, stream, peak, warmup):
    """The same timesteps with the block factors in BF16 (IPC_PREC_BF16_MAS:
    tensor-core block products, FP32 accumulation), device-timed like the main
    loop, and its block applies replayed for their roofline."""
    import torch
    sc = S.sphere_pile()
    g = ipc.Scene(sc, precision=ipc.IPC_PREC_BF16_MAS)
    for _ in range(warmup):
        g.step(1)
    g.set_state(sc["x0"], sc["v0"])
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(m)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(m)]
    its, conv = 0, 0
    torch.cuda.synchronize()
    for k in range(m):
        flush.fill_(float(k))
        e0[k].record(stream)
        st = g.step(1)
        e1[k].record(stream)
        its += st["iters"]
        conv += st["converged"]
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in zip(e0, e1))
    nv = sc["x0"].shape[0]
    nblocks = sum(int(q.max()) + 1 for q, _ in g.levels())
    byts = nblocks * (96 * 97 // 2) * 2 + 2 * 3 * nv * 4
    roof = {}
    for stg, sid, kern in (("mas_blocks", 2, "k_block_apply_plain16"), ("mas_woodbury", 4, "k_block_apply<float, true>")):
        us = 1e3 * g.profile_replay(sid, args.replays, flush=flush, stream=stream)
        ach = byts / (us * 1e-6) / 1e9
        roof[stg] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                     "bytes_per_launch": byts, "avg_us": us, "kernel": kern}
    g.close()
    return {"precision": "bf16 block factors, fp32 bulk", "timesteps": f"0..{m - 1}", "iters_per_s": its / (ms / 1e3),
            "timesteps_per_s": m / (ms / 1e3), "mean_iters_per_step": its / m, "converged_steps": conv,
            "roofline_stages": roof}


def run_stiffness_sweep(args, ipc, S, prec):
    """The paper's preconditioner comparison over material stiffness (Sec.
    5.1): two 8^3-cell cubes stacked 5 mm apart above the ground with seeded
    random vertex velocities (0.2 m/s per component, exciting the elastic
    modes), Young's modulus E in {1e4 .. 1e7} Pa (kappa follows E); from the
    same initial state, `args.stiffness_sweep` timesteps with MAS (Woodbury
    maintenance) and with 3x3 block-Jacobi preconditioning on the same PNCG
    iteration. The convergence test max |z| <= tol h bbox depends on P: a
    weak preconditioner can meet it early, so the energy each reaches is
    reported beside the iteration counts."""
    import torch
    out = []
    for E in (1e4, 1e5, 1e6, 1e7):
        sc = S.two_cubes(n=8, gap=0.005)
        sc["v0"] = 0.2 * np.random.default_rng(5).normal(size=sc["x0"].shape)
        sc["E"] = np.full_like(sc["E"], E)
        sc["params"] = S.default_params(S.bbox_diag(sc["x0"]), sc["params"]["h"], E)
        row = {"E": E}
        for name, prm in (("mas", {}), ("block_jacobi", {"mas_mode": 3})):
            g = ipc.Scene(sc, params=prm, precision=prec)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = g.step(args.stiffness_sweep)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            row[name] = {"iters_per_step": st["iters"] / args.stiffness_sweep,
                         "ms_per_step": 1e3 * dt / args.stiffness_sweep, "converged": st["converged"],
                         "final_energy": st["energy"]}
            g.close()
        out.append(row)
    return {"scene": "two_cubes(n=8, gap=0.005), random v0, E scaled", "timesteps": args.stiffness_sweep,
            "rows": out}


def run_serve_stream(args, ipc, S, rate=200.0, torus_frac=0.1, n_torus=10, slots=8, margin_gb=40.0, wall_cap_s=240.0,
                     creators=4):
    """Serving stream: timestep requests arrive as a Poisson process (`rate`
    per second, seed 3), each for a scene drawn from a pool of `args.pool`
    config-3-sized scenes (500-20k vertices, cubes, balls and rods) and, with
    probability `torus_frac`, from `n_torus` stacks of interlocked torus rings
    of 100k-300k vertices. The small scenes are made resident before the
    stream starts. A torus scene is created on its first request by a pool of
    `creators` host threads (its requests wait for it; the rest of the stream
    goes on meanwhile). Admission: while free device memory is below
    `margin_gb`, idle torus scenes are destroyed, least recently used first.
    Requests run through ipc_server (continuous batching, `slots` at once);
    latency is completion minus arrival, queueing and scene creation included.
    After `wall_cap_s` no new request is submitted (the line then reports how
    many arrived and ran)."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    rng = np.random.default_rng(3)
    t0 = time.perf_counter()
    pool = []
    for k, sc in enumerate(S.batched_scenes(n_scenes=args.pool, seed=2)):
        pool.append(ipc.Scene(sc, precision=ipc.IPC_PREC_FP32, use_torch_allocator=False))
        if k % 50 == 49:
            print(f"serving pool: {k + 1} scenes resident after {time.perf_counter() - t0:.1f} s", file=sys.stderr,
                  flush=True)
    pool_s = time.perf_counter() - t0
    sizes = np.exp(rng.uniform(np.log(1e5), np.log(3e5), size=n_torus))
    torus = {}            # id -> Scene (resident)
    creating = {}         # id -> (future, start time)
    waiting = {}          # id -> arrival times of requests waiting for the scene
    last_use = {}
    busy = {}             # scene key -> live tickets
    created = evicted = 0
    free0, total = torch.cuda.mem_get_info()
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=args.serve_stream))
    picks = [("t", int(rng.integers(n_torus))) if rng.uniform() < torus_frac else ("s", int(rng.integers(args.pool)))
             for _ in range(args.serve_stream)]

    def make_torus(i):
        return ipc.Scene(S.torus_stack(int(sizes[i]), seed=1000 + i), precision=ipc.IPC_PREC_FP32,
                         use_torch_allocator=False)

    ex = ThreadPoolExecutor(max_workers=creators)
    srv = ipc.Server(slots=slots)
    live = {}
    lat, steps_done, torus_steps, create_s = [], 0, 0, 0.0
    lat_kind = {"s": [], "t": []}
    nxt = 0
    start = time.perf_counter()
    capped = False

    def submit(scene, arr, key):
        busy[key] = busy.get(key, 0) + 1
        live[srv.submit(scene, 1)] = (arr, key)

    while nxt < len(picks) or live or creating:
        now = time.perf_counter() - start
        if now > wall_cap_s and nxt < len(picks):
            capped = True
            picks = picks[:nxt]
        while nxt < len(picks) and arrivals[nxt] <= now:
            kind, i = picks[nxt]
            if kind == "s":
                submit(pool[i], arrivals[nxt], (kind, i))
            else:
                torus_steps += 1
                last_use[i] = now
                if i in torus:
                    submit(torus[i], arrivals[nxt], (kind, i))
                else:
                    waiting.setdefault(i, []).append(arrivals[nxt])
                    if i not in creating:
                        while torch.cuda.mem_get_info()[0] < margin_gb * 1e9:
                            idle = [j for j in torus if busy.get(("t", j), 0) == 0]
                            if not idle:
                                break
                            j = min(idle, key=lambda q: last_use.get(q, 0.0))
                            torus.pop(j).close()
                            evicted += 1
                        creating[i] = (ex.submit(make_torus, i), time.perf_counter())
            nxt += 1
        for i, (fut, tc) in list(creating.items()):
            if fut.done():
                torus[i] = fut.result()
                del creating[i]
                created += 1
                create_s += time.perf_counter() - tc
                print(f"serving stream: torus scene {i} ({torus[i].nv} vertices) created in "
                      f"{time.perf_counter() - tc:.1f} s at {time.perf_counter() - start:.1f} s", file=sys.stderr,
                      flush=True)
                for arr in waiting.pop(i, []):
                    submit(torus[i], arr, ("t", i))
        done = []
        for tk, (arr, key) in live.items():
            r = srv.poll(tk)
            if r is not None:
                lat.append(1e3 * (time.perf_counter() - start - arr))
                lat_kind[key[0]].append(lat[-1])
                if key[0] == "t":
                    print(f"serving stream: torus {key[1]} step done, {r['iters']} iterations, latency "
                          f"{lat[-1]:.0f} ms", file=sys.stderr, flush=True)
                busy[key] -= 1
                steps_done += 1
                done.append(tk)
                if steps_done % 200 == 0:
                    print(f"serving stream: {steps_done} done at {time.perf_counter() - start:.1f} s, torus created "
                          f"{created}", file=sys.stderr, flush=True)
        for tk in done:
            del live[tk]
        if not done:
            time.sleep(2e-4)
    wall = time.perf_counter() - start
    ex.shutdown()
    srv.close()
    for g in pool:
        g.close()
    for g in torus.values():
        g.close()
    lat.sort()

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))] if v else None

    small = len(lat_kind["s"])
    return {"requests": len(picks), "capped_at_s": wall_cap_s if capped else None, "rate_per_s": rate,
            "pool_scenes": args.pool, "torus_scenes": n_torus, "torus_frac": torus_frac, "slots": slots,
            "creator_threads": creators, "pool_setup_s": pool_s, "device_gb_after_pool": (total - free0) / 1e9,
            "torus_created": created, "torus_evicted": evicted, "torus_create_s_summed": create_s,
            "torus_requests": torus_steps, "small_requests": small, "timesteps_per_s": steps_done / wall,
            "arrival_span_s": float(arrivals[-1]), "wall_s": wall,
            "latency_ms_p50": lat[len(lat) // 2], "latency_ms_p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
            "latency_ms_small_p50_p99": [pct(lat_kind["s"], 0.5), pct(lat_kind["s"], 0.99)],
            "latency_ms_torus_p50_p99": [pct(lat_kind["t"], 0.5), pct(lat_kind["t"], 0.99)],
            "latency": "completion minus arrival, queueing and torus scene creation included"}


def run_large(args, ipc, S, prec):
    """The large scene shaped like the paper's teaser: eight spiky balls
    (1,132,296 vertices, 2,840,064 tets), `args.large` timesteps of their drop
    and collisions, FP32 bulk; per timestep its iterations, contacts and
    device time."""
    import torch
    t0 = time.perf_counter()
    sc = S.spiky_balls()
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    g = ipc.Scene(sc, precision=prec)
    setup_s = time.perf_counter() - t0
    free, total = torch.cuda.mem_get_info()
    print(f"large scene: generated in {gen_s:.1f} s, set up in {setup_s:.1f} s, {(total - free) / 1e9:.1f} GB in use",
          file=sys.stderr, flush=True)
    rows = []
    g.profile(True)  # per-stage device times (events around each stage)
    for k in range(args.large):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = g.step(1)
        torch.cuda.synchronize()
        rows.append({"t": k, "ms": 1e3 * (time.perf_counter() - t0), "iters": st["iters"],
                     "restarts": st["restarts"], "contacts": st["n_contacts"], "converged": st["converged"],
                     "min_dist": st["min_dist"]})
        rows[-1]["stage_ms"] = {kk: round(v["ms"], 1) for kk, v in g.profile_read().items()}
        print(f"large scene timestep {k}: {rows[-1]}", file=sys.stderr, flush=True)
        g.profile(True)  # reset the counters
    g.profile(False)
    g.close()
    its = sum(r["iters"] for r in rows)
    secs = sum(r["ms"] for r in rows) / 1e3
    return {"scene": "spiky_balls(n_balls=8): 32^3-cell balls with 200 spikes each", "vertices": int(sc["x0"].shape[0]),
            "tets": int(sc["tets"].shape[0]), "generation_s": gen_s, "setup_s": setup_s,
            "device_bytes_in_use_after_setup": int(total - free), "timesteps": args.large,
            "iters_per_s": its / secs if secs else None, "timesteps_per_s": args.large / secs if secs else None,
            "peak_contacts": max((r["contacts"] for r in rows), default=0), "per_step": rows}


def run_ablation(args, ipc, S, prec):
    """The paper's ablations on the same kernels: MAS maintenance (Woodbury
    updates, full rebuild every iteration, frozen between restarts) and the
    CCD step (per subdomain, global), `args.ablation` timesteps of the
    workload each."""
    import torch
    sc = S.sphere_pile()
    out = {}
    for name, prm in (("woodbury_per_subdomain", {}), ("full_rebuild", {"mas_mode": 1}), ("freeze", {"mas_mode": 2}),
                      ("block_jacobi", {"mas_mode": 3}), ("global_alpha", {"ccd_mode": 1})):
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
        ms = g.profile_replay(sid, args.replays, flush=flush, stream=stream)
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
    prec = {"fp32": ipc.IPC_PREC_FP32, "fp64": ipc.IPC_PREC_FP64, "bf16": ipc.IPC_PREC_BF16_MAS}[args.precision]
    rsize = 8 if prec == ipc.IPC_PREC_FP64 else 4
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

    # roofline. The kernel with the largest device-time share on this
    # workload is the batched block inversion of the restarts (an ALU-bound
    # dense factorisation; profiles/launches_sphere_pile_fp32_step15.md); the
    # per-iteration HBM-bound stages (MAS apply with and without the
    # Woodbury update, H~ quadratic forms) are reported beside it. Each is
    # replayed on the final state of the timed run: reps x (256 MB L2-evicting
    # read, stage) minus reps x (read) between CUDA events on the launch
    # stream, divided by reps.
    peak, peak_kind = load_peaks()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = clk["sm_mhz"] or 2032.0
    alu_peak = fp32_alu_peak_tflops(sm_count, sm_mhz)
    by = stage_bytes(nv, nt, nblocks, rsize)
    if args.profile_replays:
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
    stage_us = {}
    for stg, sid in (("invert", 0), ("mas_blocks", 2), ("mas_woodbury", 4), ("forms", 3)):
        stage_us[stg] = 1e3 * scene.profile_replay(sid, args.replays, flush=flush, stream=stream)
    if args.profile_replays:
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    fl = invert_flops(nblocks)
    tr_inv = TRAFFIC.get(("invert", args.precision))
    # the SIMT pipes' FMA throughput measured on this GPU (outside the timed
    # region), beside the unit-count peak: the FP32 pass is the inversion
    # timed here, the FP64 pipe the precision of the paper's own design
    fma = {"fp32": ipc.fma_peak_tflops(ipc.IPC_PREC_FP32), "fp64": ipc.fma_peak_tflops(ipc.IPC_PREC_FP64)}
    roof = {
        "invert": {"bound": "alu", "achieved": fl / (stage_us["invert"] * 1e-6) / 1e12, "peak": alu_peak,
                   "unit": "TFLOP/s", "frac": fl / (stage_us["invert"] * 1e-6) / 1e12 / alu_peak,
                   "traffic": tr_inv if nblocks == 1507 else None, "flops_per_launch": fl,
                   "avg_us": stage_us["invert"],
                   "kernel": "k_invert_tiled" if prec == ipc.IPC_PREC_FP32 else "k_invert",
                   "peak_source": (f"FP32 FMA peak from unit counts: {sm_count} SMs x 128 lanes x 2 flops x "
                                   f"{sm_mhz:.0f} MHz (median SM clock of the timed region)"),
                   "measured_fma_tflops": fma,
                   "frac_of_measured_fma": (fl / (stage_us["invert"] * 1e-6) / 1e12 /
                                            fma["fp32" if prec != ipc.IPC_PREC_FP64 else "fp64"])},
    }
    for stg, kern in (("mas_blocks", "k_block_apply_plain"), ("mas_woodbury", "k_block_apply"),
                      ("forms", "k_forms_all")):
        key = "mas_blocks" if stg == "mas_woodbury" else stg
        ach = by[key] / (stage_us[stg] * 1e-6) / 1e9
        roof[stg] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                     "traffic": TRAFFIC.get((stg, args.precision)), "bytes_per_launch": by[key],
                     "avg_us": stage_us[stg], "kernel": kern,
                     "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}
    for v in roof.values():
        v["timing"] = (f"{args.replays} replays on the final state, 256 MB read before each (L2 evicted), "
                       "difference of two CUDA-event-timed loops")
    dominant = "invert"

    # stage breakdown: a separate profiled pass over the same timesteps (the
    # per-stage events need the kernels launched one by one, so the timed
    # loop above runs without them and with its CUDA graphs)
    n_prof = args.steps
    scene.set_state(sc["x0"], sc["v0"])
    scene.profile(True)
    for _ in range(n_prof):
        scene.step(1)
    prof = scene.profile_read()
    scene.profile(False)
    for stg, src in (("mas_blocks", "mas_blocks"), ("forms", "forms"), ("invert", "restart")):
        n = prof[src]["launches"]
        roof[stg]["in_loop_stage_avg_us"] = 1e3 * prof[src]["ms"] / n if n else None
        roof[stg]["in_loop_stage"] = src
        roof[stg]["in_loop_launches"] = n

    serving = run_serving(args, ipc, S) if args.serve > 0 and world == 1 else None
    ablation = run_ablation(args, ipc, S, prec) if args.ablation > 0 and world == 1 else None
    sweep = run_stiffness_sweep(args, ipc, S, prec) if args.stiffness_sweep > 0 and world == 1 else None
    large = run_large(args, ipc, S, prec) if args.large > 0 and world == 1 else None
    stream = run_serve_stream(args, ipc, S, n_torus=args.torus) if args.serve_stream > 0 and world == 1 else None
    scale = run_scale(args, ipc, S, prec, rsize, flush, stream, peak) if args.scale > 0 and world == 1 else None

    # end-to-end through the C ABI with host buffers: per step the state goes
    # host -> device, the step runs, positions and velocities come back
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(np.ascontiguousarray(sc["x0"])).pin_memory()
        vh = torch.from_numpy(np.ascontiguousarray(sc["v0"])).pin_memory()
        xo = torch.empty_like(xh).pin_memory()
        n_e2e = args.steps  # the same timesteps as the device-timed loop
        it_e2e = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(n_e2e):
            scene.set_state(xh.numpy(), vh.numpy())
            it_e2e += scene.step(1)["iters"]
            xo.copy_(torch.from_numpy(scene.positions()))
            vh.copy_(torch.from_numpy(scene.velocities()))
            xh.copy_(xo)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": world * it_e2e / dt, "unit": "PNCG iters/s", "timesteps_per_s": world * n_e2e / dt,
               "h2d_bytes_per_step": 2 * 3 * nv * 8, "d2h_bytes_per_step": 2 * 3 * nv * 8, "steps": n_e2e}

    # plain form: the same timesteps in FP64 on the GPU (the method without
    # mixed precision). Each step the FP32 form is also run, untimed, from the
    # plain form's state, and its positions compared with the plain form's
    plain = None
    m = args.steps if args.plain_steps < 0 else min(args.plain_steps, args.steps)
    if m > 0 and prec == ipc.IPC_PREC_FP32:
        s64 = ipc.Scene(sc, precision=ipc.IPC_PREC_FP64)
        s32 = ipc.Scene(sc, precision=ipc.IPC_PREC_FP32)
        for _ in range(args.warmup):
            s64.step(1)
            s32.step(1)
        s64.set_state(sc["x0"], sc["v0"])
        bbox = s64.bbox_diag()
        q0 = [torch.cuda.Event(enable_timing=True) for _ in range(m)]
        q1 = [torch.cuda.Event(enable_timing=True) for _ in range(m)]
        it64, errs = 0, []
        torch.cuda.synchronize()
        for k in range(m):
            xk, vk = s64.positions(), s64.velocities()
            flush.fill_(float(k))
            q0[k].record(stream)
            it64 += s64.step(1)["iters"]
            q1[k].record(stream)
            s32.set_state(xk, vk)
            s32.step(1)
            errs.append(float(np.abs(s32.positions() - s64.positions()).max() / bbox))
        torch.cuda.synchronize()
        ms64 = sum(a.elapsed_time(b) for a, b in zip(q0, q1))
        ms32 = sum(step_ms[:m])
        it32 = sum(st["iters"] for st in status[:m])
        plain = {"precision": "fp64", "timesteps": f"0..{m - 1}",
                 "iters_per_s": it64 / (ms64 / 1e3), "timesteps_per_s": m / (ms64 / 1e3), "iters": it64,
                 "mixed_iters_per_s": it32 / (ms32 / 1e3), "mixed_timesteps_per_s": m / (ms32 / 1e3),
                 "mixed_iters": it32, "speedup_iters_per_s": (it32 / ms32) / (it64 / ms64),
                 "speedup_timesteps": ms64 / ms32,
                 "fp32_step_err_max": max(errs), "fp32_step_err_median": statistics.median(errs),
                 "fp32_step_err_unit": "max_v |x_fp32 - x_fp64| / bbox diagonal, one timestep from the same state"}
        del s64, s32

    bf16 = None
    mb = args.steps if args.bf16_steps < 0 else min(args.bf16_steps, args.steps)
    if mb > 0 and world == 1 and prec == ipc.IPC_PREC_FP32:
        bf16 = run_bf16(args, ipc, S, mb, flush, stream, peak, args.warmup)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(sc, args.cpu_iters)

    if rank != 0:
        return
    sorted_ms = sorted(step_ms)
    p50 = statistics.median(sorted_ms)
    p99 = sorted_ms[min(len(sorted_ms) - 1, int(math.ceil(0.99 * len(sorted_ms))) - 1)]
    line = {
        "metric": METRIC,
        "value": iters_per_s,
        "unit": "PNCG iters/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if prec == ipc.IPC_PREC_FP64 else "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "scene": "sphere_pile(n_balls=64, cells=8, seed=1)",
                   "precision": args.precision, "timesteps": f"0..{args.steps - 1}",
                   "l2": "flushed before every timed step (256 MB write)", "parallelism": "replicas" if world > 1 else "single"},
        "timesteps_per_s": steps_per_s,
        "mean_iters_per_step": iters / args.steps,
        "p50_ms": p50,
        "p99_ms": p99,
        "converged_steps": sum(s["converged"] for s in status),
        "ccd_fallbacks": sum(s["ccd_fallbacks"] for s in status),
        "fp64_redo_blocks_last_restart": scene.fp64_blocks() if prec == ipc.IPC_PREC_FP32 else None,
        "plain_fp64_iters_per_s": plain["iters_per_s"] if plain else None,
        "plain_fp64_timesteps_per_s": plain["timesteps_per_s"] if plain else None,
        "fp32_vs_fp64_step_err_max": plain["fp32_step_err_max"] if plain else None,
        "vs_plain_fp64": plain,
        "bf16_mas": bf16,
        "roofline": dict(roof[dominant], kernel=roof[dominant]["kernel"]),
        "roofline_stages": roof,
        "stage_ms": {k: v["ms"] for k, v in prof.items()},
        "stage_ms_timesteps": f"0..{n_prof - 1}, a separate profiled pass (kernels launched one by one)",
        "serving": serving,
        "ablation": ablation,
        "stiffness_sweep": sweep,
        "large": large,
        "serve_stream": stream,
        "scale": scale,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
