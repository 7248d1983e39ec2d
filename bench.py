#!/usr/bin/env python3
"""MPAP hot-path benchmark: plan-edge expansions/s and ms/query on the 6D
double-integrator workload (16000 samples per roadmap, 30 boxes, 32^3 quality
grid, 4096 Monte Carlo rollouts), batched versus plain.

One step processes a batch of B seeded queries (default 64) through the whole
hot path: roadmap construction (Alg. 2 with per-edge heuristic transfers), one
lock-step batched wavefront search (Alg. 3), and batched Monte Carlo
certification of the returned plans.  The scene inputs are resident in HBM
before timing starts; every step builds ~1.6 GB of roadmaps, larger than L2, so
no L2 flush is needed between steps.

  value   plan-edge expansions of the step / step time (device CUDA events)
  e2e     the same through the C ABI with host scene buffers (copies timed)
  plain   the same queries searched one call at a time (search only), reported
          beside the batched search-only numbers

`--impl reference` times the CPU oracle (single thread, as it stands) on a bounded
sample of the same workload (one query per step) and prints the same line.
Launch with torchrun for N > 1: queries are sharded by rank (weak scaling, no
collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import scenegen  # noqa: E402

METRIC = "plan-edge expansions/s and ms/query (6D, 16k samples), batched vs plain"
UNIT = "expansions/s"
WORKLOAD = "6D double integrator, 16000 samples, 30 boxes, 32^3 grid, 4096 MC rollouts"


def log(msg):
    sys.stderr.write(f"[bench {time.strftime('%H:%M:%S')}] {msg}\n")
    sys.stderr.flush()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mpap", choices=["mpap", "reference"])
    ap.add_argument("--queries", type=int, default=64, help="queries per step per GPU")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-refine", action="store_true")
    ap.add_argument("--no-perception", action="store_true")
    ap.add_argument("--no-update", action="store_true")
    ap.add_argument("--no-errnet", action="store_true")
    ap.add_argument("--no-vio", action="store_true")
    ap.add_argument("--sur-train-plans", type=int, default=200000,
                    help="Monte Carlo-labelled candidate plans to train the surrogate on")
    ap.add_argument("--sur-train-steps", type=int, default=2000)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


def shard_seeds(rank, count):
    """Scene seeds of one rank: every rank takes its own `count` queries (weak
    scaling; the queries are independent, so no data-path collective)."""
    return [rank * count + i + 1 for i in range(count)]


def reduce_over_ranks(ms_total, exps, device=None):
    """(max over ranks of the timed region, sum over ranks of the expansions):
    the only collectives of a multi-GPU run, and only for reporting."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms_total, exps
    t = torch.tensor([float(ms_total)], dtype=torch.float64, device=device)
    e = torch.tensor([float(exps)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t[0]), float(e[0])


def scenes_for_rank(rank, count):
    cfg = scenegen.config("6d")
    calib = scenegen.load_calibration()
    out = []
    for seed in shard_seeds(rank, count):
        sc = scenegen.make_scene(cfg, seed, query_id=seed)
        key = scenegen.calib_key(cfg, seed)
        sc.extra["beta"] = calib[key]["beta"] if key in calib else None
        out.append(sc)
    return out


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0])); smax.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ GPU arm
class GpuArm:
    def __init__(self, scenes, device):
        import torch
        import paper_1705_02408_gb300 as mp
        self.mp, self.torch = mp, torch
        self.scenes = scenes
        self.device = device
        self.cfg = scenes[0].cfg
        # scene inputs resident in HBM
        self.dev_inputs = [(torch.from_numpy(s.box_lo).to(device), torch.from_numpy(s.box_hi).to(device),
                            torch.from_numpy(s.grid).to(device)) for s in scenes]
        V = self.cfg.n + 2
        # plan arena, group array and candidate overflow areas: 2^19 records per query
        self.max_plans = len(scenes) << 19
        self.ws = mp.Workspace(V * len(scenes), front_cap=64, max_plans=self.max_plans)
        self.ws1 = mp.Workspace(V, front_cap=64, max_plans=1 << 22)
        self.queries = [mp.make_query(s.extra["beta"], scenegen.LAMBDA) for s in scenes]
        self.mc = [(self.cfg.mc_rollouts, s.mc_seed, 0, s.delta_fx, s.sigma_fx, s.shift) for s in scenes]

    def build(self, host=False):
        """All roadmaps of the batch in one mpap_build_roadmaps call, rebuilt into
        the handles of the previous step (no device allocation once sizes repeat)."""
        mp = self.mp
        specs = [mp.scene_spec(s, device_inputs=None if host else d) for s, d in zip(self.scenes, self.dev_inputs)]
        self.rms = mp.build_roadmaps(specs, rms=getattr(self, "rms", None))
        return self.rms

    def step(self, host=False):
        mp = self.mp
        rms = self.build(host)
        res = mp.search_batch(self.ws, rms, self.queries)
        certs = mp.certify_batch(rms, [r.path for r in res], self.mc)
        exps = sum(r.expansions for r in res)
        self._last = (rms, res, certs)
        return exps

    def io_bytes(self):
        h2d = sum(s.box_lo.nbytes + s.box_hi.nbytes + s.grid.nbytes + s.sigma_fx.nbytes + s.shift.nbytes
                  for s in self.scenes)
        rms, res, certs = self._last
        h2d += sum(4 * len(r.path) for r in res)
        d2h = sum(4 * len(r.path) + 8 * 4 for r in res) + 16 * len(certs)
        return h2d, d2h


def run_gpu(args, rank, world, local):
    import torch
    import paper_1705_02408_gb300 as mp
    from paper_1705_02408_gb300 import build as mpbuild
    mpbuild.build()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    scenes = scenes_for_rank(rank, args.queries)
    if any(s.extra["beta"] is None for s in scenes):
        raise SystemExit("missing beta for some scenes: run python -m oracle.calibrate --seeds N")
    arm = GpuArm(scenes, device)
    stream = torch.cuda.current_stream()
    # launch shapes from the autotuner (edge block size; select/prune grids)
    tuning = None
    if not args.no_autotune:
        specs = [mp.scene_spec(s, device_inputs=d) for s, d in zip(arm.scenes, arm.dev_inputs)]
        tb, b_ms, arm.rms = mp.autotune_build(specs, reps=1)
        ts, s_ms = mp.autotune_search(arm.ws, arm.rms, arm.queries, reps=1)
        if ts["front_cap"] > arm.ws.front_cap:
            arm.ws = mp.Workspace(arm.ws.total_nodes, front_cap=ts["front_cap"], max_plans=arm.max_plans)
        tuning = {"edge_warps": tb["edge_warps"], "wave_blocks_per_sm": ts["wave_blocks_per_sm"],
                  "plan_lanes_from": ts["plan_lanes_from"], "front_cap": arm.ws.front_cap,
                  "tuned_build_ms": round(b_ms, 3), "tuned_search_ms": round(s_ms, 3)}

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    log("autotuned; warm-up")
    for _ in range(args.warmup):
        arm.step()
    log("timed region")
    # timed region: K steps, device events, library profiler off, clocks sampled
    mp.profile_enable(False)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    launches0 = mp.launch_count()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    exps = 0
    for _ in range(args.steps):
        exps += arm.step()
    e1.record(stream)
    barrier()
    launches = mp.launch_count() - launches0
    ck = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    # per-kernel breakdown in a separate pass over the same steps, with CUDA
    # events around every launch (the library profiler), so that the timed
    # value above carries no profiling overhead
    log("breakdown pass")
    mp.profile_reset()
    mp.profile_enable(True)
    for _ in range(args.steps):
        arm.step()
    torch.cuda.synchronize()
    mp.profile_enable(False)
    kern = mp.profile_read()
    ms = ms_total / args.steps
    if world > 1:
        ms_total, exps = reduce_over_ranks(ms_total, exps, device)
        ms = ms_total / args.steps
    value = exps / (ms_total / 1e3)
    rms, res, certs = arm._last
    per_query = args.queries
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+i64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "queries_per_step": per_query * world,
                      "queries_per_gpu": per_query, "l2": "inputs larger than L2 (~1.6 GB of roadmaps built per step)",
                      "lambda": scenegen.LAMBDA, "beta": "60th percentile of straight-line heuristic",
                      "parallelism": f"queries sharded over {world} GPU(s)"},
           "ms_per_query": ms / per_query,
           "gpu_launches": int(launches),
           "tuning": tuning,
           "breakdown": "per-kernel times from a second pass of the same steps with per-launch CUDA events"}
    # breakdown from the live kernel timers (timed region)
    search_k = {"k_init", "k_wave", "k_finalize", "k_candidates"}
    certify_k = {"k_mc_checkpoints", "k_mc_rollouts"}
    phase = {"build": 0.0, "search": 0.0, "certify": 0.0}
    for k, (_, t) in kern.items():
        if "." in k:
            continue    # a phase inside a kernel (k_wave.expand, ...), already in the kernel's time
        phase["search" if k in search_k else "certify" if k in certify_k else "build"] += t / args.steps
    out["kernel_ms_per_step"] = {k: round(v[1] / args.steps, 4) for k, v in sorted(kern.items())}
    out["phase_kernel_ms_per_step"] = {p: round(t, 4) for p, t in phase.items()}
    out["expansions_per_step"] = exps / args.steps
    out["solved"] = sum(1 for r in res if r.status == 0)
    out["certified_failure_rate"] = sum(c["hits_any"] for c in certs) / max(1, sum(c["rollouts"] for c in certs))
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    out["roofline"] = roofline(kern, arm, res, args.steps, sms=sms)
    # the two kernels that share most of the step, each against its own bound
    out["roofline_by_kernel"] = [roofline(kern, arm, res, args.steps, name=k, sms=sms) for k in ("k_wave", "k_edges")
                                 if k in kern]
    if ck:
        out["clocks"] = ck
    if rank == 0 and not args.no_plain:
        out["search_only"] = search_only(arm, stream)
    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e(arm, args, stream)
    log("timed region done")
    if rank == 0 and not args.no_refine:
        out["refine"] = refine_report(arm)
    if rank == 0 and not args.no_vio:
        out["vio_certify"] = vio_report(arm)
    if rank == 0 and not args.no_perception:
        out["perception_levels"] = perception_report(arm)
    if rank == 0 and not args.no_update:
        out["online_update"] = update_report(arm)
    if rank == 0 and not args.no_errnet:
        out["learned_heuristic"] = errnet_report(arm)
    if rank == 0 and world == 1 and not args.no_mixed:
        out["mixed_batch"] = mixed_report(args, stream)
    if rank == 0 and world == 1 and not args.no_surrogate:
        log("surrogate")
        out["surrogate"] = surrogate_report(args, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(scenes[:2], scenes[2:2 + 16])
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


# DRAM traffic from ncu captures, per unit of work, valid only while the kernel
# sources are the ones that were captured.
NCU_TRAFFIC = {
    # one row-pass launch over 8 roadmaps: 13.24 MB read + 89.72 MB written
    # (profiles/k_edges_6d16k.md)
    "k_edges": {"bytes_per_roadmap": (13.243392e6 + 89.717504e6) / 8,
                "sources": {"paper_1705_02408_gb300/csrc/roadmap.cu": "19dc98e00769a158323b00e07af135847edc6571",
                            "paper_1705_02408_gb300/csrc/common.cuh": "c0e30decd0d668ce9cb5dd6fa1e41da2e91baa84"}},
    # one k_wave launch of the 8-query 6D-16k step: 169.44 MB read + 58.48 MB written
    # for 12,658,585 plan-edge expansions (profiles/k_wave_6d16k_8queries.md)
    "k_wave": {"bytes_per_expansion": (169.441024e6 + 58.480896e6) / 12658585.0,
               "sources": {"paper_1705_02408_gb300/csrc/search.cu": "eb8d2718e6dbb92e69d6baa632fffd30080a7cc7",
                           "paper_1705_02408_gb300/csrc/common.cuh": "c0e30decd0d668ce9cb5dd6fa1e41da2e91baa84"}},
}


def _traffic(kernel, units, key="bytes_per_roadmap"):
    import hashlib
    t = NCU_TRAFFIC.get(kernel)
    if not t or key not in t:
        return None
    for path, sha in t["sources"].items():
        with open(os.path.join(ROOT, path), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != sha:
                return None
    return t[key] * units


def roofline(kern, arm, res, steps, name=None, sms=152):
    """Roofline of one kernel (default: the dominant one) from the live
    CUDA-event timers."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    if name is None:
        name = max(((k, v) for k, v in kern.items() if "." not in k), key=lambda kv: kv[1][1])[0]
    launches, ms = kern[name]
    V = arm.cfg.n + 2
    B = len(arm.scenes)
    exps = sum(r.expansions for r in res)
    plans = sum(r.plans for r in res)
    if name.startswith("k_edges"):
        # ALU-bound binary32 work the method requires of the edge build (FMA is
        # disabled, so every operation is one lane-op):
        #  - one exactly evaluated Near test Cost(v, u) < r of the 6D double
        #    integrator: 39 operations, for every pair the build tests (counted
        #    on the device; cells outside the neighbour ball are never tested);
        #  - per connection kept (a lower bound on the connections that pass
        #    Near): steering setup 40, collision at the 15 interior checkpoints
        #    15 x 19 (time and a 3-axis Horner step) plus their bounding box 90,
        #    and the perception transfer at the 16 checkpoints 16 x 33 (Horner 19,
        #    grid index 14): 943 operations.
        tests = sum(rm.stats()[0] for rm in arm.rms)
        edges = sum(rm.E for rm in arm.rms)
        ops_per_launch = (39.0 * tests + 943.0 * edges) * steps / max(1, launches)
        achieved = ops_per_launch / (ms / launches / 1e3) / 1e12
        sm_max = peaks.get("sm_max_mhz", 2070.0)
        peak = sms * 128 * sm_max * 1e6 / 1e12
        return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                "frac": achieved / peak, "traffic": _traffic(name, B * steps / max(1, launches)),
                "traffic_unit": "DRAM bytes per launch (ncu, scaled from an 8-roadmap capture)",
                "near_tests_per_step": tests, "edges_per_step": edges,
                "ops_per_step": 39.0 * tests + 943.0 * edges,
                "all_pairs_per_step": V * V * B,
                "peak_source": f"derived: {sms} SMs (device) x 128 FP32 lanes x max SM clock "
                               "(MEASURED_PEAKS.json sm_max_mhz)"}
    # HBM-bound search kernels: algorithmic bytes per step, the 16-byte reverse edge
    # record per plan-edge expansion and a 24-byte front entry per plan
    bytes_step = 16.0 * exps + 24.0 * plans
    per_launch = bytes_step * steps / max(1, launches)
    achieved = per_launch / (ms / launches / 1e3) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    # DRAM traffic: bytes per plan-edge expansion from an ncu capture of every
    # launch of a smaller batch, times the expansions of one launch here
    traffic = None
    if name == "k_wave":
        traffic = _traffic(name, exps * steps / max(1, launches), "bytes_per_expansion")
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "traffic_unit": "DRAM bytes per launch (ncu, per expansion of an 8-query capture)",
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback"}


def search_only(arm, stream):
    """Batched (one call) versus plain (one call per query) search on the same
    roadmaps; device time by CUDA events."""
    import torch
    mp = arm.mp
    rms = arm.build()
    torch.cuda.synchronize()
    out = {}
    for mode in ("batched", "plain"):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        reps = 3
        exps = 0
        e0.record(stream)
        for _ in range(reps):
            if mode == "batched":
                res = mp.search_batch(arm.ws, rms, arm.queries)
            else:
                res = [mp.search(arm.ws1, rm, q.beta, lam=scenegen.LAMBDA) for rm, q in zip(rms, arm.queries)]
            exps += sum(r.expansions for r in res)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[mode] = {"expansions_per_s": exps / reps / (ms / 1e3), "ms_per_query": ms / len(rms),
                     "ms_per_batch": ms}
    # search + certify per query (batched)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = mp.search_batch(arm.ws, rms, arm.queries)
    mp.certify_batch(rms, [r.path for r in res], arm.mc)
    e1.record(stream)
    torch.cuda.synchronize()
    out["batched"]["ms_per_query_with_certify"] = e0.elapsed_time(e1) / len(rms)
    return out


def e2e(arm, args, stream):
    """Same step through the C ABI with host scene buffers (H2D/D2H inside)."""
    import torch
    for _ in range(1):
        arm.step(host=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    exps = 0
    for _ in range(args.steps):
        exps += arm.step(host=True)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1)
    h2d, d2h = arm.io_bytes()
    return {"value": exps / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "wall_value": exps / wall}


# ------------------------------------------------------------------ mixed batch
def perception_report(arm, features=256, reps=10):
    """Visible-feature perception levels (mpap_feature_levels) for the first
    benchmark scene's 32^3 quality grid: eight yaw headings with a 45-degree
    half field of view and range 0.5, and the all-direction table (range 2);
    device arrays, CUDA events around `reps` launches."""
    import torch
    mp = arm.mp
    sc = arm.scenes[0]
    G = sc.cfg.grid_G
    f = torch.from_numpy(scenegen.feature_points(sc, features)).cuda()
    lo, hi = (torch.from_numpy(a).cuda() for a in (sc.box_lo, sc.box_hi))
    out = {"workload": f"{features} features, {len(sc.box_lo)} boxes, {G}^3 cells"}
    for key, Y, ch, rng in (("yaw8_fov45_range0.5", 8, float(np.float32(np.cos(np.pi / 4))), 0.5),
                            ("all_direction_range2", 1, -2.0, 2.0)):
        heads = torch.from_numpy(scenegen.yaw_headings(Y)).cuda()
        for _ in range(2):
            mp.feature_levels(3, lo, hi, f, G, heads, ch, rng)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            lv = mp.feature_levels(3, lo, hi, f, G, heads, ch, rng)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        pairs = Y * G ** 3 * features
        out[key] = {"ms_per_table": ms, "cell_feature_pairs_per_s": pairs / (ms / 1e3),
                    "mean_level": float(lv.float().mean().item())}
    return out


def errnet_report(arm, n_train=200000, steps=400, batch=8192, n_map=20000):
    """The learned error-rate heuristic (Sec. 5.1): maximum-likelihood training of
    the 7-8-8-2 network on synthetic observations, its forward pass over the mapped
    states, the weighted 8-nearest-neighbour map queried at the benchmark scenes'
    6D roadmap nodes, and the level grid (32^3) for a roadmap build; CUDA events."""
    import torch
    mp = arm.mp
    X, r = scenegen.vio_samples(n_train, 11)
    Xd, rd = torch.from_numpy(X).cuda(), torch.from_numpy(r).cuda()
    net = mp.ErrNet(seed=5, max_batch=max(batch, n_map))
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    idx = torch.randint(0, n_train, (steps, batch), device="cuda", generator=g)
    for t in range(5):
        net.train_step(Xd[idx[t]], rd[idx[t]], lr=3e-3)
    out = {"network": "7-8-8-2 ReLU, Gaussian mean and std, maximum likelihood (binary32)"}
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for t in range(steps):
        loss, _ = net.train_step(Xd[idx[t]], rd[idx[t]], lr=3e-3)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out["train"] = {"steps": steps, "batch": batch, "ms_per_step": ms / steps,
                    "samples_per_s": steps * batch / (ms / 1e3), "final_loss": float(loss)}
    # the map: network evaluated at mapped states (synthetic inputs), queried at roadmap nodes
    M = torch.from_numpy(scenegen.mapped_states(n_map, 12)).cuda()
    Xm = torch.from_numpy(scenegen.vio_samples(n_map, 13)[0]).cuda()
    e0.record()
    vals = net.forward(Xm)
    e1.record()
    torch.cuda.synchronize()
    out["forward_ms_per_map"] = e0.elapsed_time(e1)
    rms = arm.rms
    xs = [rm.export()["x"] for rm in rms[:4]]
    q = np.concatenate([np.concatenate([x.T, np.zeros((x.shape[1], 1), np.float32)], 1) for x in xs])
    qd = torch.from_numpy(np.ascontiguousarray(q, np.float32)).cuda()
    for _ in range(2):
        mp.errmap_query(M, vals, qd, k=8, w=(4.0, 1.0, 0.25))
    torch.cuda.synchronize()
    e0.record()
    mp.errmap_query(M, vals, qd, k=8, w=(4.0, 1.0, 0.25))
    e1.record()
    torch.cuda.synchronize()
    qms = e0.elapsed_time(e1)
    out["map_query"] = {"map_states": n_map, "queries": int(len(q)), "k": 8, "ms": qms,
                        "pairs_per_s": n_map * len(q) / (qms / 1e3)}
    e0.record()
    lv = mp.errmap_levels(M, vals, 6, 32, vel=(0.5, 0.0, 0.0), yaw=0.0, mu_ref=0.02, k=8)
    e1.record()
    torch.cuda.synchronize()
    out["levels_32cubed_ms"] = e0.elapsed_time(e1)
    out["levels_mean"] = float(lv.float().mean().item())
    return out


def update_report(arm, k=3, side=0.3):
    """Online update (mpap_roadmap_update_batch) of the benchmark's roadmaps in one
    call, against rebuilding all of them in one batched build; CUDA events around
    each.  Two map changes: k added boxes each with the levels of the cells inside
    one cube of the given side replaced (new features mapped there: only the edges
    near the boxes and that cube are re-tested and re-transferred), and k added
    boxes with an entirely new grid (every edge is re-transferred)."""
    import torch
    rng = np.random.default_rng(7)
    G = arm.cfg.grid_G
    cen = (np.arange(G) + 0.5) / G
    adds, local, fresh = [], [], []
    for s in arm.scenes:
        c = rng.uniform(0.2, 0.8, (k, 3)); sz = rng.uniform(0.04, 0.12, (k, 3))
        adds.append(((c - sz / 2).astype(np.float32), (c + sz / 2).astype(np.float32)))
        other = scenegen.make_scene(arm.cfg, s.seed + 1000).grid
        lo = rng.uniform(0.0, 1.0 - side, 3)
        ins = [(cen >= lo[i]) & (cen < lo[i] + side) for i in range(3)]
        m = (ins[2][:, None, None] & ins[1][None, :, None] & ins[0][None, None, :]).ravel()
        g = s.grid.copy()
        g[m] = other[m]
        local.append(g)
        fresh.append(other)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    out = {"workload": f"{len(arm.scenes)} roadmaps of {arm.cfg.n + 2} nodes, one batched update call"}
    for name, grids in (("boxes_and_local_grid", local), ("boxes_and_new_grid", fresh)):
        rms = arm.build()
        E0 = sum(rm.E for rm in rms)
        torch.cuda.synchronize()
        e0.record()
        arm.mp.roadmap_update_batch(rms, [a[0] for a in adds], [a[1] for a in adds], grids)
        e1.record()
        torch.cuda.synchronize()
        ms_update = e0.elapsed_time(e1)
        E1 = sum(rm.E for rm in rms)
        out[name] = {"change": f"{k} added boxes each and " + (f"the cells inside one cube of side {side} given "
                                                                 "new levels" if grids is local else "a new grid"),
                     "ms_per_roadmap_update": ms_update / len(rms), "edges_before": E0, "edges_after": E1}
        # the same update once more with per-launch events (a separate pass)
        rms = arm.build()
        torch.cuda.synchronize()
        arm.mp.profile_reset()
        arm.mp.profile_enable(True)
        arm.mp.roadmap_update_batch(rms, [a[0] for a in adds], [a[1] for a in adds], grids)
        torch.cuda.synchronize()
        arm.mp.profile_enable(False)
        out[name]["kernel_ms"] = {kk: round(v[1], 4) for kk, v in sorted(arm.mp.profile_read().items())}
    e0.record()
    arm.build()
    e1.record()
    torch.cuda.synchronize()
    out["ms_per_roadmap_rebuild"] = e0.elapsed_time(e1) / len(arm.scenes)
    return out


# closed-loop VIO model parameters (per checkpoint step, 2^-20 units): inertial
# noise, position-fix noise at the lowest level with a fix (falling as
# 1/sqrt(level)), LQR weights (q_p, q_w, r)
VIO_Q_A, VIO_R_MAX, VIO_FIX_FROM, VIO_LQR_WEIGHTS = 60, 2048, 3, (1.0, 0.5, 20.0)


def vio_report(arm):
    """The benchmark's 64 plans certified under the closed-loop VIO model (LQR
    tracking, inertial prediction, Kalman fixes) in one batched call, beside the
    error-walk certification of the same plans; CUDA events around each."""
    import torch
    mp = arm.mp
    rms, res, _ = arm._last
    paths = [r.path for r in res]
    kp, kv = mp.vio_lqr_gains(*VIO_LQR_WEIGHTS)
    lev = np.arange(25)
    table = np.where(lev >= VIO_FIX_FROM, np.rint(VIO_R_MAX * np.sqrt(VIO_FIX_FROM / np.maximum(lev, 1))),
                     0).astype(np.int32)
    mcs = [(m[0], m[1], m[2], m[3]) for m in arm.mc]
    vios = [(VIO_Q_A, kp, kv, table)] * len(rms)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    mp.certify_vio_batch(rms, paths, mcs, vios)          # warm-up
    torch.cuda.synchronize()
    e0.record()
    out = mp.certify_vio_batch(rms, paths, mcs, vios)
    e1.record()
    torch.cuda.synchronize()
    ms_vio = e0.elapsed_time(e1)
    e0.record()
    mp.certify_batch(rms, paths, arm.mc)
    e1.record()
    torch.cuda.synchronize()
    ms_walk = e0.elapsed_time(e1)
    R = sum(o["rollouts"] for o in out)
    return {"workload": f"{len(rms)} plans of the benchmark step, {arm.cfg.mc_rollouts} rollouts each",
            "model": {"q_a_fx": VIO_Q_A, "lqr_weights": VIO_LQR_WEIGHTS, "kp_q16": kp, "kv_q16": kv,
                      "r_fx_max": VIO_R_MAX, "fix_from_level": VIO_FIX_FROM},
            "ms_per_batch": ms_vio, "ms_per_batch_error_walk": ms_walk,
            "failure_rate": sum(o["hits_any"] for o in out) / max(1, R),
            "localisation_rate": sum(o["hits_loc"] for o in out) / max(1, R),
            "collision_rate": sum(o["hits_coll"] for o in out) / max(1, R)}


def refine_report(arm, eps=0.05, rounds=8):
    """Perception-bound refinement (Alg. 1 step 4) of the benchmark's queries on
    their roadmaps: lock-step rounds of one batched search and one batched
    certification; device time by CUDA events around the whole refinement."""
    import collections
    import torch
    from paper_1705_02408_gb300.refine import refine_batch
    rms = arm.build()
    beta0 = [q.beta for q in arm.queries]
    max_hits = [int(np.floor(eps * m[0])) for m in arm.mc]
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    res = refine_batch(arm.ws, rms, beta0, arm.mc, max_hits, max_rounds=rounds)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    first = [r.history[0] for r in res]
    passed0 = [i for i, f in enumerate(first) if f[1] == "pass"]
    ratios = [res[i].cost / first[i][2] for i in passed0 if res[i].certified]
    return {"workload": f"the {len(res)} benchmark queries on their roadmaps, failure bound {eps} "
                        f"(hits <= {max_hits[0]} of {arm.mc[0][0]}), at most {rounds} rounds",
            "ms_per_batch": ms, "ms_per_query": ms / len(res),
            "certified": sum(r.certified for r in res), "queries": len(res),
            "rounds_mean": float(np.mean([r.rounds for r in res])), "rounds_max": max(r.rounds for r in res),
            "searches": sum(r.rounds for r in res),
            "mc_calls": sum(1 for r in res for h in r.history if h[1] in ("pass", "fail")),
            "search_errors": sum(1 for r in res for h in r.history if h[1] == "error"),
            "outcome_at_beta0": dict(collections.Counter(f[1] for f in first)),
            "rescued_by_tightening": sum(1 for r, f in zip(res, first) if f[1] != "pass" and r.certified),
            "cheaper_by_loosening": sum(1 for i in passed0 if res[i].cost < first[i][2]),
            "cost_ratio_mean_vs_beta0": float(np.mean(ratios)) if ratios else None}


def mixed_report(args, stream, count=256):
    """The batched workload: 256 queries, each on its own roadmap (dimension
    uniform over 2D/3D/6D, n log-uniform in [1000, 32000] for 3D/6D and [1000,
    4000] for 2D), obstacles and grids
    seeded per query, beta from the stored oracle calibration: built in one
    call, searched in one lock-step launch with autotuned shapes and certified in
    one launch.  The front pool holds 2048 entries per node of the batch, half of
    it shared out among the queries in proportion to their nodes; every query
    draws on its own share only (MPAP_QUERY_OWN_SHARE), so whether it runs out
    does not depend on the rest of the batch, and the few 2D queries whose exact
    Pareto fronts outgrow it (single fronts above 10^5 plans) end with a capacity
    status of their own, which the report counts.  The plain arm searches the
    queries that finished in the batch one call each."""
    import torch
    import paper_1705_02408_gb300 as mp
    calib = scenegen.load_calibration()
    scenes = []
    for d, n, s in scenegen.batch_specs(count):
        cfg = scenegen.scaled_config(d, n)
        sc = scenegen.make_scene(cfg, s, query_id=s)
        key = scenegen.calib_key(cfg, s)
        if key not in calib:
            return {"skipped": f"no stored beta for {key}: run python -m oracle.calibrate --batch {count}"}
        sc.extra["beta"] = calib[key]["beta"]
        scenes.append(sc)
    out = {"workload": f"{count} queries, one roadmap each: dimension uniform over 2D/3D/6D, n log-uniform in "
                       f"[1000, 32000] (2D: [1000, 4000]), per-query obstacles and grids, beta = stored 60th "
                       f"percentile, MC rollouts 1024 (2D/3D) / 4096 (6D)"}

    def run_group(name, idx, front_cap, tune, timed_reps, plain):
        grp = [scenes[i] for i in idx]
        specs = [mp.scene_spec(sc) for sc in grp]
        queries = [mp.make_query(sc.extra["beta"], scenegen.LAMBDA, own_share=True) for sc in grp]
        mcs = [(sc.cfg.mc_rollouts, sc.mc_seed, 0, sc.delta_fx, sc.sigma_fx, sc.shift) for sc in grp]
        total = sum(sc.cfg.n + 2 for sc in grp)
        t0 = time.perf_counter()
        log(f"mixed {name}: {len(grp)} queries, {total} nodes")
        ws = mp.Workspace(total, front_cap=front_cap, max_plans=1 << 29)
        tuning = None
        if tune:
            tb, build_ms, rms = mp.autotune_build(specs, reps=1)
            ts, search_ms = mp.autotune_search(ws, rms, queries, reps=1)
            tuning = {"build": tb, "build_ms": build_ms, "search": ts, "search_ms": search_ms,
                      "autotune_s": round(time.perf_counter() - t0, 2)}
            log(f"mixed {name}: autotuned in {tuning['autotune_s']} s")
        else:
            rms = mp.build_roadmaps(specs)
        holder = {"rms": rms}

        def step():
            holder["rms"] = mp.build_roadmaps(specs, rms=holder["rms"])
            r = holder["rms"]
            res = mp.search_batch(ws, r, queries, check=False)
            ok = [i for i in range(len(grp)) if res[i].status == 0]
            if ok:
                mp.certify_batch([r[i] for i in ok], [res[i].path for i in ok], [mcs[i] for i in ok])
            return res
        for _ in range(1 if timed_reps > 1 else 0):
            step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        exps = 0
        for _ in range(timed_reps):
            res = step()
            exps += sum(r.expansions for r in res)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / timed_reps
        log(f"mixed {name}: {ms:.1f} ms per step")
        by_dim = {}
        for sc, r in zip(grp, res):
            d = by_dim.setdefault(f"{sc.cfg.dim_kind}d", {})
            d[str(r.status)] = d.get(str(r.status), 0) + 1
        g = {"queries": len(grp), "nodes": total, "ms_per_step": ms, "ms_per_query": ms / len(grp),
             "expansions_per_s": exps / timed_reps / (ms / 1e3),
             "status": {str(k): int(v) for k, v in zip(*np.unique([r.status for r in res], return_counts=True))},
             "status_by_dim": by_dim,
             "max_wavefronts": max(r.wavefronts for r in res), "front_cap": front_cap, "tuning": tuning}
        mf, pu = ws.stats()
        g["max_front"], g["pool_entries_used"], g["pool_entries"] = mf, pu, total * front_cap
        g["plans"] = int(sum(r.plans for r in res))
        if plain:
            # the same set of queries both ways: those that finished in the batch
            done = [i for i, r in enumerate(res) if r.status in (0, 1)]
            sub_rms = [holder["rms"][i] for i in done]
            sub_q = [queries[i] for i in done]
            e0.record(stream)
            mp.search_batch(ws, sub_rms, sub_q, check=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_b = e0.elapsed_time(e1)
            vmax = max(grp[i].cfg.n + 2 for i in done)
            ws1 = mp.Workspace(vmax, front_cap=min(16384, ((1 << 32) - 16) // vmax), max_plans=1 << 27)
            e0.record(stream)
            for rm, q in zip(sub_rms, sub_q):
                try:
                    mp.search(ws1, rm, q.beta, lam=scenegen.LAMBDA)
                except mp.MpapError:
                    pass            # the status is the batched one's (same fronts, same result)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_p = e0.elapsed_time(e1)
            del ws1
            g["search_only"] = {"queries": len(done), "batched_ms_per_query": ms_b / len(done),
                                "plain_ms_per_query": ms_p / len(done), "speedup": ms_p / ms_b}
        return g

    g = run_group("all", list(range(count)), 2048, True, 2, True)
    out.update(g)
    return out


# ------------------------------------------------------------------ surrogate
SUR_N, SUR_EPS, SUR_TAU, SUR_BATCH = 32000, 0.05, 0.1, 64
# algorithmic FLOPs per sample of one training step: forward 2 (48*128 + 2*128^2 +
# 128*2), weight gradients the same, input gradients of layers 2..4 2 (2*128^2 + 128*2)
MLP_TRAIN_FLOP = 2 * (48 * 128 + 2 * 128 * 128 + 128 * 2) * 2 + 2 * (2 * 128 * 128 + 128 * 2)


def _sur_batch(mp, S, ws, cfg, seeds, call_base, rollouts=None):
    scs = [scenegen.make_scene(cfg, s, query_id=s) for s in seeds]
    rms = mp.build_roadmaps([mp.scene_spec(sc) for sc in scs])
    res = mp.search_batch(ws, rms, [mp.make_query(1 << 62, scenegen.LAMBDA, goal_stop=False) for _ in scs])
    cands = S.collect_candidates(ws, res, 64)
    mcs = [(rollouts or cfg.mc_rollouts, sc.mc_seed, 0, sc.delta_fx, sc.sigma_fx, sc.shift) for sc in scs]
    return rms, res, cands, mcs


def surrogate_report(args, stream):
    """Batched search + learned screen versus the plain GPU search on the same 64
    queries (6D, 32000 samples, 64 candidate goal plans each, 4096-rollout Monte
    Carlo as judge), at one certified failure bound.  The network is first trained
    on the GPU on Monte Carlo-labelled candidates of separate training queries."""
    import torch
    import paper_1705_02408_gb300 as mp
    from paper_1705_02408_gb300 import surrogate as S
    cfg = scenegen.surrogate_config(SUR_N)
    ws = mp.Workspace(SUR_BATCH * (SUR_N + 2), front_cap=128, max_plans=1 << 25)
    # training set: candidates of seeds 100001.. until enough plans
    t0 = time.perf_counter()
    X, Y, q = [], [], 0
    while sum(len(x) for x in X) < args.sur_train_plans:
        seeds = range(100001 + q, 100001 + q + SUR_BATCH)
        rms, res, cands, mcs = _sur_batch(mp, S, ws, cfg, seeds, 10000)
        for f, r in zip(S.candidate_features(rms, cands), S.mc_rates(rms, cands, mcs, call_base=10000)):
            X.append(f); Y.append(r[:, :2])
        q += SUR_BATCH
    X, Y = np.concatenate(X)[:args.sur_train_plans], np.concatenate(Y)[:args.sur_train_plans]
    gen_s = time.perf_counter() - t0
    net = mp.Mlp(seed=3, max_batch=4096)
    S.train(net, X, Y, steps=20, batch=4096, lr=2e-3, seed=1)        # warm-up
    net = mp.Mlp(seed=3, max_batch=4096)
    mp.profile_reset(); mp.profile_enable(True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    losses = S.train(net, X, Y, steps=args.sur_train_steps, batch=4096, lr=2e-3, seed=1)
    e1.record(stream)
    torch.cuda.synchronize()
    mp.profile_enable(False)
    kern = mp.profile_read()
    train_ms = e0.elapsed_time(e1)
    gl, gms = kern.get("k_gemm_tc", (0, 0.0))
    flop = MLP_TRAIN_FLOP * 4096.0 * args.sur_train_steps
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = peaks.get("bf16_tflops", 1900.0)
    train = {"plans": int(len(X)), "queries": q, "label_rollouts": cfg.mc_rollouts,
             "generate_s": round(gen_s, 2), "steps": args.sur_train_steps, "batch": 4096,
             "loss_first": float(losses[0]), "loss_last50": float(np.mean(losses[-50:])),
             "ms_per_step": train_ms / args.sur_train_steps,
             "samples_per_s": 4096.0 * args.sur_train_steps / (train_ms / 1e3),
             "kernel_ms_per_step": {k: round(v[1] / args.sur_train_steps, 4) for k, v in sorted(kern.items())},
             "roofline": {"kernel": "k_gemm_tc", "bound": "tensor",
                          "achieved": flop / (gms / 1e3) / 1e12 if gms else None,
                          "peak": peak, "unit": "TFLOP/s",
                          "frac": (flop / (gms / 1e3) / 1e12) / peak if gms else None,
                          "launches": int(gl), "traffic": None,
                          "note": "algorithmic bf16 FLOPs of the 11 products of a step over the tensor-core "
                                  "kernel's time; 128-wide layers leave it latency-bound",
                          "peak_source": "MEASURED_PEAKS.json bf16_tflops (measured)" if peaks else "fallback"}}
    # evaluation on 64 held-out queries at one certified failure bound, wall
    # time from the search to the certified plan of every query:
    #   plain_gpu  one mpap_search per query, then its candidates certified in
    #              solution order one Monte Carlo call at a time
    #   batched    one batched search, candidates certified in solution order
    #              in lock-step batched rounds (mpap_surrogate_screen, no network)
    #   screened   the same with the network's screened order
    ev = {}
    seeds = range(1, 1 + SUR_BATCH)
    rms, res, cands, mcs = _sur_batch(mp, S, ws, cfg, seeds, 0)
    qs = [mp.make_query(1 << 62, scenegen.LAMBDA, goal_stop=False) for _ in rms]
    ws1 = mp.Workspace(SUR_N + 2, front_cap=128, max_plans=1 << 22)
    sel = {}
    for mode in ("plain_gpu", "batched", "screened") * 2:      # second pass is the timed one
        torch.cuda.synchronize()
        t = time.perf_counter()
        if mode == "plain_gpu":
            cq = []
            for rm, q in zip(rms, qs):
                r = mp.search(ws1, rm, q.beta, lam=scenegen.LAMBDA, goal_stop=False)
                cq.append(mp.search_candidates(ws1, 0, cap=64) if r.status == 0 else None)
            t1 = t2 = time.perf_counter()
            chosen = np.full(len(rms), -1, np.int64)
            calls = np.zeros(len(rms), np.int64)
            for i, c in enumerate(cq):
                for j, path in enumerate(c["paths"] if c else []):
                    ro, seed, base, d, sig, sh = mcs[i]
                    ct = mp.certify(rms[i], path, ro, seed, base + j, d, sig, sh)
                    calls[i] += 1
                    if ct["hits_any"] <= SUR_EPS * ct["rollouts"]:
                        chosen[i] = j
                        break
            out = S.Selection(chosen, calls, int(calls.max()) if len(calls) else 0)
        else:
            res = mp.search_batch(ws, rms, qs)
            cq = S.collect_candidates(ws, res, 64)
            t1 = time.perf_counter()
            out = S.screen(net, rms, cq, mcs, SUR_EPS, SUR_TAU, use_net=(mode == "screened"))
            t2 = t1
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        dt = t3 - t
        sel[mode] = out
        cands = cq
        ev[mode] = {"ms_per_batch": dt * 1e3, "ms_per_query": dt * 1e3 / len(rms),
                    "phase_ms": {"search_and_candidates": (t1 - t) * 1e3, "certify": (t3 - t2) * 1e3},
                    "mc_calls": int(out.mc_calls.sum()), "mc_rounds": out.rounds,
                    "mc_rollouts": int(out.mc_calls.sum()) * cfg.mc_rollouts,
                    "solved": int((out.chosen >= 0).sum())}
    a, b = sel["plain_gpu"], sel["screened"]
    assert np.array_equal(a.chosen >= 0, b.chosen >= 0)
    ratios = [cands[i]["cost"][b.chosen[i]] / cands[i]["cost"][a.chosen[i]]
              for i in range(len(rms)) if a.chosen[i] >= 0]
    return {"workload": f"6D double integrator, {SUR_N} samples, 30 boxes, 32^3 grid, twice the 6D MC noise, "
                        f"beta unbounded, exhaustive search (no goal stop), 64 candidates/query, "
                        f"{cfg.mc_rollouts}-rollout MC judge",
            "queries": len(rms), "certified_failure_bound": SUR_EPS, "screen_threshold": SUR_TAU,
            "plain_gpu": ev["plain_gpu"], "batched": ev["batched"], "screened": ev["screened"],
            "mc_calls_ratio": ev["screened"]["mc_calls"] / max(1, ev["plain_gpu"]["mc_calls"]),
            "speedup_vs_plain_gpu": ev["plain_gpu"]["ms_per_batch"] / ev["screened"]["ms_per_batch"],
            "speedup_vs_batched": ev["batched"]["ms_per_batch"] / ev["screened"]["ms_per_batch"],
            "cost_ratio_mean": float(np.mean(ratios)) if ratios else None,
            "cost_ratio_max": float(np.max(ratios)) if ratios else None,
            "train": train}


# ------------------------------------------------------------------ CPU oracle
def oracle_query(sc):
    import oracle
    cfg = sc.cfg
    rm = oracle.build_roadmap(sc)
    beta = sc.extra.get("beta")
    if beta is None:
        beta = oracle.beta_percentile(rm)
    res = oracle.explore(rm, beta, oracle.group_width(scenegen.LAMBDA, cfg.r))
    if res.status == 0:
        oracle.certify(rm, res.path, cfg.mc_rollouts, sc.mc_seed, 0, sc.delta_fx, sc.sigma_fx, sc.shift)
    return res.expansions


def host_cpu():
    """(logical cores, CPU model) of the machine the oracle runs on."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return os.cpu_count() or 1, model or "unknown"


def cpu_baseline(scenes, threaded_scenes):
    """The oracle as it stands on the host cores: one thread over two queries,
    then one query per thread over all cores (the oracle's calls release the
    interpreter lock, so the threads run in parallel)."""
    import concurrent.futures as cf
    import oracle
    oracle.build()
    ncores, model = host_cpu()
    t0 = time.perf_counter()
    exps = sum(oracle_query(s) for s in scenes)
    dt = time.perf_counter() - t0
    out = {"value": exps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{len(scenes)} of the benchmark's 6D-16k queries (roadmap + search + 4096-rollout MC), "
                     f"single thread, {dt:.1f} s", "ms_per_query": dt * 1e3 / len(scenes),
           "host_cores": ncores, "cpu_model": model}
    nt = min(ncores, len(threaded_scenes))
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=nt) as ex:
        texps = sum(ex.map(oracle_query, threaded_scenes[:nt]))
    tdt = time.perf_counter() - t0
    out["threaded"] = {"value": texps / tdt, "unit": UNIT, "cores": nt, "queries": nt,
                       "sample": f"{nt} queries, one per thread on {nt} threads, {tdt:.1f} s wall",
                       "ms_per_query": tdt * 1e3 / nt}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle
    oracle.build()
    scenes = scenes_for_rank(0, args.steps + args.warmup)
    for s in scenes[:args.warmup]:
        oracle_query(s)
    t0 = time.perf_counter()
    exps = sum(oracle_query(s) for s in scenes[args.warmup:])
    dt = time.perf_counter() - t0
    value = exps / dt
    ms = dt * 1e3 / args.steps
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "queries_per_step": 1,
                       "note": "CPU oracle, one query per step (bounded sample)"},
            "ms_per_query": ms,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} timed 6D-16k queries, one per step",
                             "host_cores": host_cpu()[0], "cpu_model": host_cpu()[1]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_gpu(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
