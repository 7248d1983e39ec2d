"""Writes scenegen/calibration.json: the perception bound beta of every benchmark
scene, computed by the oracle only (nearest-rank 60th percentile of the
straight-line heuristic from x_init to every roadmap node), plus the mean
out-degree that fixed the double-integrator radius r.

Usage: python -m oracle.calibrate [--procs 8] [--seeds 64] [--batch 256]

--batch N adds the first N queries of the mixed batched workload
(scenegen.batch_specs: dimension and size drawn per query).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mpr
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _one(job):
    import numpy as np
    import oracle
    import scenegen
    name, seed, n = job
    cfg = scenegen.config(name) if n is None else scenegen.scaled_config(
        {"2d": 2, "3d": 3, "6d": 6}[name], n)
    if n is not None:
        seed = int(seed)
    sc = scenegen.make_scene(cfg, seed, query_id=seed)
    rm = oracle.build_roadmap(sc)
    g = rm.graph()
    beta = oracle.beta_percentile(rm, cfg.beta_pct)
    return scenegen.calib_key(cfg, seed), dict(beta=int(beta), V=int(g.V), E=int(g.dst.size),
                                               mean_degree=float(np.diff(g.row_ptr).mean()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 4)
    ap.add_argument("--seeds", type=int, default=64)
    ap.add_argument("--batch", type=int, default=0)
    args = ap.parse_args()
    import scenegen
    jobs = [("6d", s, None) for s in range(1, args.seeds + 1)]
    names = {2: "2d", 3: "3d", 6: "6d"}
    # largest first, so the pool is not left waiting on one big roadmap
    batch = sorted(scenegen.batch_specs(args.batch), key=lambda t: -t[1]) if args.batch else []
    jobs += [(names[d], s, n) for d, n, s in batch]
    t0 = time.time()
    ctx = mpr.get_context("spawn")
    with ctx.Pool(args.procs) as pool:
        out = dict(pool.map(_one, jobs))
    data = out          # the file holds exactly the scenes of this run
    path = os.path.join(ROOT, "scenegen", "calibration.json")
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    degs = [v["mean_degree"] for v in out.values()]
    print(f"wrote {len(out)} entries in {time.time() - t0:.0f}s; mean degree {sum(degs) / len(degs):.1f}")


if __name__ == "__main__":
    main()
