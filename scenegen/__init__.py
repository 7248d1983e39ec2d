"""Seeded synthetic inputs for the MPAP hot path.

This module only *draws inputs*: axis-aligned box obstacles, a perception-quality
grid, start and goal states, the Monte Carlo noise tables and the query bounds.
It holds none of the planning arithmetic (no sampling of roadmap nodes, no edge
costs, no heuristic stepping, no search), so it can feed both the CPU oracle and
the CUDA library without coupling them.

Workload shapes follow the paper's numerical experiments (Sec. 4: AABB obstacles,
a perception quality field standing in for visible-feature counts with n_f = 12,
group factor lambda = 0.5) and the five configurations this project measures:

* ``2d``   unit square, 8 boxes (sides U[0.05, 0.2]), n = 1000, r = 0.08, 64^2 grid
* ``3d``   unit cube, 20 boxes, n = 8000, r = 0.12, 32^3 grid, MC with 1024 rollouts
* ``6d``   6D double integrator (|v| <= 1), 30 boxes, n = 16000, T = 0.25,
           16 sub-steps per edge (15 interior collision checkpoints), 32^3 grid,
           MC with 4096 rollouts
* ``batch`` 256 queries, n log-uniform in [1k, 32k], dimension uniform over
           {2d, 3d, 6d}, each with its own obstacles and grid
* the 6D surrogate configuration (n = 32000) is ``6d`` with ``n`` overridden.

Everything is deterministic in ``seed`` (numpy's PCG64 via ``default_rng``).
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field, replace

import numpy as np

# Heuristic constants (Sec. 4.1): n_f features offset the drift; K = 2 n_f quality
# levels so that the mean level of the normalised field sits at n_f.
N_F = 12
K_LEVELS = 24
M_STEPS = 16          # sub-steps per edge: 15 interior checkpoints + endpoint
LAMBDA = 0.5          # group cost factor used throughout the paper's experiments
GOAL_RADIUS = 0.05
FIXED_SHIFT = 20      # Monte Carlo positions are integers in units of 2^-20

DIM_2D, DIM_3D, DIM_DI6 = 2, 3, 6

_CALIB_PATH = os.path.join(os.path.dirname(__file__), "calibration.json")


@dataclass
class Config:
    name: str
    dim_kind: int            # 2, 3 or 6 (6 = 3D double integrator)
    n: int                   # free samples (V = n + 2 with x_init = 0, x_goal = 1)
    nb: int                  # obstacle boxes
    r: float                 # r_n-disc radius in cost units
    grid_G: int              # quality cells per axis
    T_edge: float = 0.25     # edge duration for the double integrator
    M: int = M_STEPS
    side_lo: float = 0.05
    side_hi: float = 0.2
    mc_rollouts: int = 1024
    # Monte Carlo model (integer error walk): per-step noise scale sigma in units of
    # 2^-20 at the worst and best quality level, and the localisation bound delta.
    sigma_max: float = 0.0016
    sigma_min: float = 0.0002
    delta_loc: float = 0.05
    beta_pct: float = 60.0   # beta = this percentile of straight-line heuristics


CONFIGS = {
    "2d": Config("2d", DIM_2D, 1000, 8, 0.08, 64, mc_rollouts=1024),
    "3d": Config("3d", DIM_3D, 8000, 20, 0.12, 32, mc_rollouts=1024),
    # r for the double integrator is calibrated once for a mean out-degree near 48
    # (see oracle/calibrate.py) and frozen here.
    "6d": Config("6d", DIM_DI6, 16000, 30, 12.0, 32, mc_rollouts=4096,
                 sigma_max=0.0012, sigma_min=0.00015),
}


def config(name: str, **overrides) -> Config:
    cfg = CONFIGS[name]
    return replace(cfg, **overrides) if overrides else cfg


def pos_dims(dim_kind: int) -> int:
    return 2 if dim_kind == DIM_2D else 3


@dataclass
class Scene:
    cfg: Config
    seed: int
    query_id: int
    box_lo: np.ndarray       # float32 [nb, 3] (z spans [0, 1] in 2D and is ignored)
    box_hi: np.ndarray
    grid: np.ndarray         # uint8 [G^Dp], x fastest
    x_init: np.ndarray       # float32 [6]
    x_goal: np.ndarray       # float32 [6]
    sample_seed: int         # 64-bit key for the counter-based node sampler
    mc_seed: int             # 64-bit key for the Monte Carlo rollouts
    sigma_fx: np.ndarray     # int32 [K+1]
    shift: np.ndarray        # int32 [K+1]
    delta_fx: int
    extra: dict = field(default_factory=dict)

    @property
    def dim_kind(self) -> int:
        return self.cfg.dim_kind

    @property
    def n(self) -> int:
        return self.cfg.n


def _value_noise(rng: np.random.Generator, G: int, dp: int, lattice: int = 8) -> np.ndarray:
    """Smooth value noise in [0, 1] at the G^dp cell centres (x fastest)."""
    vals = rng.random((lattice,) * dp)
    c = (np.arange(G, dtype=np.float64) + 0.5) / G * (lattice - 1)
    i0 = np.minimum(np.floor(c).astype(np.int64), lattice - 2)
    f = c - i0
    w = f * f * (3.0 - 2.0 * f)
    if dp == 2:
        # axes: [y, x]
        y0, x0 = np.meshgrid(i0, i0, indexing="ij")
        wy, wx = np.meshgrid(w, w, indexing="ij")
        v00 = vals[y0, x0]; v01 = vals[y0, x0 + 1]
        v10 = vals[y0 + 1, x0]; v11 = vals[y0 + 1, x0 + 1]
        a = v00 * (1 - wx) + v01 * wx
        b = v10 * (1 - wx) + v11 * wx
        q = a * (1 - wy) + b * wy
    else:
        z0, y0, x0 = np.meshgrid(i0, i0, i0, indexing="ij")
        wz, wy, wx = np.meshgrid(w, w, w, indexing="ij")
        def lerp_x(zz, yy):
            return vals[zz, yy, x0] * (1 - wx) + vals[zz, yy, x0 + 1] * wx
        a = lerp_x(z0, y0) * (1 - wy) + lerp_x(z0, y0 + 1) * wy
        b = lerp_x(z0 + 1, y0) * (1 - wy) + lerp_x(z0 + 1, y0 + 1) * wy
        q = a * (1 - wz) + b * wz
    q = (q - q.min()) / max(q.max() - q.min(), 1e-12)
    return q


def quality_levels(q: np.ndarray, K: int = K_LEVELS) -> np.ndarray:
    return np.minimum(K, np.floor(q * (K + 1))).astype(np.uint8)


def _box_hits_ball(lo, hi, c, rad) -> bool:
    d = np.maximum(0.0, np.maximum(lo - c, c - hi))
    return float(np.sum(d * d)) <= rad * rad


def mc_tables(cfg: Config):
    """Per-level noise scale and relocalisation shift for the Monte Carlo model.

    sigma_k falls linearly with quality from sigma_max (level 0) to sigma_min
    (level K).  Levels at or above n_f relocalise: the error contracts by a factor
    (1 - 2^-s_k) per step, with s_k shrinking (stronger contraction) as quality
    rises; s_k = 0 means no contraction.
    """
    K = K_LEVELS
    scale = float(1 << FIXED_SHIFT)
    k = np.arange(K + 1, dtype=np.float64)
    sigma = cfg.sigma_min + (cfg.sigma_max - cfg.sigma_min) * (1.0 - k / K)
    sigma_fx = np.rint(sigma * scale).astype(np.int32)
    shift = np.zeros(K + 1, dtype=np.int32)
    for kk in range(N_F, K + 1):
        shift[kk] = max(1, 6 - (kk - N_F) // 2)
    delta_fx = int(round(cfg.delta_loc * scale))
    return sigma_fx, shift, delta_fx


def make_scene(name_or_cfg, seed: int, query_id: int = 0, **overrides) -> Scene:
    cfg = name_or_cfg if isinstance(name_or_cfg, Config) else config(name_or_cfg, **overrides)
    dp = pos_dims(cfg.dim_kind)
    rng = np.random.default_rng([int(seed), int(cfg.dim_kind), 0x4D504150])
    start = np.full(3, 0.05); goal = np.full(3, 0.95)
    if dp == 2:
        start[2] = goal[2] = 0.0
    lo = np.zeros((cfg.nb, 3)); hi = np.zeros((cfg.nb, 3))
    keep = 0
    while keep < cfg.nb:
        c = rng.random(dp)
        s = rng.uniform(cfg.side_lo, cfg.side_hi, dp)
        blo = np.clip(c - s / 2, 0.0, 1.0); bhi = np.clip(c + s / 2, 0.0, 1.0)
        if (_box_hits_ball(blo, bhi, start[:dp], GOAL_RADIUS + 0.02)
                or _box_hits_ball(blo, bhi, goal[:dp], GOAL_RADIUS + 0.02)):
            continue
        lo[keep, :dp] = blo; hi[keep, :dp] = bhi
        if dp == 2:
            lo[keep, 2] = 0.0; hi[keep, 2] = 1.0
        keep += 1
    grid = quality_levels(_value_noise(rng, cfg.grid_G, dp))
    x_init = np.zeros(6, np.float32); x_goal = np.zeros(6, np.float32)
    x_init[:3] = start; x_goal[:3] = goal
    sample_seed = int(rng.integers(0, 2**63 - 1))
    mc_seed = int(rng.integers(0, 2**63 - 1))
    sigma_fx, shift, delta_fx = mc_tables(cfg)
    return Scene(cfg=cfg, seed=int(seed), query_id=int(query_id),
                 box_lo=lo.astype(np.float32), box_hi=hi.astype(np.float32),
                 grid=grid.reshape(-1).copy(), x_init=x_init, x_goal=x_goal,
                 sample_seed=sample_seed, mc_seed=mc_seed,
                 sigma_fx=sigma_fx, shift=shift, delta_fx=delta_fx)


FEATURE_OFFSET = 0.004   # features sit this far off the surface they mark


def feature_points(scene: Scene, count: int = 256) -> np.ndarray:
    """Mapped visual features for the visible-feature perception levels: ``count``
    points, float32 [count, 3] (z = 0 in 2D), drawn alternately on the faces of
    the scene's boxes and on the walls of the unit square/cube, each moved
    FEATURE_OFFSET off its surface into free space (outward from a box, inward
    from a wall); a point inside or on another box is drawn again.
    Deterministic in the scene's seed."""
    dp = pos_dims(scene.cfg.dim_kind)
    rng = np.random.default_rng([int(scene.seed), int(scene.cfg.dim_kind), 0x46454154])
    nb = len(scene.box_lo)
    blo = scene.box_lo.astype(np.float64)[:, :dp]
    bhi = scene.box_hi.astype(np.float64)[:, :dp]
    out = np.zeros((count, 3))
    k = 0
    for attempt in range(64 * count + 64):
        if k == count:
            break
        on_box = nb > 0 and attempt % 2 == 0
        axis = int(rng.integers(0, dp))
        side = int(rng.integers(0, 2))
        u = rng.random(3)
        if on_box:
            b = int(rng.integers(0, nb))
            lo, hi = scene.box_lo[b].astype(np.float64), scene.box_hi[b].astype(np.float64)
            p = lo + u * (hi - lo)
            p[axis] = (hi[axis] + FEATURE_OFFSET) if side else (lo[axis] - FEATURE_OFFSET)
        else:
            p = u.copy()
            p[axis] = (1.0 - FEATURE_OFFSET) if side else FEATURE_OFFSET
        p = np.clip(p, 0.0, 1.0)
        if dp == 2:
            p[2] = 0.0
        if nb and ((p[None, :dp] >= blo) & (p[None, :dp] <= bhi)).all(1).any():
            continue           # inside (or on) another box: draw again
        out[k] = p
        k += 1
    return out[:k].astype(np.float32)


def yaw_headings(bins: int) -> np.ndarray:
    """Unit camera headings (cos, sin) of ``bins`` evenly spaced yaw angles
    2 pi b / bins, float32 [bins, 2] (rounded once from double)."""
    a = 2.0 * np.pi * np.arange(bins) / bins
    return np.stack([np.cos(a), np.sin(a)], 1).astype(np.float32)


def scaled_config(dim_kind: int, n: int) -> Config:
    """A configuration of dimension ``dim_kind`` resized to ``n`` samples with the
    connection radius rescaled so that the mean out-degree stays near that of the
    reference configuration (r ~ n^(-1/d); for the double integrator the energy
    budget r - T shrinks like n^(-1/3))."""
    base = {DIM_2D: CONFIGS["2d"], DIM_3D: CONFIGS["3d"], DIM_DI6: CONFIGS["6d"]}[dim_kind]
    ratio = base.n / float(n)
    if dim_kind == DIM_2D:
        r = base.r * ratio ** 0.5
    elif dim_kind == DIM_3D:
        r = base.r * ratio ** (1.0 / 3.0)
    else:
        r = base.T_edge + (base.r - base.T_edge) * ratio ** (1.0 / 3.0)
    return replace(base, name=f"{base.name}_n{n}", n=int(n), r=float(np.float32(r)))


def surrogate_config(n: int = 32000) -> Config:
    """Workload of the certification surrogate: the double integrator resized to
    n samples (radius as scaled_config) with twice the 6D Monte Carlo noise, so
    that the cheapest goal plan often fails a 5% bound and the screen has
    alternatives to choose among; 4096 rollouts."""
    base = scaled_config(DIM_DI6, n)
    return replace(base, name=f"6d_sur_n{n}", sigma_max=2 * CONFIGS["6d"].sigma_max,
                   sigma_min=2 * CONFIGS["6d"].sigma_min, mc_rollouts=4096)


def batch_specs(count: int = 256, seed: int = 7, n_lo: int = 1000, n_hi: int = 32000, n_hi_2d: int = 4000):
    """(dim_kind, n, scene_seed) for the batched workload: dimension uniform over
    {2d, 3d, 6d}, n log-uniform in [n_lo, n_hi] ([n_lo, min(n_hi, n_hi_2d)] for
    2D, whose Pareto fronts grow without bound with n: the 2D heuristic gains are
    continuous in edge length, so almost every path has its own h)."""
    rng = np.random.default_rng([int(seed), 0xBA7C4])
    dims = rng.choice([DIM_2D, DIM_3D, DIM_DI6], size=count)
    u = rng.uniform(0.0, 1.0, size=count)
    seeds = rng.integers(1, 2**31 - 1, size=count)
    out = []
    for d, uu, s in zip(dims, u, seeds):
        hi = min(n_hi, n_hi_2d) if d == DIM_2D else n_hi
        hi = max(hi, n_lo)
        n = int(math.exp(math.log(n_lo) + uu * (math.log(hi) - math.log(n_lo))))
        out.append((int(d), n, int(s)))
    return out


def load_calibration() -> dict:
    """Stored perception bounds beta (h units) per scene, written by
    oracle/calibrate.py from the oracle's straight-line heuristic percentile."""
    if not os.path.exists(_CALIB_PATH):
        return {}
    with open(_CALIB_PATH) as f:
        return json.load(f)


def calib_key(cfg: Config, seed: int) -> str:
    return f"{cfg.name}:{cfg.dim_kind}:{cfg.n}:{seed}"


# ---------------------------------------------------------------------------
# Synthetic observations for the learned error-rate heuristic.  The paper fits
# its network to error rates of a real visual-inertial estimator measured
# against motion capture; that data is not available, so observations come from
# an invented sensor model: the rate r of the position-error magnitude is
# Gaussian with mean 0.02 (1 + 0.5 |v| + 0.3 |w|) (1 - n / 12) (negative when
# more than 12 features are visible: the estimate relocalises) and standard
# deviation 0.004 (1 + |v|) + 0.002 |w|, for speed |v| <= 1, angular rate
# |w| <= 2 and n = 0 .. 24 visible features.
# ---------------------------------------------------------------------------
def vio_samples(n: int, seed: int):
    """(X [n, 7] float32 = (v, w, n_visible), r [n] float32) drawn from the model above."""
    rng = np.random.default_rng([int(seed), 0x710])
    d = rng.normal(0.0, 1.0, (n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    v = d * rng.uniform(0.0, 1.0, (n, 1))
    a = rng.normal(0.0, 1.0, (n, 3))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    w = a * rng.uniform(0.0, 2.0, (n, 1))
    nv = rng.integers(0, 25, (n, 1)).astype(np.float64)
    sv, sw = np.linalg.norm(v, axis=1), np.linalg.norm(w, axis=1)
    mean = 0.02 * (1 + 0.5 * sv + 0.3 * sw) * (1 - nv[:, 0] / 12.0)
    std = 0.004 * (1 + sv) + 0.002 * sw
    r = mean + std * rng.normal(0.0, 1.0, n)
    return np.concatenate([v, w, nv], 1).astype(np.float32), r.astype(np.float32)


def mapped_states(n: int, seed: int):
    """[n, 7] float32 mapped states (position in the unit cube, velocity in the
    unit ball, yaw in [-pi, pi)) for the heuristic map."""
    rng = np.random.default_rng([int(seed), 0x3A9])
    p = rng.uniform(0.0, 1.0, (n, 3))
    d = rng.normal(0.0, 1.0, (n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    v = d * rng.uniform(0.0, 1.0, (n, 1)) ** (1.0 / 3.0)
    y = rng.uniform(-np.pi, np.pi, (n, 1))
    return np.concatenate([p, v, y], 1).astype(np.float32)
