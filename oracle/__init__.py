"""CPU oracle for the MPAP hot path -- TEST INFRASTRUCTURE ONLY.

Python (ctypes) access to ``mpap_oracle.cpp``: a plain, single-threaded C++
restatement of the paper's Alg. 2 (BuildGraph), the grid form of the Sec. 4.1
perception heuristic, Alg. 3 (Explore, with RemoveDominated) and the Monte Carlo
certifier.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with the
CUDA library ``paper_1705_02408_gb300``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpap_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

INT64_MAX = (1 << 63) - 1


def build(force: bool = False) -> str:
    """Compile the oracle (g++, -O2, no floating-point contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", "-o", tmp, _SRC]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_build_roadmap.restype = P
        L.orc_build_roadmap.argtypes = [C.c_int, C.c_int, f32p, f32p, C.c_int, u8p, C.c_int,
                                        C.c_int, C.c_uint32, C.c_uint64, C.c_uint32, C.c_float,
                                        C.c_float, C.c_int, f32p, f32p, C.c_float]
        L.orc_build_roadmap_from_points.restype = P
        L.orc_build_roadmap_from_points.argtypes = [C.c_int, C.c_int, f32p, f32p, C.c_int, u8p,
                                                    C.c_int, C.c_int, C.c_uint32, f32p,
                                                    C.c_float, C.c_float, C.c_int, C.c_float]
        L.orc_build_roadmap_heading.restype = P
        L.orc_build_roadmap_heading.argtypes = [C.c_int, C.c_int, f32p, f32p, C.c_int, u8p, C.c_int,
                                                C.c_int, C.c_uint32, C.c_uint64, C.c_uint32, C.c_float,
                                                C.c_float, C.c_int, f32p, f32p, C.c_float, C.c_int, u8p]
        L.orc_build_roadmap_from_points_heading.restype = P
        L.orc_build_roadmap_from_points_heading.argtypes = [C.c_int, C.c_int, f32p, f32p, C.c_int, u8p,
                                                            C.c_int, C.c_int, C.c_uint32, f32p, C.c_float,
                                                            C.c_float, C.c_int, C.c_float, C.c_int, u8p,
                                                            C.c_void_p]
        L.orc_roadmap_yaw.argtypes = [P, f32p]
        L.orc_roadmap_from_csr.restype = P
        L.orc_roadmap_from_csr.argtypes = [C.c_uint32, u32p, u32p, i32p, i32p, i32p, u8p]
        L.orc_roadmap_free.argtypes = [P]
        L.orc_roadmap_V.restype = C.c_uint32
        L.orc_roadmap_V.argtypes = [P]
        L.orc_roadmap_E.restype = C.c_uint32
        L.orc_roadmap_E.argtypes = [P]
        L.orc_roadmap_get.argtypes = [P, f32p, u8p, u32p, u32p, i32p, i32p, i32p]
        L.orc_edge_eval.restype = C.c_int
        L.orc_edge_eval.argtypes = [P, C.c_uint32, C.c_uint32, f32p, f32p, f32p, i64p, f32p, f32p]
        L.orc_segment_hits_box.restype = C.c_int
        L.orc_segment_hits_box.argtypes = [C.c_int, f32p, f32p, f32p, f32p]
        L.orc_feature_levels.restype = None
        L.orc_feature_levels.argtypes = [C.c_int, C.c_int, f32p, f32p, C.c_int, f32p, C.c_int, C.c_int, f32p,
                                         C.c_float, C.c_float, C.c_int, u8p]
        L.orc_explore.restype = P
        L.orc_explore.argtypes = [P, C.c_int64, C.c_int64, C.c_uint32, C.c_int, C.c_uint64, C.c_int]
        L.orc_roadmap_from_csr_peaks.restype = P
        L.orc_roadmap_from_csr_peaks.argtypes = [C.c_uint32, u32p, u32p, i32p, i32p, i32p, i32p, i32p, u8p]
        L.orc_roadmap_get_peaks.argtypes = [P, i32p, i32p]
        L.orc_result_free.argtypes = [P]
        L.orc_result_summary.argtypes = [P] + [C.c_void_p] * 8
        L.orc_result_get.argtypes = [P, u32p, u32p, i64p, i64p]
        L.orc_certify.restype = C.c_int
        L.orc_certify.argtypes = [P, u32p, C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint32,
                                  C.c_int64, i32p, i32p, u32p]
        L.orc_straight_line_h.argtypes = [P, i64p]
        L.orc_certify_vio.restype = C.c_int
        L.orc_certify_vio.argtypes = [P, u32p, C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint32, C.c_int64,
                                      C.c_int32, C.c_int32, C.c_int32, i32p, u32p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]
        L.orc_result_candidates.restype = C.c_int
        L.orc_result_candidates.argtypes = [P, C.c_uint32, i64p, i64p, u32p, u32p, C.c_uint32,
                                            C.POINTER(C.c_uint32)]
        L.orc_plan_features.argtypes = [P, C.c_uint32, u32p, u32p, f32p]
        _lib = L
    return _lib


def philox4x32_10(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


@dataclass
class Graph:
    V: int
    row_ptr: np.ndarray
    dst: np.ndarray
    cost_q: np.ndarray
    S: np.ndarray
    C: np.ndarray
    is_goal: np.ndarray
    x: np.ndarray           # [6, V]
    Smax: np.ndarray = None  # per-edge peaks of the transfers (interior check)
    Cmax: np.ndarray = None


class Roadmap:
    """Owns an oracle roadmap handle."""

    def __init__(self, handle, dim: int = 0, M: int = 16):
        if not handle:
            raise RuntimeError("oracle roadmap construction failed")
        self.h = handle
        self.dim = dim
        self.M = M

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_roadmap_free(self.h)
            self.h = None

    @property
    def V(self) -> int:
        return lib().orc_roadmap_V(self.h)

    @property
    def E(self) -> int:
        return lib().orc_roadmap_E(self.h)

    def graph(self) -> Graph:
        V, E = self.V, self.E
        x = np.zeros(6 * V, np.float32)
        g = np.zeros(V, np.uint8)
        rp = np.zeros(V + 1, np.uint32)
        dst = np.zeros(max(E, 1), np.uint32)
        cq = np.zeros(max(E, 1), np.int32)
        S = np.zeros(max(E, 1), np.int32)
        Cc = np.zeros(max(E, 1), np.int32)
        lib().orc_roadmap_get(self.h, x, g, rp, dst, cq, S, Cc)
        Sm = np.zeros(max(E, 1), np.int32)
        Cm = np.zeros(max(E, 1), np.int32)
        lib().orc_roadmap_get_peaks(self.h, Sm, Cm)
        return Graph(V, rp, dst[:E], cq[:E], S[:E], Cc[:E], g, x.reshape(6, V), Sm[:E], Cm[:E])

    def edge_eval(self, u: int, v: int):
        M = self.M
        cost = np.zeros(1, np.float32); J = np.zeros(1, np.float32)
        ck = np.zeros(3 * M, np.float32); d = np.zeros(M, np.int64)
        a0 = np.zeros(3, np.float32); jk = np.zeros(3, np.float32)
        hit = lib().orc_edge_eval(self.h, u, v, cost, J, ck, d, a0, jk)
        return dict(cost=float(cost[0]), J=float(J[0]), ckpt=ck.reshape(M, 3), d=d,
                    a0=a0, jerk=jk, collides=bool(hit))

    def yaw(self) -> np.ndarray:
        out = np.zeros(self.V, np.float32)
        lib().orc_roadmap_yaw(self.h, out)
        return out

    def straight_line_h(self) -> np.ndarray:
        out = np.zeros(self.V, np.int64)
        lib().orc_straight_line_h(self.h, out)
        return out


def build_roadmap(scene, n=None, r=None, M=None, heading=None) -> Roadmap:
    """heading: None (grid form) or a uint8 array [Y][G^Dp] of level tables, table y
    for the camera heading 2 pi y / Y (the camera-heading form: node yaws drawn
    from Philox, yaw interpolated along every edge)."""
    cfg = scene.cfg
    n = cfg.n if n is None else n
    r = cfg.r if r is None else r
    M = cfg.M if M is None else M
    from scenegen import N_F, K_LEVELS, GOAL_RADIUS
    args = (cfg.dim_kind, cfg.nb, scene.box_lo.reshape(-1), scene.box_hi.reshape(-1), cfg.grid_G, scene.grid,
            N_F, K_LEVELS, n, scene.sample_seed, scene.query_id, r, cfg.T_edge, M, scene.x_init, scene.x_goal,
            GOAL_RADIUS)
    if heading is None:
        h = lib().orc_build_roadmap(*args)
    else:
        head = np.ascontiguousarray(heading, np.uint8)
        h = lib().orc_build_roadmap_heading(*args, head.shape[0], head.reshape(-1))
    return Roadmap(h, cfg.dim_kind, M)


def build_roadmap_from_points(dim, box_lo, box_hi, grid, G, x, r, T=0.25, M=16,
                              goal_radius=0.05, n_f=12, K=24, heading=None, yaw=None) -> Roadmap:
    box_lo = np.ascontiguousarray(box_lo, np.float32).reshape(-1)
    box_hi = np.ascontiguousarray(box_hi, np.float32).reshape(-1)
    if box_lo.size == 0:
        box_lo = np.zeros(3, np.float32); box_hi = np.zeros(3, np.float32)
        nb = 0
    else:
        nb = box_lo.size // 3
    x = np.ascontiguousarray(x, np.float32)
    V = x.shape[1]
    if heading is None:
        h = lib().orc_build_roadmap_from_points(dim, nb, box_lo, box_hi, G,
                                                np.ascontiguousarray(grid, np.uint8), n_f, K, V,
                                                x.reshape(-1), r, T, M, goal_radius)
    else:
        head = np.ascontiguousarray(heading, np.uint8)
        yw = None if yaw is None else np.ascontiguousarray(yaw, np.float32)
        h = lib().orc_build_roadmap_from_points_heading(dim, nb, box_lo, box_hi, G,
                                                        np.ascontiguousarray(grid, np.uint8), n_f, K, V,
                                                        x.reshape(-1), r, T, M, goal_radius, head.shape[0],
                                                        head.reshape(-1), None if yw is None else yw.ctypes.data)
    return Roadmap(h, dim, M)


def roadmap_from_csr(row_ptr, dst, cost_q, S, Cc, is_goal, Smax=None, Cmax=None) -> Roadmap:
    """A roadmap given as a CSR graph; without Smax/Cmax every edge is one step
    (its peak is its end value)."""
    row_ptr = np.ascontiguousarray(row_ptr, np.uint32)
    V = row_ptr.size - 1
    E = int(row_ptr[-1])
    pad = lambda a, t: np.ascontiguousarray(a if E else np.zeros(1), t)
    if Smax is None:
        h = lib().orc_roadmap_from_csr(V, row_ptr, pad(dst, np.uint32), pad(cost_q, np.int32),
                                       pad(S, np.int32), pad(Cc, np.int32),
                                       np.ascontiguousarray(is_goal, np.uint8))
    else:
        h = lib().orc_roadmap_from_csr_peaks(V, row_ptr, pad(dst, np.uint32), pad(cost_q, np.int32),
                                             pad(S, np.int32), pad(Cc, np.int32), pad(Smax, np.int32),
                                             pad(Cmax, np.int32), np.ascontiguousarray(is_goal, np.uint8))
    return Roadmap(h, 0, 16)


@dataclass
class ExploreResult:
    status: int
    cost: int
    h: int
    path: np.ndarray
    wavefronts: int
    expansions: int
    plans_created: int
    front_ptr: np.ndarray
    front_cost: np.ndarray
    front_h: np.ndarray
    # P_candidates in solution order (when asked for): dict(cost, h, paths, total)
    candidates: dict | None = None

    def front(self, v: int):
        a, b = int(self.front_ptr[v]), int(self.front_ptr[v + 1])
        return list(zip(self.front_cost[a:b].tolist(), self.front_h[a:b].tolist()))


def explore(rm: Roadmap, beta: int, Lambda: int, max_iters: int = 1 << 20,
            goal_termination: bool = True, max_plans: int = 1 << 28,
            candidates: int = 0, check_interior: bool = False) -> ExploreResult:
    L = lib()
    r = L.orc_explore(rm.h, int(beta), int(Lambda), int(max_iters), int(goal_termination),
                      int(max_plans), int(check_interior))
    try:
        st = C.c_int(); cost = C.c_int64(); hv = C.c_int64(); pl = C.c_uint32()
        wf = C.c_uint32(); ex = C.c_uint64(); pc = C.c_uint64(); ft = C.c_uint32()
        L.orc_result_summary(r, C.byref(st), C.byref(cost), C.byref(hv), C.byref(pl), C.byref(wf),
                             C.byref(ex), C.byref(pc), C.byref(ft))
        path = np.zeros(max(pl.value, 1), np.uint32)
        fp = np.zeros(rm.V + 1, np.uint32)
        fc = np.zeros(max(ft.value, 1), np.int64)
        fh = np.zeros(max(ft.value, 1), np.int64)
        L.orc_result_get(r, path, fp, fc, fh)
        cand = None
        if candidates and st.value == 0:
            k = C.c_uint32()
            cc = np.zeros(candidates, np.int64); ch = np.zeros(candidates, np.int64)
            cp = np.zeros(candidates + 1, np.uint32)
            cap = 1 << 22
            cpath = np.zeros(cap, np.uint32)
            tot = L.orc_result_candidates(r, candidates, cc, ch, cp, cpath, cap, C.byref(k))
            assert tot >= 0
            n = k.value
            cand = dict(cost=cc[:n], h=ch[:n], paths=[cpath[cp[i]:cp[i + 1]].copy() for i in range(n)],
                        total=tot)
        return ExploreResult(st.value, cost.value, hv.value, path[:pl.value], wf.value, ex.value,
                             pc.value, fp, fc[:ft.value], fh[:ft.value], cand)
    finally:
        L.orc_result_free(r)


def certify(rm: Roadmap, path, rollouts: int, seed: int, call_id: int, delta_fx: int,
            sigma_fx, shift):
    hits = np.zeros(4, np.uint32)
    path = np.ascontiguousarray(path, np.uint32)
    if path.size == 0:
        path = np.zeros(1, np.uint32); plen = 0
    else:
        plen = path.size
    lib().orc_certify(rm.h, path, plen, rollouts, seed, call_id, int(delta_fx),
                      np.ascontiguousarray(sigma_fx, np.int32), np.ascontiguousarray(shift, np.int32),
                      hits)
    return dict(hits_loc=int(hits[0]), hits_coll=int(hits[1]), hits_any=int(hits[2]),
                rollouts=int(hits[3]))


def certify_vio(rm: Roadmap, path, rollouts: int, seed: int, call_id: int, delta_fx: int, q_a: int,
                kp_q16: int, kv_q16: int, r_fx, trace: bool = False):
    """Closed-loop VIO Monte Carlo certification (LQR tracking, inertial
    prediction, Kalman position fixes; see certify_vio in mpap_oracle.cpp).  With
    trace: also the final axis-0 estimation error of every rollout, the Q16 Kalman
    gains (Lp, Lw) and the posterior position variance of every step, and the
    final axis-0 executed deviation of every rollout."""
    hits = np.zeros(4, np.uint32)
    path = np.ascontiguousarray(path, np.uint32)
    plen = path.size
    if plen == 0:
        path = np.zeros(1, np.uint32)
    r_fx = np.ascontiguousarray(r_fx, np.int32)
    ep = gains = p00 = None
    ptrs = [None, None, None]
    if trace and plen >= 2:
        steps = (plen - 1) * rm.M
        ep = np.zeros((max(rollouts, 1), 2), np.int64)
        gains = np.zeros((steps, 2), np.int32)
        p00 = np.zeros(steps, np.float64)
        ptrs = [ep.ctypes.data, gains.ctypes.data, p00.ctypes.data]
    lib().orc_certify_vio(rm.h, path, plen, rollouts, seed, call_id, int(delta_fx), int(q_a), int(kp_q16),
                          int(kv_q16), r_fx, hits, *ptrs)
    out = dict(hits_loc=int(hits[0]), hits_coll=int(hits[1]), hits_any=int(hits[2]), rollouts=int(hits[3]))
    if trace:
        out.update(ep_last=ep[:, 0].copy(), p_last=ep[:, 1].copy(), gains=gains, p00=p00)
    return out


def feature_levels(dp: int, box_lo, box_hi, features, G: int, headings=None, cos_half: float = -2.0,
                   range_: float = 2.0, K: int = 24) -> np.ndarray:
    """Perception levels [Y, G^dp] from mapped features: per yaw heading and grid
    cell centre, the features in range, inside the horizontal field of view and
    not occluded by a box, capped at K.  headings: [Y, 2] float32 unit vectors
    (default one bin, (1, 0)); cos_half = -2 disables the field-of-view test."""
    lo = np.ascontiguousarray(box_lo, np.float32).reshape(-1)
    hi = np.ascontiguousarray(box_hi, np.float32).reshape(-1)
    nb = lo.size // 3
    if nb == 0:
        lo = np.zeros(3, np.float32); hi = np.zeros(3, np.float32)
    feat = np.ascontiguousarray(features, np.float32).reshape(-1)
    nf = feat.size // 3
    if nf == 0:
        feat = np.zeros(3, np.float32)
    head = np.ascontiguousarray([[1.0, 0.0]] if headings is None else headings, np.float32).reshape(-1)
    Y = head.size // 2
    cells = G ** dp
    out = np.zeros(Y * cells, np.uint8)
    lib().orc_feature_levels(int(dp), int(nb), lo, hi, int(nf), feat, int(G), int(Y), head,
                             float(cos_half), float(range_), int(K), out)
    return out.reshape(Y, cells)


def group_width(lam: float, r: float) -> int:
    """Lambda = round(lambda r_n 2^24): the group cost threshold quantum (Alg. 3)."""
    return int(np.rint(np.float64(np.float32(lam)) * np.float64(np.float32(r)) * 2.0**24))


def beta_percentile(rm: Roadmap, pct: float = 60.0) -> int:
    """beta = nearest-rank percentile of the straight-line heuristic from x_init to
    every node."""
    h = np.sort(rm.straight_line_h())
    k = int(np.ceil(pct / 100.0 * h.size)) - 1
    return int(h[max(0, min(h.size - 1, k))])


def plan_features(rm: Roadmap, paths) -> np.ndarray:
    """[len(paths), 48] float32 trajectory features (surrogate input)."""
    n = len(paths)
    ptr = np.zeros(n + 1, np.uint32)
    ptr[1:] = np.cumsum([len(p) for p in paths])
    flat = np.ascontiguousarray(np.concatenate([np.asarray(p, np.uint32) for p in paths])
                                if n else np.zeros(1, np.uint32), np.uint32)
    out = np.zeros((max(n, 1), 48), np.float32)
    lib().orc_plan_features(rm.h, n, ptr, flat, out)
    return out[:n]
