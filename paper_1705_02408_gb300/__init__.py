"""Python binding of libmpap, the GB300 (sm_103a) MPAP hot-path library.

Argument marshalling only: every step of roadmap construction (Alg. 2), the
wavefront multiobjective search (Alg. 3) and Monte Carlo certification runs in
the library's CUDA kernels.  The library must have been built
(``paper_1705_02408_gb300.build.build()``); importing the binding without it
raises, and there is no CPU fallback.

Streams: calls take ``stream`` (a ``torch.cuda.Stream`` or a raw handle); by default
torch's current stream on the current device is used.  Scene arrays may be numpy
arrays (host, copied) or CUDA torch tensors (device, read in place).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpap.so")

MPAP_OK, MPAP_NO_SOLUTION = 0, 1
MPAP_ERR_INVALID_ARG, MPAP_ERR_CAPACITY, MPAP_ERR_TIMEOUT = -1, -2, -3
MPAP_ERR_ITER_LIMIT, MPAP_ERR_CUDA, MPAP_ERR_SAMPLING = -4, -5, -6
MPAP_MEM_HOST, MPAP_MEM_DEVICE = 0, 1
MPAP_QUERY_NO_GOAL_STOP = 1
MPAP_QUERY_CHECK_INTERIOR = 2
MPAP_QUERY_OWN_SHARE = 4

EXPORTS = ["mpap_status_string", "mpap_last_error", "mpap_build_roadmap", "mpap_build_roadmaps",
           "mpap_build_roadmap_from_points", "mpap_roadmap_from_csr", "mpap_roadmap_info",
           "mpap_roadmap_export", "mpap_roadmap_stats", "mpap_roadmap_free", "mpap_workspace_create",
           "mpap_workspace_free", "mpap_search", "mpap_search_batch", "mpap_search_fronts",
           "mpap_certify", "mpap_certify_batch", "mpap_certify_noalloc", "mpap_profile_enable", "mpap_profile_reset",
           "mpap_launch_count", "mpap_profile_read", "mpap_search_candidates", "mpap_plan_features",
           "mpap_mlp_create", "mpap_mlp_free", "mpap_mlp_get_params", "mpap_mlp_set_params",
           "mpap_mlp_forward", "mpap_mlp_train_step", "mpap_tuning_get", "mpap_tuning_set",
           "mpap_tuning_clear", "mpap_tuning_export", "mpap_autotune_build", "mpap_autotune_search",
           "mpap_search_candidates_batch", "mpap_plan_features_batch", "mpap_roadmap_from_csr_peaks",
           "mpap_roadmap_export_peaks", "mpap_roadmap_export_reverse", "mpap_feature_levels",
           "mpap_roadmap_update", "mpap_roadmap_update_batch", "mpap_refine_advance", "mpap_refine_batch",
           "mpap_surrogate_screen", "mpap_errnet_create", "mpap_errnet_free", "mpap_errnet_get_params",
           "mpap_errnet_set_params", "mpap_errnet_forward", "mpap_errnet_train_step", "mpap_errmap_query",
           "mpap_errmap_levels", "mpap_workspace_stats", "mpap_certify_vio_batch",
           "mpap_vio_lqr_gains", "mpap_roadmap_export_yaw"]


class mpap_scene(C.Structure):
    _fields_ = [("dim_kind", C.c_int32), ("nb", C.c_int32), ("box_lo", C.c_void_p),
                ("box_hi", C.c_void_p), ("grid_G", C.c_int32), ("grid_level", C.c_void_p),
                ("n_f", C.c_int32), ("K", C.c_int32), ("mem", C.c_int32), ("n_heading", C.c_int32),
                ("heading_levels", C.c_void_p)]


class mpap_roadmap_params(C.Structure):
    _fields_ = [("n", C.c_uint32), ("query_id", C.c_uint32), ("seed", C.c_uint64),
                ("r", C.c_float), ("T_edge", C.c_float), ("M", C.c_int32),
                ("x_init", C.c_float * 6), ("x_goal", C.c_float * 6), ("goal_radius", C.c_float)]


class mpap_query(C.Structure):
    _fields_ = [("beta", C.c_int64), ("group_width_q", C.c_int64), ("lambda_", C.c_float),
                ("max_iters", C.c_uint32), ("flags", C.c_uint32), ("wait_us", C.c_uint32)]


class mpap_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("cost", C.c_int64), ("h", C.c_int64),
                ("path_len", C.c_uint32), ("path_cap", C.c_uint32),
                ("path", C.POINTER(C.c_uint32)), ("wavefronts", C.c_uint32),
                ("expansions", C.c_uint64), ("plans", C.c_uint64)]


class mpap_mc_params(C.Structure):
    _fields_ = [("rollouts", C.c_uint32), ("call_id", C.c_uint32), ("seed", C.c_uint64),
                ("delta_fx", C.c_int64), ("sigma_fx", C.POINTER(C.c_int32)),
                ("shift", C.POINTER(C.c_int32))]


class mpap_tuning(C.Structure):
    _fields_ = [("edge_warps", C.c_uint32), ("wave_blocks_per_sm", C.c_uint32),
                ("plan_lanes_from", C.c_uint32), ("front_cap", C.c_uint32),
                ("grid_merge_from", C.c_uint32)]


class mpap_vio_params(C.Structure):
    _fields_ = [("q_a", C.c_int32), ("kp_q16", C.c_int32), ("kv_q16", C.c_int32),
                ("r_fx", C.POINTER(C.c_int32))]


class mpap_cert(C.Structure):
    _fields_ = [("hits_loc", C.c_uint32), ("hits_coll", C.c_uint32), ("hits_any", C.c_uint32),
                ("rollouts", C.c_uint32)]


MPAP_REFINE_PASS, MPAP_REFINE_FAIL, MPAP_REFINE_NONE, MPAP_REFINE_ERROR = 0, 1, 2, 3


class mpap_refine_bounds(C.Structure):
    _fields_ = [("lo", C.c_int64), ("lo_cost", C.c_int64), ("hi", C.c_int64), ("none", C.c_int64)]


class mpap_refine_round(C.Structure):
    _fields_ = [("beta", C.c_int64), ("cost", C.c_int64), ("outcome", C.c_int32), ("hits", C.c_int32)]


class mpap_refine_result(C.Structure):
    _fields_ = [("certified", C.c_int32), ("status", C.c_int32), ("beta", C.c_int64), ("cost", C.c_int64),
                ("h", C.c_int64), ("path_len", C.c_uint32), ("path_cap", C.c_uint32),
                ("path", C.POINTER(C.c_uint32)), ("cert", mpap_cert), ("rounds", C.c_uint32),
                ("hist_cap", C.c_uint32), ("history", C.POINTER(mpap_refine_round))]


_NP_SCALAR = {C.c_int32: "i4", C.c_uint32: "u4", C.c_int64: "i8", C.c_uint64: "u8", C.c_float: "f4"}


def _np_dtype(cls):
    """numpy structured dtype with the byte layout of the ctypes struct `cls`
    (pointers as uint64 addresses), so that a whole batch of structs is filled
    column by column and handed to the library as one array."""
    assert C.sizeof(C.c_void_p) == 8
    names, formats, offsets = [], [], []
    for name, ct in cls._fields_:
        if ct in _NP_SCALAR:
            fmt = _NP_SCALAR[ct]
        elif issubclass(ct, C.Array):
            fmt = (_NP_SCALAR[ct._type_], (ct._length_,))
        else:                                   # c_void_p and POINTER(...)
            fmt = "u8"
        names.append(name)
        formats.append(fmt)
        offsets.append(getattr(cls, name).offset)
    dt = np.dtype({"names": names, "formats": formats, "offsets": offsets, "itemsize": C.sizeof(cls)})
    assert dt.itemsize == C.sizeof(cls)
    return dt


SCENE_DT, PARAMS_DT, QUERY_DT, RESULT_DT, MC_DT, CERT_DT = (
    _np_dtype(t) for t in (mpap_scene, mpap_roadmap_params, mpap_query, mpap_result, mpap_mc_params, mpap_cert))


def _as(a, cls):
    """A numpy struct array as a ctypes pointer to `cls`."""
    return a.ctypes.data_as(C.POINTER(cls))


_lib = None


def lib():
    """The loaded libmpap.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmpap.so not built at {LIB_PATH}: run "
                              "paper_1705_02408_gb300.build.build() (nvcc, sm_103a)")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        i32 = C.c_int32
        L.mpap_status_string.restype = C.c_char_p
        L.mpap_status_string.argtypes = [i32]
        L.mpap_last_error.restype = C.c_char_p
        L.mpap_build_roadmap.restype = i32
        L.mpap_build_roadmap.argtypes = [C.POINTER(mpap_scene), C.POINTER(mpap_roadmap_params),
                                         C.POINTER(P), P]
        L.mpap_build_roadmaps.restype = i32
        L.mpap_build_roadmaps.argtypes = [C.c_uint32, C.POINTER(mpap_scene), C.POINTER(mpap_roadmap_params),
                                          C.POINTER(P), P]
        L.mpap_build_roadmap_from_points.restype = i32
        L.mpap_build_roadmap_from_points.argtypes = [C.POINTER(mpap_scene), C.c_uint32, P, C.c_float,
                                                     C.c_float, i32, C.c_float, C.POINTER(P), P]
        L.mpap_roadmap_from_csr.restype = i32
        L.mpap_roadmap_from_csr.argtypes = [C.c_uint32, P, P, P, P, P, P, C.POINTER(P), P]
        L.mpap_roadmap_info.restype = i32
        L.mpap_roadmap_info.argtypes = [P, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)]
        L.mpap_roadmap_export.restype = i32
        L.mpap_roadmap_export.argtypes = [P, P, P, P, P, P, P, P, P]
        L.mpap_roadmap_free.argtypes = [P]
        L.mpap_roadmap_stats.restype = i32
        L.mpap_roadmap_stats.argtypes = [P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)]
        L.mpap_workspace_create.restype = i32
        L.mpap_workspace_create.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.POINTER(P)]
        L.mpap_workspace_free.argtypes = [P]
        L.mpap_workspace_stats.restype = i32
        L.mpap_workspace_stats.argtypes = [P, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)]
        L.mpap_search.restype = i32
        L.mpap_search.argtypes = [P, P, C.POINTER(mpap_query), C.POINTER(mpap_result), P]
        L.mpap_search_batch.restype = i32
        L.mpap_search_batch.argtypes = [P, C.POINTER(P), C.POINTER(mpap_query), C.c_uint32,
                                        C.POINTER(mpap_result), P]
        L.mpap_search_fronts.restype = i32
        L.mpap_search_fronts.argtypes = [P, C.c_uint32, P, P, P, C.c_uint64,
                                         C.POINTER(C.c_uint64), P]
        L.mpap_certify.restype = i32
        L.mpap_certify.argtypes = [P, P, C.c_uint32, C.POINTER(mpap_mc_params),
                                   C.POINTER(mpap_cert), P]
        L.mpap_certify_noalloc.restype = i32
        L.mpap_certify_noalloc.argtypes = [P, P, C.c_uint32, C.POINTER(mpap_mc_params),
                                           C.POINTER(mpap_cert), P]
        L.mpap_certify_batch.restype = i32
        L.mpap_certify_batch.argtypes = [C.POINTER(P), C.POINTER(P), P, C.POINTER(mpap_mc_params),
                                         C.c_uint32, C.POINTER(mpap_cert), P]
        L.mpap_roadmap_export_yaw.restype = i32
        L.mpap_roadmap_export_yaw.argtypes = [P, P, P]
        L.mpap_vio_lqr_gains.restype = i32
        L.mpap_vio_lqr_gains.argtypes = [C.c_double, C.c_double, C.c_double, C.POINTER(C.c_int32),
                                         C.POINTER(C.c_int32)]
        L.mpap_certify_vio_batch.restype = i32
        L.mpap_certify_vio_batch.argtypes = [C.POINTER(P), C.POINTER(P), P, C.POINTER(mpap_mc_params),
                                             C.POINTER(mpap_vio_params), C.c_uint32, C.POINTER(mpap_cert), P]
        L.mpap_profile_enable.restype = i32
        L.mpap_profile_enable.argtypes = [i32]
        L.mpap_profile_reset.restype = i32
        L.mpap_launch_count.restype = C.c_uint64
        L.mpap_profile_read.restype = i32
        L.mpap_profile_read.argtypes = [C.c_uint32, P, P, P, C.POINTER(C.c_uint32)]
        u32p = C.POINTER(C.c_uint32)
        L.mpap_search_candidates.restype = i32
        L.mpap_search_candidates.argtypes = [P, C.c_uint32, C.c_uint32, P, P, P, P, C.c_uint32, u32p, u32p, P]
        L.mpap_roadmap_from_csr_peaks.restype = i32
        L.mpap_roadmap_from_csr_peaks.argtypes = [C.c_uint32, P, P, P, P, P, P, P, P, C.POINTER(P), P]
        L.mpap_roadmap_export_peaks.restype = i32
        L.mpap_roadmap_export_peaks.argtypes = [P, P, P, P]
        L.mpap_roadmap_export_reverse.restype = i32
        L.mpap_roadmap_export_reverse.argtypes = [P, P, P, P, P, P, P, P, P]
        L.mpap_roadmap_update.restype = i32
        L.mpap_roadmap_update.argtypes = [P, i32, P, P, P, i32, P]
        L.mpap_roadmap_update_batch.restype = i32
        L.mpap_roadmap_update_batch.argtypes = [C.POINTER(P), C.c_uint32, P, C.POINTER(P), C.POINTER(P),
                                                C.POINTER(P), i32, P]
        L.mpap_feature_levels.restype = i32
        L.mpap_feature_levels.argtypes = [i32, i32, P, P, C.c_uint32, P, i32, C.c_uint32, P, C.c_float,
                                          C.c_float, i32, P, i32, P]
        L.mpap_search_candidates_batch.restype = i32
        L.mpap_search_candidates_batch.argtypes = [P, C.c_uint32, C.c_uint32, P, P, P, P, C.c_uint32, P, P, P]
        L.mpap_plan_features_batch.restype = i32
        L.mpap_plan_features_batch.argtypes = [C.POINTER(P), C.c_uint32, P, P, P, P, P]
        L.mpap_plan_features.restype = i32
        L.mpap_plan_features.argtypes = [P, C.c_uint32, P, P, P, P]
        L.mpap_mlp_create.restype = i32
        L.mpap_mlp_create.argtypes = [C.c_uint64, C.c_uint32, C.POINTER(P)]
        L.mpap_mlp_free.argtypes = [P]
        L.mpap_mlp_get_params.restype = i32
        L.mpap_mlp_get_params.argtypes = [P, P, P]
        L.mpap_mlp_set_params.restype = i32
        L.mpap_mlp_set_params.argtypes = [P, P, P]
        L.mpap_mlp_forward.restype = i32
        L.mpap_mlp_forward.argtypes = [P, P, C.c_uint32, P, i32, P]
        L.mpap_mlp_train_step.restype = i32
        L.mpap_mlp_train_step.argtypes = [P, P, P, C.c_uint32, C.c_float, i32, C.POINTER(C.c_float), P, i32, P]
        L.mpap_errnet_create.argtypes = [C.c_uint64, C.c_uint32, C.POINTER(P)]
        L.mpap_errnet_free.argtypes = [P]
        L.mpap_errnet_free.restype = None
        L.mpap_errnet_get_params.argtypes = [P, P, P]
        L.mpap_errnet_set_params.argtypes = [P, P, P]
        L.mpap_errnet_forward.argtypes = [P, P, C.c_uint32, P, i32, P]
        L.mpap_errnet_train_step.argtypes = [P, P, P, C.c_uint32, C.c_float, i32, C.POINTER(C.c_float), P, i32, P]
        L.mpap_errmap_query.argtypes = [P, P, C.c_uint32, P, C.c_uint32, C.c_uint32, P, P, i32, P]
        L.mpap_errmap_levels.argtypes = [P, P, C.c_uint32, C.c_uint32, P, i32, i32, P, C.c_float, C.c_float, i32,
                                         i32, P, i32, P]
        L.mpap_refine_advance.argtypes = [C.POINTER(mpap_refine_bounds), C.c_int64, C.c_int32, C.c_int64,
                                          C.POINTER(C.c_int64)]
        L.mpap_refine_batch.argtypes = [P, C.POINTER(P), C.POINTER(mpap_query), C.POINTER(mpap_mc_params),
                                        P, C.c_uint32, C.c_uint32, C.POINTER(mpap_refine_result), P]
        L.mpap_surrogate_screen.argtypes = [P, C.POINTER(P), C.c_uint32, P, P, P, P, C.POINTER(mpap_mc_params),
                                            C.c_double, C.c_float, i32, C.c_uint32, P, P,
                                            C.POINTER(C.c_uint32), P, P]
        TP = C.POINTER(mpap_tuning)
        L.mpap_tuning_get.restype = i32
        L.mpap_tuning_get.argtypes = [i32, C.c_uint32, TP]
        L.mpap_tuning_set.restype = i32
        L.mpap_tuning_set.argtypes = [i32, C.c_uint32, TP]
        L.mpap_tuning_clear.restype = i32
        L.mpap_tuning_export.restype = i32
        L.mpap_tuning_export.argtypes = [C.c_uint32, P, P, P, C.POINTER(C.c_uint32)]
        L.mpap_autotune_build.restype = i32
        L.mpap_autotune_build.argtypes = [C.c_uint32, C.POINTER(mpap_scene), C.POINTER(mpap_roadmap_params),
                                          C.POINTER(P), C.c_uint32, TP, C.POINTER(C.c_double), P]
        L.mpap_autotune_search.restype = i32
        L.mpap_autotune_search.argtypes = [P, C.POINTER(P), C.POINTER(mpap_query), C.c_uint32, C.c_uint32, TP,
                                           C.POINTER(C.c_double), P]
        _lib = L
    return _lib


def profile_enable(on=True):
    lib().mpap_profile_enable(1 if on else 0)


def profile_reset():
    lib().mpap_profile_reset()


def launch_count() -> int:
    return int(lib().mpap_launch_count())


def profile_read():
    """{kernel name: (launches, total device ms)} since the last reset."""
    cap = 64
    names = C.create_string_buffer(64 * cap)
    launches = np.zeros(cap, np.uint64); ms = np.zeros(cap, np.float64)
    n = C.c_uint32()
    _check(lib().mpap_profile_read(cap, names, launches.ctypes.data_as(C.c_void_p),
                                   ms.ctypes.data_as(C.c_void_p), C.byref(n)), "mpap_profile_read")
    out = {}
    raw = names.raw
    for i in range(min(n.value, cap)):
        nm = raw[64 * i:64 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[i]), float(ms[i]))
    return out


class MpapError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        L = lib()
        msg = L.mpap_last_error().decode(errors="replace")
        super().__init__(f"{what}: {L.mpap_status_string(status).decode()} ({status}): {msg}")


def _check(status, what):
    if status < 0:
        raise MpapError(status, what)
    return status


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _ptr(a, dtype):
    """(pointer, keepalive, is_device) for a numpy array or a torch tensor."""
    if a is None:
        return None, None, False
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr()), a, bool(a.is_cuda)
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(C.c_void_p), arr, False


def _addr(a, dtype):
    """(address, keepalive, is_device, element count) for a numpy array or a torch tensor."""
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a, bool(a.is_cuda), a.numel()
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.__array_interface__["data"][0], arr, False, arr.size


def make_scene_struct(dim_kind, box_lo, box_hi, grid, grid_G, n_f=12, K=24, heading=None):
    """An mpap_scene over numpy (host) or CUDA tensor (device) arrays.  heading:
    None, or the camera-heading form's level tables [Y][G^Dp] (uint8, same
    memory kind as the grid)."""
    lo_p, lo_k, lo_d = _ptr(box_lo, np.float32)
    hi_p, hi_k, hi_d = _ptr(box_hi, np.float32)
    g_p, g_k, g_d = _ptr(grid, np.uint8)
    nb = (lo_k.numel() if hasattr(lo_k, "numel") else lo_k.size) // 3
    kinds = {lo_d, hi_d, g_d}
    h_p, h_k, Y = None, None, 0
    if heading is not None:
        h_p, h_k, h_d = _ptr(heading, np.uint8)
        kinds.add(h_d)
        Y = int(heading.shape[0])
    if len(kinds) != 1:
        raise ValueError("scene arrays must all be on the host or all on the device")
    s = mpap_scene(dim_kind=dim_kind, nb=nb, box_lo=lo_p if nb else None,
                   box_hi=hi_p if nb else None, grid_G=grid_G, grid_level=g_p, n_f=n_f, K=K,
                   mem=MPAP_MEM_DEVICE if g_d else MPAP_MEM_HOST, n_heading=Y, heading_levels=h_p)
    return s, (lo_k, hi_k, g_k, h_k)


class Roadmap:
    """An mpap_roadmap handle (device CSR graph with per-edge transfers)."""

    def __init__(self, handle, M=16, K=24):
        self.h = handle
        self.M = M
        self.K = K

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.mpap_roadmap_free(self.h)
            self.h = None

    def info(self):
        V = C.c_uint32(); E = C.c_uint64()
        _check(lib().mpap_roadmap_info(self.h, C.byref(V), C.byref(E)), "mpap_roadmap_info")
        return V.value, E.value

    def stats(self):
        """(Near tests evaluated by the last build, nodes in X_goal)."""
        nt = C.c_uint64(); ng = C.c_uint32()
        _check(lib().mpap_roadmap_stats(self.h, C.byref(nt), C.byref(ng)), "mpap_roadmap_stats")
        return nt.value, ng.value

    @property
    def V(self):
        return self.info()[0]

    @property
    def E(self):
        return self.info()[1]

    def export(self, stream=None):
        V, E = self.info()
        x = np.zeros(6 * V, np.float32); g = np.zeros(V, np.uint8)
        rp = np.zeros(V + 1, np.uint32)
        dst = np.zeros(max(E, 1), np.uint32); cq = np.zeros(max(E, 1), np.int32)
        S = np.zeros(max(E, 1), np.int32); Cc = np.zeros(max(E, 1), np.int32)
        vp = lambda a: a.ctypes.data_as(C.c_void_p)
        _check(lib().mpap_roadmap_export(self.h, vp(x), vp(g), vp(rp), vp(dst), vp(cq), vp(S), vp(Cc),
                                         _stream(stream)), "mpap_roadmap_export")
        return dict(V=V, E=E, x=x.reshape(6, V), is_goal=g, row_ptr=rp, dst=dst[:E], cost_q=cq[:E],
                    S=S[:E], C=Cc[:E])

    def export_reverse(self, stream=None):
        """mpap_roadmap_export_reverse: the in-edge CSR, rows sorted by source."""
        V, E = self.info()
        rp = np.zeros(V + 1, np.uint32)
        cols = [np.zeros(max(E, 1), t) for t in (np.uint32, np.int32, np.int32, np.int32, np.int32, np.int32)]
        vp = lambda a: a.ctypes.data_as(C.c_void_p)
        _check(lib().mpap_roadmap_export_reverse(self.h, vp(rp), *[vp(c) for c in cols], _stream(stream)),
               "mpap_roadmap_export_reverse")
        src, cq, S, Cc, Sm, Cm = (c[:E] for c in cols)
        return dict(V=V, E=E, rev_ptr=rp, src=src, cost_q=cq, S=S, C=Cc, Smax=Sm, Cmax=Cm)

    def update(self, add_lo=None, add_hi=None, grid=None, stream=None):
        """mpap_roadmap_update: append boxes (float [k, 3] each) and/or replace
        the quality grid (uint8 [G^Dp]); numpy arrays or CUDA tensors."""
        dev = any(hasattr(a, "is_cuda") and a.is_cuda for a in (add_lo, add_hi, grid) if a is not None)
        keep = []

        def ptr(a, dtype):
            if a is None:
                return None, 0
            if hasattr(a, "data_ptr"):
                if not a.is_contiguous():
                    raise ValueError("arrays must be contiguous")
                keep.append(a)
                return C.c_void_p(a.data_ptr()), a.numel()
            arr = np.ascontiguousarray(a, dtype)
            keep.append(arr)
            return arr.ctypes.data_as(C.c_void_p), arr.size

        lo, n_lo = ptr(add_lo, np.float32)
        hi, n_hi = ptr(add_hi, np.float32)
        if n_lo != n_hi or n_lo % 3:
            raise ValueError("add_lo and add_hi must both be [k, 3]")
        g, _ = ptr(grid, np.uint8)
        _check(lib().mpap_roadmap_update(self.h, n_lo // 3, lo if n_lo else None, hi if n_hi else None, g,
                                         MPAP_MEM_DEVICE if dev else MPAP_MEM_HOST, _stream(stream)),
               "mpap_roadmap_update")
        return self

    def yaw(self, stream=None):
        """mpap_roadmap_export_yaw: node yaws (camera-heading form; zeros otherwise)."""
        out = np.zeros(self.V, np.float32)
        _check(lib().mpap_roadmap_export_yaw(self.h, out.ctypes.data_as(C.c_void_p), _stream(stream)),
               "mpap_roadmap_export_yaw")
        return out

    def peaks(self, stream=None):
        """(Smax, Cmax) per edge, in the order of export()."""
        E = self.info()[1]
        Sm = np.zeros(max(E, 1), np.int32); Cm = np.zeros(max(E, 1), np.int32)
        _check(lib().mpap_roadmap_export_peaks(self.h, Sm.ctypes.data_as(C.c_void_p),
                                               Cm.ctypes.data_as(C.c_void_p), _stream(stream)),
               "mpap_roadmap_export_peaks")
        return Sm[:E], Cm[:E]


def build_roadmap(dim_kind, box_lo, box_hi, grid, grid_G, n, seed, r, x_init, x_goal,
                  goal_radius=0.05, T=0.25, M=16, query_id=0, n_f=12, K=24, heading=None, stream=None) -> Roadmap:
    """mpap_build_roadmap: V = {x_init, x_goal} + SampleFree(n), r-disc graph (Alg. 2)."""
    sc, keep = make_scene_struct(dim_kind, box_lo, box_hi, grid, grid_G, n_f, K, heading)
    p = mpap_roadmap_params(n=n, query_id=query_id, seed=seed, r=r, T_edge=T, M=M,
                            goal_radius=goal_radius)
    for i in range(6):
        p.x_init[i] = float(x_init[i]); p.x_goal[i] = float(x_goal[i])
    h = C.c_void_p()
    _check(lib().mpap_build_roadmap(C.byref(sc), C.byref(p), C.byref(h), _stream(stream)),
           "mpap_build_roadmap")
    return Roadmap(h, M, K)


def _params(n, seed, r, x_init, x_goal, goal_radius, T, M, query_id):
    p = mpap_roadmap_params(n=n, query_id=query_id, seed=seed, r=r, T_edge=T, M=M, goal_radius=goal_radius)
    for i in range(6):
        p.x_init[i] = float(x_init[i]); p.x_goal[i] = float(x_goal[i])
    return p


def _batch_structs(specs):
    """mpap_scene and mpap_roadmap_params arrays (numpy, C layout) for a list of
    build_roadmap keyword dicts, plus the arrays they point into."""
    n = len(specs)
    scenes = np.zeros(n, SCENE_DT)
    params = np.zeros(n, PARAMS_DT)
    keep = []
    lo, hi, gl, nb, mem, heads = [], [], [], [], [], []
    for sp in specs:
        a_lo, k_lo, d_lo, n_lo = _addr(sp["box_lo"], np.float32)
        a_hi, k_hi, d_hi, _ = _addr(sp["box_hi"], np.float32)
        a_g, k_g, d_g, _ = _addr(sp["grid"], np.uint8)
        if not (d_lo == d_hi == d_g):
            raise ValueError("scene arrays must all be on the host or all on the device")
        hd = sp.get("heading")
        if hd is not None:
            a_h, k_h, d_h, _ = _addr(hd, np.uint8)
            if d_h != d_g:
                raise ValueError("scene arrays must all be on the host or all on the device")
            heads.append((int(hd.shape[0]), a_h))
        else:
            k_h = None
            heads.append((0, 0))
        keep.append((k_lo, k_hi, k_g, k_h))
        nb.append(n_lo // 3)
        lo.append(a_lo if n_lo else 0)
        hi.append(a_hi if n_lo else 0)
        gl.append(a_g)
        mem.append(MPAP_MEM_DEVICE if d_g else MPAP_MEM_HOST)
    g = lambda k, d: [sp.get(k, d) for sp in specs]
    scenes["dim_kind"] = [sp["dim_kind"] for sp in specs]
    scenes["nb"] = nb
    scenes["box_lo"] = lo
    scenes["box_hi"] = hi
    scenes["grid_G"] = [sp["grid_G"] for sp in specs]
    scenes["grid_level"] = gl
    scenes["n_f"] = g("n_f", 12)
    scenes["K"] = g("K", 24)
    scenes["mem"] = mem
    scenes["n_heading"] = [h[0] for h in heads]
    scenes["heading_levels"] = [h[1] for h in heads]
    params["n"] = [sp["n"] for sp in specs]
    params["query_id"] = g("query_id", 0)
    params["seed"] = [sp["seed"] for sp in specs]
    params["r"] = [sp["r"] for sp in specs]
    params["T_edge"] = g("T", 0.25)
    params["M"] = g("M", 16)
    params["x_init"] = np.asarray([sp["x_init"] for sp in specs], np.float32).reshape(n, 6)
    params["x_goal"] = np.asarray([sp["x_goal"] for sp in specs], np.float32).reshape(n, 6)
    params["goal_radius"] = g("goal_radius", 0.05)
    return scenes, params, keep


def _adopt(specs, rms, hs):
    out = []
    for i in range(len(specs)):
        if rms[i] is not None:
            rms[i].h = C.c_void_p(hs[i]) if hs[i] else None
            rms[i].M = specs[i].get("M", 16)
            out.append(rms[i])
        else:
            out.append(Roadmap(C.c_void_p(hs[i]), specs[i].get("M", 16), specs[i].get("K", 24)) if hs[i] else None)
    return out


def build_roadmaps(specs, rms=None, stream=None):
    """mpap_build_roadmaps: build every roadmap of `specs` in one pass.

    specs: list of dicts with the keyword arguments of build_roadmap.  rms: an
    optional list of Roadmap handles (or None entries) rebuilt in place."""
    n = len(specs)
    scenes, params, keep = _batch_structs(specs)
    rms = list(rms) if rms is not None else [None] * n
    hs = (C.c_void_p * n)(*[rm.h.value if rm is not None and rm.h else None for rm in rms])
    rc = lib().mpap_build_roadmaps(n, _as(scenes, mpap_scene), _as(params, mpap_roadmap_params), hs,
                                   _stream(stream))
    out = _adopt(specs, rms, hs)
    _check(rc, "mpap_build_roadmaps")
    return out


def feature_levels(dim_kind, box_lo, box_hi, features, grid_G, headings=None, cos_half_fov=-2.0, range_=2.0,
                   K=24, stream=None):
    """mpap_feature_levels: perception levels [Y, G^Dp] (uint8) from mapped features
    for Y camera headings (default one, (1, 0)); numpy in and out, or CUDA tensors
    (all arrays on the device; levels returned as a uint8 tensor)."""
    dp = 2 if dim_kind == 2 else 3
    cells = int(grid_G) ** dp
    dev = hasattr(features, "is_cuda") and features.is_cuda
    if dev:
        import torch
        head = headings if headings is not None else torch.tensor([[1.0, 0.0]], device=features.device)
        for a in (box_lo, box_hi, features, head):
            if a.dtype != torch.float32 or not a.is_cuda or not a.is_contiguous():
                raise ValueError("feature_levels: device arrays must be contiguous float32 CUDA tensors")
        Y = head.numel() // 2
        out = torch.empty((Y, cells), dtype=torch.uint8, device=features.device)
        nb = box_lo.numel() // 3
        nf = features.numel() // 3
        ptr = lambda a: C.c_void_p(a.data_ptr()) if a.numel() else None
        _check(lib().mpap_feature_levels(int(dim_kind), nb, ptr(box_lo), ptr(box_hi), nf, ptr(features),
                                         int(grid_G), Y, ptr(head), float(cos_half_fov), float(range_), int(K),
                                         C.c_void_p(out.data_ptr()), MPAP_MEM_DEVICE, _stream(stream)),
               "mpap_feature_levels")
        return out
    lo = np.ascontiguousarray(box_lo, np.float32).reshape(-1)
    hi = np.ascontiguousarray(box_hi, np.float32).reshape(-1)
    f = np.ascontiguousarray(features, np.float32).reshape(-1)
    head = np.ascontiguousarray([[1.0, 0.0]] if headings is None else headings, np.float32).reshape(-1)
    Y = head.size // 2
    out = np.zeros((Y, cells), np.uint8)
    vp = lambda a: a.ctypes.data_as(C.c_void_p) if a.size else None
    _check(lib().mpap_feature_levels(int(dim_kind), lo.size // 3, vp(lo), vp(hi), f.size // 3, vp(f), int(grid_G),
                                     Y, vp(head), float(cos_half_fov), float(range_), int(K),
                                     out.ctypes.data_as(C.c_void_p), MPAP_MEM_HOST, _stream(stream)),
           "mpap_feature_levels")
    return out


def roadmap_update_batch(rms, adds_lo, adds_hi, grids=None, stream=None):
    """mpap_roadmap_update_batch: roadmap j gets the boxes adds_lo[j], adds_hi[j]
    (float [k_j, 3], k_j may be 0) and, when given, the levels grids[j] (uint8
    [G^Dp] or None); host numpy arrays."""
    n = len(rms)
    keep = []

    def arr(a, dtype):
        if a is None:
            return None
        x = np.ascontiguousarray(a, dtype)
        keep.append(x)
        return x.ctypes.data if x.size else None

    los = [arr(a, np.float32) for a in adds_lo]
    his = [arr(a, np.float32) for a in adds_hi]
    nb = np.array([0 if a is None else np.asarray(a).size // 3 for a in adds_lo], np.int32)
    gs = [arr(g, np.uint8) for g in grids] if grids is not None else None
    hs = (C.c_void_p * n)(*[rm.h for rm in rms])
    lp = (C.c_void_p * n)(*los)
    hp = (C.c_void_p * n)(*his)
    gp = (C.c_void_p * n)(*gs) if gs is not None else None
    _check(lib().mpap_roadmap_update_batch(hs, n, nb.ctypes.data_as(C.c_void_p), lp, hp, gp, MPAP_MEM_HOST,
                                           _stream(stream)), "mpap_roadmap_update_batch")
    return rms


def scene_spec(scene, n=None, r=None, M=None, device_inputs=None, heading=None):
    """Keyword arguments of build_roadmap for a scenegen.Scene (device_inputs: a
    (box_lo, box_hi, grid) triple of CUDA tensors to read in place; heading: the
    camera-heading form's level tables [Y][G^Dp], or None)."""
    cfg = scene.cfg
    lo, hi, grid = (scene.box_lo, scene.box_hi, scene.grid) if device_inputs is None else device_inputs
    return dict(dim_kind=cfg.dim_kind, box_lo=lo, box_hi=hi, grid=grid, grid_G=cfg.grid_G,
                n=cfg.n if n is None else n, seed=scene.sample_seed, r=cfg.r if r is None else r,
                x_init=scene.x_init, x_goal=scene.x_goal, T=cfg.T_edge, M=cfg.M if M is None else M,
                query_id=scene.query_id, heading=heading)


def build_roadmap_from_points(dim_kind, box_lo, box_hi, grid, grid_G, x, r, T=0.25, M=16,
                              goal_radius=0.05, n_f=12, K=24, stream=None) -> Roadmap:
    box_lo = np.asarray(box_lo, np.float32).reshape(-1, 3) if not hasattr(box_lo, "is_cuda") else box_lo
    box_hi = np.asarray(box_hi, np.float32).reshape(-1, 3) if not hasattr(box_hi, "is_cuda") else box_hi
    sc, keep = make_scene_struct(dim_kind, box_lo, box_hi, grid, grid_G, n_f, K)
    x = np.ascontiguousarray(x, np.float32)
    h = C.c_void_p()
    _check(lib().mpap_build_roadmap_from_points(C.byref(sc), x.shape[1], x.ctypes.data_as(C.c_void_p), r, T,
                                                M, goal_radius, C.byref(h), _stream(stream)),
           "mpap_build_roadmap_from_points")
    return Roadmap(h, M, K)


def roadmap_from_csr(row_ptr, dst, cost_q, S, Cc, is_goal, Smax=None, Cmax=None, stream=None) -> Roadmap:
    """mpap_roadmap_from_csr (or _peaks when Smax/Cmax are given)."""
    arrs = [np.ascontiguousarray(row_ptr, np.uint32), np.ascontiguousarray(dst, np.uint32),
            np.ascontiguousarray(cost_q, np.int32), np.ascontiguousarray(S, np.int32),
            np.ascontiguousarray(Cc, np.int32)]
    goal = np.ascontiguousarray(is_goal, np.uint8)
    arrs = [a if a.size else np.zeros(1, a.dtype) for a in arrs]
    vp = lambda a: a.ctypes.data_as(C.c_void_p)
    h = C.c_void_p()
    if Smax is None:
        _check(lib().mpap_roadmap_from_csr(len(row_ptr) - 1, *[vp(a) for a in arrs], vp(goal), C.byref(h),
                                           _stream(stream)), "mpap_roadmap_from_csr")
    else:
        pk = [np.ascontiguousarray(Smax, np.int32), np.ascontiguousarray(Cmax, np.int32)]
        pk = [a if a.size else np.zeros(1, a.dtype) for a in pk]
        _check(lib().mpap_roadmap_from_csr_peaks(len(row_ptr) - 1, *[vp(a) for a in arrs + pk], vp(goal),
                                                 C.byref(h), _stream(stream)), "mpap_roadmap_from_csr_peaks")
    return Roadmap(h)


def build_roadmap_for_scene(scene, n=None, r=None, M=None, device_inputs=False, heading=None,
                            stream=None) -> Roadmap:
    """Convenience: build from a scenegen.Scene (host arrays, or device copies;
    heading: the camera-heading form's level tables [Y][G^Dp], or None)."""
    cfg = scene.cfg
    lo, hi, grid = scene.box_lo, scene.box_hi, scene.grid
    if device_inputs:
        import torch
        lo = torch.from_numpy(np.ascontiguousarray(lo)).cuda()
        hi = torch.from_numpy(np.ascontiguousarray(hi)).cuda()
        grid = torch.from_numpy(np.ascontiguousarray(grid)).cuda()
        if heading is not None:
            heading = torch.from_numpy(np.ascontiguousarray(heading)).cuda()
    return build_roadmap(cfg.dim_kind, lo, hi, grid, cfg.grid_G, cfg.n if n is None else n,
                         scene.sample_seed, cfg.r if r is None else r, scene.x_init, scene.x_goal,
                         T=cfg.T_edge, M=cfg.M if M is None else M, query_id=scene.query_id,
                         heading=heading, stream=stream)


class Workspace:
    """An mpap_workspace: device fronts, plan arena and work lists for searches of
    up to ``total_nodes`` nodes (summed over one batch)."""

    def __init__(self, total_nodes, front_cap=64, max_plans=1 << 24):
        h = C.c_void_p()
        _check(lib().mpap_workspace_create(int(total_nodes), int(front_cap), int(max_plans), C.byref(h)),
               "mpap_workspace_create")
        self.h = h
        self.total_nodes = int(total_nodes)
        self.front_cap = int(front_cap)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.mpap_workspace_free(self.h)
            self.h = None

    def stats(self):
        """mpap_workspace_stats: (largest front, pool entries used) of the last search."""
        mf = C.c_uint32(); pu = C.c_uint64()
        _check(lib().mpap_workspace_stats(self.h, C.byref(mf), C.byref(pu)), "mpap_workspace_stats")
        return mf.value, pu.value

    def fronts(self, index=0, stream=None):
        """Final (cost, h) fronts of query `index` of the last search: (ptr, cost, h)."""
        tot = C.c_uint64()
        lib().mpap_search_fronts(self.h, index, None, None, None, 0, C.byref(tot), _stream(stream))
        n = tot.value
        # V from the last search: ask with a large pointer array
        cost = np.zeros(max(n, 1), np.int64); hh = np.zeros(max(n, 1), np.int64)
        ptr = np.zeros(self.total_nodes + 1, np.uint32)
        _check(lib().mpap_search_fronts(self.h, index, ptr.ctypes.data_as(C.c_void_p),
                                        cost.ctypes.data_as(C.c_void_p), hh.ctypes.data_as(C.c_void_p),
                                        n, C.byref(tot), _stream(stream)), "mpap_search_fronts")
        return ptr, cost[:n], hh[:n]


@dataclass
class SearchResult:
    status: int
    cost: int
    h: int
    path: np.ndarray
    wavefronts: int
    expansions: int
    plans: int


def make_query(beta, lam=0.5, group_width_q=0, max_iters=100000, goal_stop=True, interior=False, wait_us=0,
               own_share=False):
    flags = (0 if goal_stop else MPAP_QUERY_NO_GOAL_STOP) | (MPAP_QUERY_CHECK_INTERIOR if interior else 0) | \
        (MPAP_QUERY_OWN_SHARE if own_share else 0)
    return mpap_query(beta=int(beta), group_width_q=int(group_width_q), lambda_=float(lam),
                      max_iters=int(max_iters), flags=flags, wait_us=int(wait_us))


def _result(r, buf):
    n = r.path_len if r.status == MPAP_OK else 0
    return SearchResult(r.status, r.cost, r.h, buf[:n].copy(), r.wavefronts, r.expansions, r.plans)


def search(ws: Workspace, rm: Roadmap, beta, lam=0.5, group_width_q=0, max_iters=100000,
           goal_stop=True, path_cap=4096, stream=None, interior=False, wait_us=0) -> SearchResult:
    """mpap_search: Alg. 3 Explore for one query."""
    q = make_query(beta, lam, group_width_q, max_iters, goal_stop, interior, wait_us)
    buf = np.zeros(path_cap, np.uint32)
    r = mpap_result(path_cap=path_cap, path=buf.ctypes.data_as(C.POINTER(C.c_uint32)))
    _check(lib().mpap_search(ws.h, rm.h, C.byref(q), C.byref(r), _stream(stream)), "mpap_search")
    return _result(r, buf)


def _result_array(nq, path_cap):
    """mpap_result array (numpy, C layout) whose path pointers tile one
    [nq, path_cap] uint32 buffer (row i receives query i's plan)."""
    bufs = np.zeros((nq, path_cap), np.uint32)
    rs = np.zeros(nq, RESULT_DT)
    rs["path_cap"] = path_cap
    rs["path"] = bufs.__array_interface__["data"][0] + 4 * path_cap * np.arange(nq, dtype=np.uint64)
    return rs, bufs


def search_batch(ws: Workspace, rms, queries, path_cap=4096, stream=None, check=True):
    """mpap_search_batch: independent queries in one lock-step wavefront loop."""
    nq = len(rms)
    hs = (C.c_void_p * nq)(*[rm.h for rm in rms])
    qs = (mpap_query * nq)(*queries)
    rs, bufs = _result_array(nq, path_cap)
    rc = lib().mpap_search_batch(ws.h, hs, qs, nq, _as(rs, mpap_result), _stream(stream))
    if check:
        _check(rc, "mpap_search_batch")
    cols = [rs[k].tolist() for k in ("status", "cost", "h", "path_len", "wavefronts", "expansions", "plans")]
    return [SearchResult(st, c, h, bufs[i, :n].copy() if st == MPAP_OK else bufs[i, :0].copy(), w, e, pl)
            for i, (st, c, h, n, w, e, pl) in enumerate(zip(*cols))]


def make_mc(rollouts, seed, call_id, delta_fx, sigma_fx, shift):
    sig = np.ascontiguousarray(sigma_fx, np.int32); sh = np.ascontiguousarray(shift, np.int32)
    p = mpap_mc_params(rollouts=rollouts, call_id=call_id, seed=seed, delta_fx=int(delta_fx),
                       sigma_fx=sig.ctypes.data_as(C.POINTER(C.c_int32)),
                       shift=sh.ctypes.data_as(C.POINTER(C.c_int32)))
    return p, (sig, sh)


def certify(rm: Roadmap, path, rollouts, seed, call_id, delta_fx, sigma_fx, shift, stream=None):
    """mpap_certify: Monte Carlo rollouts along a plan."""
    p, keep = make_mc(rollouts, seed, call_id, delta_fx, sigma_fx, shift)
    path = np.ascontiguousarray(path, np.uint32)
    out = mpap_cert()
    _check(lib().mpap_certify(rm.h, path.ctypes.data_as(C.c_void_p), path.size, C.byref(p), C.byref(out),
                              _stream(stream)), "mpap_certify")
    return dict(hits_loc=out.hits_loc, hits_coll=out.hits_coll, hits_any=out.hits_any, rollouts=out.rollouts)


def certify_noalloc(rm: Roadmap, path, rollouts, seed, call_id, delta_fx, sigma_fx, shift, stream=None):
    """mpap_certify_noalloc: the same rollouts as certify() with the kernels'
    scratch in a fixed device array inside the library (no device allocation),
    for callers that cannot allocate while running."""
    p, keep = make_mc(rollouts, seed, call_id, delta_fx, sigma_fx, shift)
    path = np.ascontiguousarray(path, np.uint32)
    out = mpap_cert()
    _check(lib().mpap_certify_noalloc(rm.h, path.ctypes.data_as(C.c_void_p), path.size, C.byref(p),
                                      C.byref(out), _stream(stream)), "mpap_certify_noalloc")
    return dict(hits_loc=out.hits_loc, hits_coll=out.hits_coll, hits_any=out.hits_any, rollouts=out.rollouts)


def _mc_array(mcs):
    """mpap_mc_params array (numpy, C layout) for (rollouts, seed, call_id,
    delta_fx, sigma_fx, shift) tuples, plus the arrays it points into."""
    ms = np.zeros(len(mcs), MC_DT)
    keep = [(np.ascontiguousarray(m[4], np.int32), np.ascontiguousarray(m[5], np.int32)) for m in mcs]
    ms["rollouts"] = [m[0] for m in mcs]
    ms["seed"] = [m[1] for m in mcs]
    ms["call_id"] = [m[2] for m in mcs]
    ms["delta_fx"] = [int(m[3]) for m in mcs]
    ms["sigma_fx"] = [k[0].__array_interface__["data"][0] for k in keep]
    ms["shift"] = [k[1].__array_interface__["data"][0] for k in keep]
    return ms, keep


def certify_batch(rms, paths, mcs, stream=None):
    """mpap_certify_batch. mcs: list of (rollouts, seed, call_id, delta_fx, sigma_fx, shift)."""
    n = len(rms)
    hs = (C.c_void_p * n)(*[rm.h for rm in rms])
    arrs = [np.ascontiguousarray(p, np.uint32) if len(p) else np.zeros(1, np.uint32) for p in paths]
    pp = np.array([a.__array_interface__["data"][0] for a in arrs], np.uint64)
    lens = np.array([len(p) for p in paths], np.uint32)
    ms, keep = _mc_array(mcs)
    outs = np.zeros(n, CERT_DT)
    _check(lib().mpap_certify_batch(hs, pp.ctypes.data_as(C.POINTER(C.c_void_p)), lens.ctypes.data_as(C.c_void_p),
                                    _as(ms, mpap_mc_params), n, _as(outs, mpap_cert), _stream(stream)),
           "mpap_certify_batch")
    cols = [outs[k].tolist() for k in ("hits_loc", "hits_coll", "hits_any", "rollouts")]
    return [dict(hits_loc=a, hits_coll=b, hits_any=c, rollouts=d) for a, b, c, d in zip(*cols)]


def certify_vio_batch(rms, paths, mcs, vios, stream=None):
    """mpap_certify_vio_batch: the closed-loop VIO model.  mcs: list of (rollouts,
    seed, call_id, delta_fx); vios: list of (q_a, kp_q16, kv_q16, r_fx)."""
    n = len(rms)
    hs = (C.c_void_p * n)(*[rm.h for rm in rms])
    arrs = [np.ascontiguousarray(p, np.uint32) if len(p) else np.zeros(1, np.uint32) for p in paths]
    pp = np.array([a.__array_interface__["data"][0] for a in arrs], np.uint64)
    lens = np.array([len(p) for p in paths], np.uint32)
    ms = (mpap_mc_params * n)()
    vs = (mpap_vio_params * n)()
    keep = []
    for i, (m, v) in enumerate(zip(mcs, vios)):
        ms[i].rollouts, ms[i].seed, ms[i].call_id, ms[i].delta_fx = int(m[0]), int(m[1]), int(m[2]), int(m[3])
        r = np.ascontiguousarray(v[3], np.int32)
        keep.append(r)
        vs[i].q_a, vs[i].kp_q16, vs[i].kv_q16 = int(v[0]), int(v[1]), int(v[2])
        vs[i].r_fx = r.ctypes.data_as(C.POINTER(C.c_int32))
    outs = (mpap_cert * n)()
    _check(lib().mpap_certify_vio_batch(hs, pp.ctypes.data_as(C.POINTER(C.c_void_p)),
                                        lens.ctypes.data_as(C.c_void_p), ms, vs, n, outs, _stream(stream)),
           "mpap_certify_vio_batch")
    return [dict(hits_loc=o.hits_loc, hits_coll=o.hits_coll, hits_any=o.hits_any, rollouts=o.rollouts)
            for o in outs]


def vio_lqr_gains(q_p, q_w, r):
    """mpap_vio_lqr_gains: (kp_q16, kv_q16) of the VIO model's LQR tracker."""
    kp = C.c_int32(); kv = C.c_int32()
    _check(lib().mpap_vio_lqr_gains(float(q_p), float(q_w), float(r), C.byref(kp), C.byref(kv)),
           "mpap_vio_lqr_gains")
    return kp.value, kv.value


def certify_vio(rm: Roadmap, path, rollouts, seed, call_id, delta_fx, q_a, kp_q16, kv_q16, r_fx, stream=None):
    """One plan under the closed-loop VIO model (a batch of one)."""
    return certify_vio_batch([rm], [path], [(rollouts, seed, call_id, delta_fx)],
                             [(q_a, kp_q16, kv_q16, r_fx)], stream)[0]


# ---------------------------------------------------------------------------
# Candidate plans and the certification surrogate
# ---------------------------------------------------------------------------
MLP_PARAMS = 39554
N_FEATURES = 48


def search_candidates(ws: Workspace, index=0, cap=64, path_cap=1 << 16, stream=None):
    """P_candidates of query `index` of the last search on ws, in solution order:
    dict(cost, h (int64 arrays), paths (list of uint32 arrays), total)."""
    cost = np.zeros(max(cap, 1), np.int64)
    hh = np.zeros(max(cap, 1), np.int64)
    ptr = np.zeros(cap + 1, np.uint32)
    path = np.zeros(max(path_cap, 1), np.uint32)
    n = C.c_uint32()
    tot = C.c_uint32()
    vp = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(lib().mpap_search_candidates(ws.h, index, cap, vp(cost), vp(hh), vp(ptr), vp(path), path_cap,
                                        C.byref(n), C.byref(tot), _stream(stream)), "mpap_search_candidates")
    k = n.value
    paths = [path[ptr[i]:ptr[i + 1]].copy() for i in range(k)]
    return dict(cost=cost[:k].copy(), h=hh[:k].copy(), paths=paths, total=tot.value)


def plan_features(rm: Roadmap, paths, stream=None) -> np.ndarray:
    """mpap_plan_features: [len(paths), 48] float32 features of node sequences on rm."""
    n = len(paths)
    if n == 0:
        return np.zeros((0, N_FEATURES), np.float32)
    ptr = np.zeros(n + 1, np.uint32)
    ptr[1:] = np.cumsum([len(p) for p in paths])
    flat = np.ascontiguousarray(np.concatenate([np.asarray(p, np.uint32) for p in paths]), np.uint32)
    out = np.zeros((n, N_FEATURES), np.float32)
    vp = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(lib().mpap_plan_features(rm.h, n, vp(ptr), vp(flat), vp(out), _stream(stream)), "mpap_plan_features")
    return out


class Mlp:
    """An mpap_mlp: the 48-128-128-128-2 certification surrogate (bf16 tensor-core
    products, fp32 master weights, Adam).  Inputs and outputs are numpy arrays
    (host) or contiguous CUDA tensors (device, float32)."""

    def __init__(self, seed=0, max_batch=4096):
        h = C.c_void_p()
        _check(lib().mpap_mlp_create(int(seed), int(max_batch), C.byref(h)), "mpap_mlp_create")
        self.h = h
        self.max_batch = int(max_batch)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.mpap_mlp_free(self.h)
            self.h = None

    def get_params(self, stream=None) -> np.ndarray:
        out = np.zeros(MLP_PARAMS, np.float32)
        _check(lib().mpap_mlp_get_params(self.h, out.ctypes.data_as(C.c_void_p), _stream(stream)),
               "mpap_mlp_get_params")
        return out

    def set_params(self, params, stream=None):
        p = np.ascontiguousarray(params, np.float32)
        assert p.size == MLP_PARAMS
        _check(lib().mpap_mlp_set_params(self.h, p.ctypes.data_as(C.c_void_p), _stream(stream)),
               "mpap_mlp_set_params")

    def forward(self, x, stream=None):
        xp, xk, dev = _ptr(x, np.float32)
        n = int(x.shape[0])
        if dev:
            import torch
            out = torch.empty((n, 2), dtype=torch.float32, device=x.device)
            op = C.c_void_p(out.data_ptr())
        else:
            out = np.zeros((n, 2), np.float32)
            op = out.ctypes.data_as(C.c_void_p)
        _check(lib().mpap_mlp_forward(self.h, xp, n, op, 1 if dev else 0, _stream(stream)), "mpap_mlp_forward")
        return out

    def train_step(self, x, y, lr=1e-3, apply=True, want_grads=False, stream=None):
        """One step; returns (loss, grads or None)."""
        xp, xk, dev = _ptr(x, np.float32)
        yp, yk, _ = _ptr(y, np.float32)
        n = int(x.shape[0])
        loss = C.c_float()
        g = None
        gp = None
        if want_grads:
            if dev:
                import torch
                g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=x.device)
                gp = C.c_void_p(g.data_ptr())
            else:
                g = np.zeros(MLP_PARAMS, np.float32)
                gp = g.ctypes.data_as(C.c_void_p)
        _check(lib().mpap_mlp_train_step(self.h, xp, yp, n, float(lr), 1 if apply else 0, C.byref(loss), gp,
                                         1 if dev else 0, _stream(stream)), "mpap_mlp_train_step")
        return loss.value, g


# ---------------------------------------------------------------------------
# Learned error-rate heuristic (Sec. 5.1)
# ---------------------------------------------------------------------------
ERRNET_PARAMS = 154


class ErrNet:
    """An mpap_errnet: the 7-8-8-2 error-rate network (mean and standard
    deviation of the Gaussian rate of the position error), trained by maximum
    likelihood on the GPU.  Arrays are numpy (host) or contiguous CUDA tensors."""

    def __init__(self, seed=0, max_batch=1 << 16):
        h = C.c_void_p()
        _check(lib().mpap_errnet_create(int(seed), int(max_batch), C.byref(h)), "mpap_errnet_create")
        self.h = h
        self.max_batch = int(max_batch)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.mpap_errnet_free(self.h)
            self.h = None

    def get_params(self, stream=None) -> np.ndarray:
        out = np.zeros(ERRNET_PARAMS, np.float32)
        _check(lib().mpap_errnet_get_params(self.h, out.ctypes.data_as(C.c_void_p), _stream(stream)),
               "mpap_errnet_get_params")
        return out

    def set_params(self, params, stream=None):
        p = np.ascontiguousarray(params, np.float32)
        assert p.size == ERRNET_PARAMS
        _check(lib().mpap_errnet_set_params(self.h, p.ctypes.data_as(C.c_void_p), _stream(stream)),
               "mpap_errnet_set_params")

    def forward(self, x, stream=None):
        """[n, 2] (mean, std) of inputs x [n, 7]."""
        xp, xk, dev = _ptr(x, np.float32)
        n = int(x.shape[0])
        if dev:
            import torch
            out = torch.empty((n, 2), dtype=torch.float32, device=x.device)
            op = C.c_void_p(out.data_ptr())
        else:
            out = np.zeros((n, 2), np.float32)
            op = out.ctypes.data_as(C.c_void_p)
        _check(lib().mpap_errnet_forward(self.h, xp, n, op, 1 if dev else 0, _stream(stream)), "mpap_errnet_forward")
        return out

    def train_step(self, x, r, lr=1e-3, apply=True, want_grads=False, stream=None):
        """One maximum-likelihood step on rates r [n]; returns (loss, grads or None)."""
        xp, xk, dev = _ptr(x, np.float32)
        rp, rk, _ = _ptr(r, np.float32)
        n = int(x.shape[0])
        loss = C.c_float()
        g, gp = None, None
        if want_grads:
            if dev:
                import torch
                g = torch.empty(ERRNET_PARAMS, dtype=torch.float32, device=x.device)
                gp = C.c_void_p(g.data_ptr())
            else:
                g = np.zeros(ERRNET_PARAMS, np.float32)
                gp = g.ctypes.data_as(C.c_void_p)
        _check(lib().mpap_errnet_train_step(self.h, xp, rp, n, float(lr), 1 if apply else 0, C.byref(loss), gp,
                                            1 if dev else 0, _stream(stream)), "mpap_errnet_train_step")
        return loss.value, g


def errmap_query(map_state, map_val, q, k=8, w=(1.0, 1.0, 1.0), stream=None):
    """mpap_errmap_query: (mean, std) [Q, 2] at query states q [Q, 7] from the
    mapped states [N, 7] and their values [N, 2] (host or device arrays)."""
    sp, sk, dev = _ptr(map_state, np.float32)
    vp, vk, _ = _ptr(map_val, np.float32)
    qp, qk, _ = _ptr(q, np.float32)
    ww = np.ascontiguousarray(w, np.float32)
    nq = int(q.shape[0])
    if dev:
        import torch
        out = torch.empty((nq, 2), dtype=torch.float32, device=q.device)
        op = C.c_void_p(out.data_ptr())
    else:
        out = np.zeros((nq, 2), np.float32)
        op = out.ctypes.data_as(C.c_void_p)
    _check(lib().mpap_errmap_query(sp, vp, int(map_state.shape[0]), qp, nq, int(k), ww.ctypes.data_as(C.c_void_p),
                                   op, 1 if dev else 0, _stream(stream)), "mpap_errmap_query")
    return out


def errmap_levels(map_state, map_val, dim_kind, grid_G, vel=(0.0, 0.0, 0.0), yaw=0.0, mu_ref=0.02, k=8,
                  w=(1.0, 1.0, 1.0), n_f=12, K=24, stream=None):
    """mpap_errmap_levels: uint8 quality levels [G^Dp] of the mapped mean rate at
    the grid's cell centres (host arrays)."""
    sp, sk, dev = _ptr(map_state, np.float32)
    vp, vk, _ = _ptr(map_val, np.float32)
    ww = np.ascontiguousarray(w, np.float32)
    vv = np.ascontiguousarray(vel, np.float32)
    cells = grid_G ** (2 if dim_kind == 2 else 3)     # 2: the unit square, else the unit cube
    if dev:
        import torch
        out = torch.empty(cells, dtype=torch.uint8, device=map_state.device)
        op = C.c_void_p(out.data_ptr())
    else:
        out = np.zeros(cells, np.uint8)
        op = out.ctypes.data_as(C.c_void_p)
    _check(lib().mpap_errmap_levels(sp, vp, int(map_state.shape[0]), int(k), ww.ctypes.data_as(C.c_void_p),
                                    int(dim_kind), int(grid_G), vv.ctypes.data_as(C.c_void_p), float(yaw),
                                    float(mu_ref), int(n_f), int(K), op, 1 if dev else 0, _stream(stream)),
           "mpap_errmap_levels")
    return out


# ---------------------------------------------------------------------------
# Launch-shape tuning
# ---------------------------------------------------------------------------
def _tuning_dict(t):
    return dict(edge_warps=t.edge_warps, wave_blocks_per_sm=t.wave_blocks_per_sm,
                plan_lanes_from=t.plan_lanes_from, front_cap=t.front_cap, grid_merge_from=t.grid_merge_from)


def tuning_get(dim_kind, V):
    t = mpap_tuning()
    _check(lib().mpap_tuning_get(int(dim_kind), int(V), C.byref(t)), "mpap_tuning_get")
    return _tuning_dict(t)


def tuning_set(dim_kind, V, edge_warps=8, wave_blocks_per_sm=8, plan_lanes_from=8, front_cap=64,
               grid_merge_from=2048):
    t = mpap_tuning(edge_warps, wave_blocks_per_sm, plan_lanes_from, front_cap, grid_merge_from)
    _check(lib().mpap_tuning_set(int(dim_kind), int(V), C.byref(t)), "mpap_tuning_set")


def tuning_clear():
    lib().mpap_tuning_clear()


def tuning_export():
    """[(dim_kind, bucket, tuning dict)] of the stored entries (bucket = floor(log2 V))."""
    n = C.c_uint32()
    lib().mpap_tuning_export(0, None, None, None, C.byref(n))
    k = n.value
    dims = np.zeros(max(k, 1), np.int32)
    bks = np.zeros(max(k, 1), np.uint32)
    ts = (mpap_tuning * max(k, 1))()
    _check(lib().mpap_tuning_export(k, dims.ctypes.data_as(C.c_void_p), bks.ctypes.data_as(C.c_void_p),
                                    C.cast(ts, C.c_void_p), C.byref(n)), "mpap_tuning_export")
    return [(int(dims[i]), int(bks[i]), _tuning_dict(ts[i])) for i in range(k)]


def autotune_build(specs, rms=None, reps=2, stream=None):
    """mpap_autotune_build on a batch of build specs; returns (tuning, ms per build, roadmaps)."""
    n = len(specs)
    scenes, params, keep = _batch_structs(specs)
    rms = list(rms) if rms is not None else [None] * n
    hs = (C.c_void_p * n)(*[rm.h.value if rm is not None and rm.h else None for rm in rms])
    t = mpap_tuning()
    ms = C.c_double()
    rc = lib().mpap_autotune_build(n, _as(scenes, mpap_scene), _as(params, mpap_roadmap_params), hs, int(reps),
                                   C.byref(t), C.byref(ms), _stream(stream))
    out = _adopt(specs, rms, hs)
    _check(rc, "mpap_autotune_build")
    return _tuning_dict(t), ms.value, out


def autotune_search(ws, rms, queries, reps=2, stream=None):
    """mpap_autotune_search on a batch of queries; returns (tuning, ms per search)."""
    nq = len(rms)
    hs = (C.c_void_p * nq)(*[rm.h for rm in rms])
    qs = (mpap_query * nq)(*queries)
    t = mpap_tuning()
    ms = C.c_double()
    _check(lib().mpap_autotune_search(ws.h, hs, qs, nq, int(reps), C.byref(t), C.byref(ms), _stream(stream)),
           "mpap_autotune_search")
    return _tuning_dict(t), ms.value


def search_candidates_batch(ws: Workspace, nq, cap=64, path_cap=1 << 14, stream=None):
    """mpap_search_candidates_batch: candidates of queries 0..nq-1 of the last search
    (one launch); a list of dicts as search_candidates, None for unsolved queries."""
    cost = np.zeros((max(nq, 1), cap), np.int64)
    hh = np.zeros((max(nq, 1), cap), np.int64)
    ptr = np.zeros((max(nq, 1), cap + 1), np.uint32)
    path = np.zeros((max(nq, 1), path_cap), np.uint32)
    n = np.zeros(max(nq, 1), np.uint32)
    tot = np.zeros(max(nq, 1), np.uint32)
    vp = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(lib().mpap_search_candidates_batch(ws.h, nq, cap, vp(cost), vp(hh), vp(ptr), vp(path), path_cap,
                                              vp(n), vp(tot), _stream(stream)), "mpap_search_candidates_batch")
    out = []
    for i in range(nq):
        k = int(n[i])
        if k == 0:
            out.append(None)
            continue
        out.append(dict(cost=cost[i, :k].copy(), h=hh[i, :k].copy(), total=int(tot[i]),
                        paths=[path[i, ptr[i, j]:ptr[i, j + 1]].copy() for j in range(k)]))
    return out


def plan_features_batch(rms, paths_per_rm, stream=None):
    """mpap_plan_features_batch: features of the plans of several roadmaps in one
    launch; returns one [k_r, 48] array per roadmap."""
    n_rm = len(rms)
    counts = [len(p) for p in paths_per_rm]
    plan_ptr = np.zeros(n_rm + 1, np.uint32)
    plan_ptr[1:] = np.cumsum(counts)
    flat_paths = [np.asarray(p, np.uint32) for ps in paths_per_rm for p in ps]
    n = len(flat_paths)
    if n == 0:
        return [np.zeros((0, N_FEATURES), np.float32) for _ in rms]
    path_ptr = np.zeros(n + 1, np.uint32)
    path_ptr[1:] = np.cumsum([len(p) for p in flat_paths])
    flat = np.ascontiguousarray(np.concatenate(flat_paths), np.uint32)
    feat = np.zeros((n, N_FEATURES), np.float32)
    hs = (C.c_void_p * n_rm)(*[rm.h for rm in rms])
    vp = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(lib().mpap_plan_features_batch(hs, n_rm, vp(plan_ptr), vp(path_ptr), vp(flat), vp(feat),
                                          _stream(stream)), "mpap_plan_features_batch")
    return [feat[plan_ptr[r]:plan_ptr[r + 1]] for r in range(n_rm)]
