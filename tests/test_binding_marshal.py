"""Host-side argument marshalling of the Python binding (no GPU): the batch calls
fill numpy arrays with the C structs' layout column by column; every struct they
produce must be byte-identical to the one the per-struct ctypes constructors
build, and the result/path pointers must tile one path buffer."""
import ctypes as C

import numpy as np

import scenegen
import paper_1705_02408_gb300 as mp


def _specs():
    out = []
    for name, seed in (("2d", 1), ("3d", 2), ("6d", 3), ("6d", 4)):
        sc = scenegen.make_scene(name, seed, query_id=seed)
        sp = mp.scene_spec(sc)
        sp["goal_radius"] = 0.05 + 0.01 * seed
        out.append(sp)
    # an empty box list (nb = 0 gives null box pointers)
    sp = dict(out[0])
    sp["box_lo"] = np.zeros(0, np.float32)
    sp["box_hi"] = np.zeros(0, np.float32)
    out.append(sp)
    return out


def test_struct_layouts_match_ctypes():
    for dt, cls in ((mp.SCENE_DT, mp.mpap_scene), (mp.PARAMS_DT, mp.mpap_roadmap_params),
                    (mp.QUERY_DT, mp.mpap_query), (mp.RESULT_DT, mp.mpap_result),
                    (mp.MC_DT, mp.mpap_mc_params), (mp.CERT_DT, mp.mpap_cert)):
        assert dt.itemsize == C.sizeof(cls)
        for name, _ in cls._fields_:
            assert dt.fields[name][1] == getattr(cls, name).offset, (cls.__name__, name)


def test_batch_structs_bytes_equal_ctypes_constructors():
    specs = _specs()
    scenes, params, keep = mp._batch_structs(specs)
    for i, sp in enumerate(specs):
        s_old, _ = mp.make_scene_struct(sp["dim_kind"], sp["box_lo"], sp["box_hi"], sp["grid"], sp["grid_G"],
                                        sp.get("n_f", 12), sp.get("K", 24))
        p_old = mp._params(sp["n"], sp["seed"], sp["r"], sp["x_init"], sp["x_goal"], sp["goal_radius"],
                           sp["T"], sp["M"], sp["query_id"])
        assert scenes[i].tobytes() == bytes(s_old), i
        assert params[i].tobytes() == bytes(p_old), i
    assert scenes[-1]["nb"] == 0 and scenes[-1]["box_lo"] == 0 and scenes[-1]["box_hi"] == 0


def test_mc_array_equals_make_mc():
    mcs = []
    for seed in (5, 6, 7):
        sc = scenegen.make_scene("6d", seed, query_id=seed)
        mcs.append((4096 + seed, sc.mc_seed, 7 * seed, sc.delta_fx, sc.sigma_fx, sc.shift))
    ms, keep = mp._mc_array(mcs)
    for i, m in enumerate(mcs):
        ref, _ = mp.make_mc(*m)
        assert ms[i].tobytes() == bytes(ref), i


def test_result_array_tiles_one_path_buffer():
    rs, bufs = mp._result_array(5, 37)
    base = bufs.__array_interface__["data"][0]
    for i in range(5):
        r = mp.mpap_result.from_buffer_copy(rs[i].tobytes())
        assert r.path_cap == 37 and r.status == 0 and r.path_len == 0
        assert C.cast(r.path, C.c_void_p).value == base + 4 * 37 * i
