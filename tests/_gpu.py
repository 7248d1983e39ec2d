"""Shared helpers for the GPU parity tests."""
import numpy as np

import scenegen

BIG = 1 << 62


def gpu_roadmap(mp, scene, n=None, r=None, M=None, device_inputs=False):
    return mp.build_roadmap_for_scene(scene, n=n, r=r, M=M, device_inputs=device_inputs)


def assert_same_graph(gpu, g):
    assert gpu["V"] == g.V
    np.testing.assert_array_equal(gpu["x"], g.x)
    np.testing.assert_array_equal(gpu["is_goal"], g.is_goal)
    np.testing.assert_array_equal(gpu["row_ptr"], g.row_ptr)
    np.testing.assert_array_equal(gpu["dst"], g.dst)
    np.testing.assert_array_equal(gpu["cost_q"], g.cost_q)
    np.testing.assert_array_equal(gpu["S"], g.S)
    np.testing.assert_array_equal(gpu["C"], g.C)


def assert_same_search(res_gpu, res_orc, ws=None, index=0, fronts=True):
    assert res_gpu.status == res_orc.status
    if res_orc.status == 0:
        assert (res_gpu.cost, res_gpu.h) == (res_orc.cost, res_orc.h)
        np.testing.assert_array_equal(res_gpu.path, res_orc.path)
    if res_orc.status >= 0:
        assert res_gpu.wavefronts == res_orc.wavefronts
        assert res_gpu.expansions == res_orc.expansions
    if fronts and ws is not None and res_orc.status >= 0:
        ptr, cost, h = ws.fronts(index)
        V = len(res_orc.front_ptr) - 1
        np.testing.assert_array_equal(ptr[:V + 1], res_orc.front_ptr)
        np.testing.assert_array_equal(cost, res_orc.front_cost)
        np.testing.assert_array_equal(h, res_orc.front_h)


def scene_beta(orc, rm_orc):
    return orc.beta_percentile(rm_orc)


def assert_reverse_is_transpose(rm):
    """The reverse CSR on the device (in-edges, read by the search's pull step)
    holds exactly one record per forward edge, with its fields: the transpose of
    the forward CSR."""
    f = rm.export()
    Smax, Cmax = rm.peaks()
    r = rm.export_reverse()
    V, E = f["V"], f["E"]
    assert r["E"] == E
    src = np.repeat(np.arange(V, dtype=np.uint32), np.diff(f["row_ptr"]).astype(np.int64))
    dst = f["dst"]
    order = np.lexsort((src, dst))
    want_ptr = np.zeros(V + 1, np.uint32)
    np.cumsum(np.bincount(dst, minlength=V), out=want_ptr[1:])
    np.testing.assert_array_equal(r["rev_ptr"], want_ptr)
    np.testing.assert_array_equal(r["src"], src[order])
    for k, a in (("cost_q", f["cost_q"]), ("S", f["S"]), ("C", f["C"]), ("Smax", Smax), ("Cmax", Cmax)):
        np.testing.assert_array_equal(r[k], a[order], err_msg=k)
