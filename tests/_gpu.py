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
