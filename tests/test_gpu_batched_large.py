"""A batched build and lock-step search of full-size roadmaps of all three
dimensions -- a 16k-sample 2D roadmap (Pareto fronts of hundreds of plans), a
32k-sample 3D roadmap and a 32k-sample 6D roadmap -- against the oracle: every
CSR array, every node's final front, the solutions, the counters and the
certification counts, bit-exact.  The perception bounds are percentiles of the
oracle's straight-line heuristic chosen so that the oracle's own search finishes
in seconds (its fronts are kept in plain lists)."""
import numpy as np
import pytest

import scenegen
from _gpu import assert_same_graph, assert_same_search

pytestmark = pytest.mark.gpu

CASES = [(scenegen.DIM_2D, 16000, 1, 45.0), (scenegen.DIM_3D, 32000, 2, 30.0), (scenegen.DIM_DI6, 32000, 3, 60.0)]


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    return m


def test_large_mixed_batch_matches_oracle(mp, orc):
    scs = [scenegen.make_scene(scenegen.scaled_config(d, n), s, query_id=s) for d, n, s, _ in CASES]
    rms = mp.build_roadmaps([mp.scene_spec(sc) for sc in scs])
    ros = [orc.build_roadmap(sc) for sc in scs]
    for rg, ro in zip(rms, ros):
        assert_same_graph(rg.export(), ro.graph())
    betas = [orc.beta_percentile(ro, pct) for ro, (_, _, _, pct) in zip(ros, CASES)]
    ws = mp.Workspace(sum(rg.V for rg in rms), front_cap=1024, max_plans=1 << 24)
    res = mp.search_batch(ws, rms, [mp.make_query(b, 0.5) for b in betas])
    for i, (sc, ro, b) in enumerate(zip(scs, ros, betas)):
        a = orc.explore(ro, b, orc.group_width(0.5, sc.cfg.r))
        assert a.status == 0
        assert_same_search(res[i], a, ws, index=i)
    mcs = [(1024, sc.mc_seed, 1, sc.delta_fx, sc.sigma_fx, sc.shift) for sc in scs]
    got = mp.certify_batch(rms, [r.path for r in res], mcs)
    for ro, r, m, g in zip(ros, res, mcs, got):
        assert g == orc.certify(ro, r.path, *m)
