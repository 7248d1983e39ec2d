"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares (no GPU needed: no compute call is made)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(mpap_[a-z0-9_]+)\s*\(",
                            txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1705_02408_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for n in ["mpap_build_roadmap", "mpap_search", "mpap_certify", "mpap_search_batch"]:
        assert n in names


def test_library_exports_all_declared(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    import paper_1705_02408_gb300 as mp
    assert sorted(mp.EXPORTS) == _declared()
    L = mp.lib()
    assert L.mpap_status_string(-2).decode() == "capacity exceeded"


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1705_02408_gb300 as mp
    monkeypatch.setattr(mp, "_lib", None)
    monkeypatch.setattr(mp, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        mp.lib()


def test_host_side_argument_checks(libpath):
    """Invalid arguments are rejected on the host before any device work."""
    import numpy as np
    import paper_1705_02408_gb300 as mp
    with pytest.raises(mp.MpapError) as e:
        mp.build_roadmap(4, np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(4, np.uint8), 2, 10, 1, 0.1,
                         np.zeros(6), np.zeros(6))
    assert e.value.status == mp.MPAP_ERR_INVALID_ARG
    with pytest.raises(mp.MpapError) as e:
        mp.build_roadmap(2, np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(9, np.uint8), 3, 10, 1, 0.1,
                         np.zeros(6), np.zeros(6))
    assert e.value.status == mp.MPAP_ERR_INVALID_ARG
    with pytest.raises(mp.MpapError) as e:
        mp.roadmap_from_csr([0, 1, 1], [5], [1], [0], [0], [0, 1])
    assert e.value.status == mp.MPAP_ERR_INVALID_ARG
    with pytest.raises(mp.MpapError) as e:
        mp.Workspace(0)
    assert e.value.status == mp.MPAP_ERR_INVALID_ARG


def test_feature_levels_argument_checks(libpath):
    """Invalid sizes are rejected on the host before any device work."""
    import numpy as np
    import paper_1705_02408_gb300 as mp
    nob = np.zeros((0, 3), np.float32)
    f = np.zeros((4, 3), np.float32)
    for kw in (dict(grid_G=6), dict(grid_G=2048), dict(K=256), dict(range_=-1.0), dict(dim_kind=4),
               dict(headings=np.zeros((0, 2), np.float32))):
        args = dict(dim_kind=2, box_lo=nob, box_hi=nob, features=f, grid_G=4)
        args.update(kw)
        with pytest.raises(mp.MpapError) as e:
            mp.feature_levels(**args)
        assert e.value.status == mp.MPAP_ERR_INVALID_ARG


def test_roadmap_update_argument_checks(libpath):
    import paper_1705_02408_gb300 as mp
    L = mp.lib()
    assert L.mpap_roadmap_update(None, 0, None, None, None, 0, None) == mp.MPAP_ERR_INVALID_ARG


def test_new_entry_points_argument_checks(libpath):
    """Null handles and arrays of the workspace statistics, yaw export and VIO
    certification are rejected on the host before any device work."""
    import ctypes as C
    import paper_1705_02408_gb300 as mp
    L = mp.lib()
    mf, pu = C.c_uint32(), C.c_uint64()
    assert L.mpap_workspace_stats(None, C.byref(mf), C.byref(pu)) == mp.MPAP_ERR_INVALID_ARG
    assert L.mpap_roadmap_export_yaw(None, None, None) == mp.MPAP_ERR_INVALID_ARG
    out = mp.mpap_cert()
    assert L.mpap_certify_vio_batch(None, None, None, None, None, 1, C.byref(out), None) == mp.MPAP_ERR_INVALID_ARG
    assert L.mpap_certify_vio_batch(None, None, None, None, None, 0, None, None) == mp.MPAP_OK
    kp, kv = C.c_int32(), C.c_int32()
    assert L.mpap_vio_lqr_gains(1.0, 1.0, 1.0, None, C.byref(kv)) == mp.MPAP_ERR_INVALID_ARG
    assert L.mpap_vio_lqr_gains(1.0, 1.0, 1.0, C.byref(kp), C.byref(kv)) == mp.MPAP_OK
    assert kp.value > 0 and kv.value > 0
