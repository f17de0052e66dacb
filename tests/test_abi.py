"""The C ABI library loads and exports every symbol include/numa.h declares (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import paper_1702_04316_gb300 as p
    if not os.path.exists(p.LIB_PATH):
        from paper_1702_04316_gb300 import build
        build.build()
    return p


def _declared():
    src = open(os.path.join(ROOT, "include", "numa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(numa_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(pkg):
    L = pkg.lib()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert sorted(pkg.EXPORTS) == names


def test_invalid_arguments_are_rejected_before_any_device_call(pkg):
    L = pkg.lib()
    h = ctypes.c_void_p()
    bad = [pkg.MeshDesc(0, 4, 4, 1e4, 1e4, 1e4, 300.0, 0.0),
           pkg.MeshDesc(4, 4, 4, -1.0, 1e4, 1e4, 300.0, 0.0),
           pkg.MeshDesc(4, 4, 4, 1e4, 1e4, 1e4, 300.0, -1.0)]
    for d in bad:
        assert L.numa_init(ctypes.byref(d), 4, 1.0, None, ctypes.byref(h)) == 1
        assert not h.value
    ok = pkg.MeshDesc(4, 4, 4, 1e4, 1e4, 1e4, 300.0, 0.0)
    assert L.numa_init(ctypes.byref(ok), 0, 1.0, None, ctypes.byref(h)) == 1    # N < 1
    assert L.numa_init(ctypes.byref(ok), 9, 1.0, None, ctypes.byref(h)) == 1    # N > 8
    assert L.numa_init(ctypes.byref(ok), 4, -1.0, None, ctypes.byref(h)) == 1   # dt < 0
    assert L.numa_init(ctypes.byref(ok), 4, 1.0, None, None) == 1               # out NULL
    big = pkg.MeshDesc(1 << 12, 1 << 12, 1 << 8, 1e4, 1e4, 1e4, 300.0, 0.0)
    assert L.numa_init(ctypes.byref(big), 8, 1.0, None, ctypes.byref(h)) == 1   # int32 ids overflow


def test_host_tableaux_match_the_oracle(pkg):
    from oracle import ark2, rk35
    a, at, b = pkg.ark2_tableau()
    oa, oat, ob, _ = ark2.tableau()
    np.testing.assert_allclose(a, oa, rtol=0, atol=1e-15)
    np.testing.assert_allclose(at, oat, rtol=0, atol=1e-15)
    np.testing.assert_allclose(b, ob, rtol=0, atol=1e-15)
    al, be = pkg.rk35_coefficients()
    np.testing.assert_array_equal(al, rk35.ALPHA)
    np.testing.assert_array_equal(be, rk35.BETA)


def test_ark3_tableau_matches_the_oracle_bitwise():
    """The host ARK3 tableau (each coefficient one correctly rounded division of the
    published rationals) equals the oracle's float tableau bit for bit."""
    import numpy as np
    import paper_1702_04316_gb300 as pkg
    from oracle import ark3
    a, at, b = pkg.ark3_tableau()
    A, AT, B, _ = ark3.tableau()
    assert np.array_equal(a, A) and np.array_equal(at, AT) and np.array_equal(b, B)


@pytest.mark.parametrize("scheme", ["ark3", "ark4", "ark5"])
def test_ark_tableaux_match_the_oracle_bitwise(scheme):
    """numa_ark_tableau: every coefficient of ARK3 - ARK5 (each a correctly rounded division
    of a rational) equals the oracle's float tableau bit for bit; ARK2 to rounding."""
    import numpy as np
    import paper_1702_04316_gb300 as pkg
    from oracle import ark2
    a, at, b = pkg.ark_tableau(scheme)
    A, AT, B, _ = ark2.scheme_tableau(scheme)
    assert a.shape == A.shape
    assert np.array_equal(a, A) and np.array_equal(at, AT) and np.array_equal(b, B)
    a2, at2, b2 = pkg.ark_tableau("ark2")
    np.testing.assert_allclose(at2, ark2.tableau()[1], rtol=0, atol=1e-15)


def test_partition_plan_rejects_bad_grids_without_a_gpu(pkg):
    """numa_part_plan is host only: bad grids are rejected, good ones planned, no device."""
    L = pkg.lib()
    g = pkg.MeshDesc(8, 6, 2, 8e3, 6e3, 4e3, 300.0, 0.0)
    info = pkg.PartInfo()
    for px, py, rank in [(0, 1, 0), (2, 2, 4), (2, 2, -1), (5, 1, 0), (1, 4, 0)]:
        d = pkg.PartDesc(px, py, rank)       # (5, 1) and (1, 4): rectangles narrower than 2
        assert L.numa_part_plan(ctypes.byref(g), 3, ctypes.byref(d), ctypes.byref(info)) == 1
    d = pkg.PartDesc(2, 3, 5)
    assert L.numa_part_plan(ctypes.byref(g), 3, ctypes.byref(d), ctypes.byref(info)) == 0
    assert (info.ex0, info.ex1, info.ey0, info.ey1) == (4, 8, 4, 6)
    assert (info.wx0, info.wx1, info.wy0, info.wy1) == (3, 8, 3, 6)
    assert info.window.nex == 5 and info.window.ney == 3 and info.window.nez == 2
    assert info.window.Lx / info.window.nex == 8e3 / 8      # the element size, bit for bit
    assert info.nneigh == 3 and list(info.neigh[:3]) == [2, 3, 4]
    one = pkg.PartDesc(1, 1, 0)
    assert L.numa_part_plan(ctypes.byref(g), 3, ctypes.byref(one), ctypes.byref(info)) == 0
    assert info.nneigh == 0 and (info.own_x1, info.own_y1) == (25, 19)
    assert L.numa_part_columns(ctypes.byref(g), 3, ctypes.byref(d), 3, None, None) == 1
