"""CPU checks of the C-ABI boundary: the library builds, loads and exports every
symbol that include/mpjacobi.h declares.  No compute call is made (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mpj_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2211_03339_gb300 import build
    build.build()
    import paper_2211_03339_gb300 as m
    return m.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("mpj_syevj_mp", "mpj_syevj_plain", "mpj_gesvj_mp", "mpj_gesvj_plain",
                 "mpj_mgs", "mpj_congruence", "mpj_sweeps", "mpj_stage1_syevj32"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), name


def test_binding_lists_match_header():
    import paper_2211_03339_gb300 as m
    assert set(m.EXPORTS) <= _declared()


def test_host_only_entry_points(lib):
    assert lib.mpj_version().startswith(b"mpjacobi")
    assert lib.mpj_status_string(0) == b"success"
    assert lib.mpj_status_string(3).startswith(b"not converged")
    assert lib.mpj_syevj_workspace_bytes(0) == 0
    assert lib.mpj_syevj_workspace_bytes(4096) > 2 * 4096 * 4096 * 8
    assert lib.mpj_gesvj_workspace_bytes(10, 20) == 0        # m < n rejected
    assert lib.mpj_gesvj_workspace_bytes(4096, 2048) > 4096 * 2048 * 8


def test_bad_arguments_rejected_before_any_device_work(lib):
    import paper_2211_03339_gb300 as m
    st = m.Stats()
    p = ctypes.c_void_p(0)
    # NULL pointers and n < 1 are refused on the host with MPJ_BAD_ARG
    rc = lib.mpj_syevj_mp(p, 8, 8, p, p, 8, 1e-12, None, ctypes.byref(st), p, 0, p)
    assert rc == 1
    rc = lib.mpj_syevj_plain(ctypes.c_void_p(16), 0, 1, ctypes.c_void_p(16), ctypes.c_void_p(16),
                             1, 1e-12, None, None, p, 0, p)
    assert rc == 1
    rc = lib.mpj_gesvj_mp(ctypes.c_void_p(16), 4, 8, 4, ctypes.c_void_p(16), ctypes.c_void_p(16), 4,
                          ctypes.c_void_p(16), 8, 1e-12, None, None, p, 0, p)
    assert rc == 1   # m < n
    rc = lib.mpj_syevj_mp(ctypes.c_void_p(16), 8, 4, ctypes.c_void_p(16), ctypes.c_void_p(16), 8,
                          1e-12, None, None, p, 0, p)
    assert rc == 1   # lda < n
    rc = lib.mpj_syevj_mp(ctypes.c_void_p(16), 8, 8, ctypes.c_void_p(16), ctypes.c_void_p(16), 8,
                          -1.0, None, None, p, 0, p)
    assert rc == 1   # tol <= 0


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2211_03339_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "oracle.c" not in txt, f


def test_profile_counters_host_only(lib):
    """The diagnostics are host state: every class has a name, the counters read
    zero after a reset, and an out-of-range class or a missing output is rejected.
    The byte count of the FP32 tile pass is a class of its own."""
    import paper_2211_03339_gb300 as m
    lib.mpj_profile_reset()
    names = [lib.mpj_profile_name(k).decode() for k in range(lib.mpj_profile_classes())]
    assert len(set(names)) == len(names) and all(names)
    assert "tile_f32" in names and "solve2_f32" in names
    assert all(v == 0.0 for v in m.profile_units().values())
    assert all(v == (0, 0.0) for v in m.profile_read().values())
    v = ctypes.c_double(1.0)
    assert lib.mpj_profile_units(lib.mpj_profile_classes(), ctypes.byref(v)) != 0
    assert lib.mpj_profile_units(-1, ctypes.byref(v)) != 0
    assert lib.mpj_profile_units(0, None) != 0
