"""The C-ABI library builds, loads without a GPU and exports every symbol the header declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "swense.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(swense_[a-z_0-9]+)\s*\(",
                                 text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2005_12716_gb300 import build
    build.build()
    from paper_2005_12716_gb300 import _swense
    return _swense.load()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("swense_fields_on_grid", "swense_interp", "swense_fv_divergence",
                 "swense_strerror", "swense_last_error", "swense_release"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2005_12716_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(swense_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        getattr(lib, n)


def test_binding_names_match_header(lib):
    from paper_2005_12716_gb300 import _swense
    assert set(_swense.exported_symbols()) == set(_declared())


def test_host_side_calls_without_gpu(lib):
    from paper_2005_12716_gb300 import _swense
    assert _swense.swense_version() == 100
    assert _swense.swense_strerror(-3) == "SWENSE_ERR_LEVELS"
    assert _swense.swense_strerror(0) == "SWENSE_OK"


def test_argument_validation_launches_nothing(lib):
    """Invalid arguments are rejected on the host before any CUDA call."""
    import ctypes
    import numpy as np
    from paper_2005_12716_gb300 import _swense as S
    z = np.array([-1, -0.5, 0.0, 0.1], np.float32)
    desc = S.make_grid_desc(9, z)          # pad_n must lie in 1..8
    m = S.swense_modes(8, 1, 1.0, 1.0, 0.0, 1, 16, 16, 16, None, 0.0)
    st = lib.swense_fields_on_grid(ctypes.byref(m), 1, None, ctypes.byref(desc), 16, 16, None)
    assert st == -1 and b"pad_n" in lib.swense_last_error()
    desc0 = S.make_grid_desc(0, z)
    assert lib.swense_fields_on_grid(ctypes.byref(m), 1, None, ctypes.byref(desc0), 16, 16, None) == -1
    # a padding factor that is not a power of two needs the workspace: the allocation-free entry
    # point and the autotuner decline it before any CUDA call
    desc3 = S.make_grid_desc(3, z)
    assert lib.swense_fields_on_grid_noalloc(ctypes.byref(m), 1, None, ctypes.byref(desc3), 16, 16, None) == -7
    lpc, chunk, rv = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
    assert lib.swense_autotune_grid(ctypes.byref(m), 1, None, ctypes.byref(desc3), 16, 16, ctypes.byref(lpc),
                                    ctypes.byref(chunk), ctypes.byref(rv), None) == -7
    desc = S.make_grid_desc(1, z[::-1].copy())
    st = lib.swense_fields_on_grid(ctypes.byref(m), 1, None, ctypes.byref(desc), 16, 16, None)
    assert st == -3
    m2 = S.swense_modes(12, 1, 1.0, 1.0, 0.0, 1, 16, 16, 16, None, 0.0)
    st = lib.swense_fields_on_grid(ctypes.byref(m2), 1, None, ctypes.byref(S.make_grid_desc(1, z)),
                                   16, 16, None)
    assert st == -2
    g = S.make_grid(16, 16, 16, 1, 4, 1, 1.0, 1.0, z, [0.0])
    st = lib.swense_interp(ctypes.byref(g), 0.0, 16, 10, None, None, None, None, None, 7, 1e3,
                           9.81, None, None)
    assert st == -1 and b"p_mode" in lib.swense_last_error()
    g = S.make_grid(16, 16, 16, 1, 4, 5, 1.0, 1.0, z, [0.0, 1, 2, 3, 4])
    st = lib.swense_interp(ctypes.byref(g), 0.0, 16, 10, None, None, None, None, None, 0, 1e3,
                           9.81, None, None)
    assert st == -1


def test_validation_of_tuning_plan_and_direct_entry_points(lib):
    """The newer entry points reject bad arguments on the host, before any CUDA call."""
    import ctypes
    import numpy as np
    from paper_2005_12716_gb300 import _swense as S
    S.load()
    assert lib.swense_set_grid_tune(64, 32, 1, 12, 3, 32 << 20, 0) == -1          # lpc 3
    assert lib.swense_set_grid_tune(64, 32, 1, 12, 2, 1024, 0) == -1              # chunk < 1 MiB
    assert lib.swense_set_grid_tune(64, 32, 1, 12, 2, 32 << 20, 6) == -1          # variant 6
    assert lib.swense_set_grid_tune(64, 32, 1, 12, -1, 32 << 20, 0) == 0          # forget: fine
    assert lib.swense_interp_plan_bytes(0) == 0
    assert lib.swense_interp_plan_bytes(1) == 16 and lib.swense_interp_plan_bytes(1025) == 32
    z = np.array([-1, -0.5, 0.0, 0.1], np.float32)
    g = S.make_grid(16, 16, 16, 1, 4, 1, 1.0, 1.0, z, [0.0])
    st = lib.swense_interp_with_plan(ctypes.byref(g), 0.0, 16, 10, None, None, None, None, None,
                                     None, 0, 1e3, 9.81, None, None)
    assert st == -1 and b"plan" in lib.swense_last_error()
    st = lib.swense_interp_with_plan(ctypes.byref(g), 0.0, 16, 10, 24, None, None, None, None,
                                     None, 0, 1e3, 9.81, None, None)
    assert st == -1                                                                # misaligned
    m = S.swense_modes(8, 4, 1.0, 1.0, 0.0, 1, 16, 16, 16, None, 0.0)
    st = lib.swense_direct(ctypes.byref(m), 0.0, 16, 4, None, None, None, None, None, 0, 1e3,
                           9.81, 7, None)
    assert st == -1 and b"precision" in lib.swense_last_error()


def test_relax_cells_validation(lib):
    """Bad zones and sizes are rejected on the host before any CUDA call."""
    import ctypes
    from paper_2005_12716_gb300 import _swense as S
    S.load()
    Z = S.swense_relax_zone

    def call(zones, n=None, nc=10):
        arr = (Z * max(1, len(zones)))(*[Z(*z) for z in zones])
        return lib.swense_relax_cells(None, None, None, nc, ctypes.cast(arr, ctypes.c_void_p),
                                      len(zones) if n is None else n, None, None, None, None, None)
    assert call([(S.ZONE_X, 1.0, 2.0, 0, 0)] * 9) == -1                     # more than 8 zones
    assert call([(7, 1.0, 2.0, 0, 0)]) == -1 and b"kind" in lib.swense_last_error()
    assert call([(S.ZONE_RADIAL, 2.0, 2.0, 0, 0)]) == -1                     # empty zone
    assert call([(S.ZONE_Y, float("nan"), 2.0, 0, 0)]) == -1
    assert call([], n=-1) == -1
    assert call([(S.ZONE_X, 1.0, 2.0, 0, 0)], nc=-5) == -1
    assert call([(S.ZONE_X, 1.0, 2.0, 0, 0)]) == -1 and b"NULL" in lib.swense_last_error()
    assert call([(S.ZONE_X, 1.0, 2.0, 0, 0)], nc=0) == 0                     # nothing to do


def test_tank_modes_validation(lib):
    import ctypes
    from paper_2005_12716_gb300 import _swense as S
    S.load()
    m = S.swense_modes()
    call = lambda nx, ny, ns=1, L=4.0: lib.swense_tank_modes(8, 8, 8, nx, ny, ns, L, 2.0, 1.0, 8, 8, 8,  # noqa: E731
                                                             ctypes.byref(m), None)
    assert call(4, 1) == -2                  # 2 (4 - 1) = 6 is not a power of two
    assert call(2, 1) == -2
    assert call(65, 4) == -2
    assert call(65, 33, ns=0) == -1
    assert call(65, 33, ns=5) == -1
    assert call(65, 33, L=-1.0) == -1
    assert lib.swense_tank_modes(None, 8, 8, 65, 33, 1, 4.0, 2.0, 1.0, 8, 8, 8, ctypes.byref(m), None) == -1


def test_grid_node_count_rules(lib):
    """Gathers take even node counts (powers of two, or a padding factor such as 3 times one);
    odd counts are rejected, and the learned correction declines counts that are not powers of
    two, all before any CUDA call."""
    import ctypes
    import numpy as np
    from paper_2005_12716_gb300 import _swense as S
    S.load()
    z = np.array([-1, -0.5, -0.2, 0.0, 0.1], np.float32)
    odd = S.make_grid(256, 256, 385, 64, 5, 1, 8.0, 4.0, z, [0.0])
    assert lib.swense_interp(ctypes.byref(odd), 0.0, 16, 10, None, None, None, None, None, 0, 1e3,
                             9.81, None, None) == -2
    assert lib.swense_bin_points(ctypes.byref(odd), 16, 10, 16, 16, None) == -2
    three = S.make_grid(256, 256, 384, 192, 5, 1, 8.0, 4.0, z, [0.0])     # padding factor 3
    assert lib.swense_interp_learned(ctypes.byref(three), 0.0, 16, 10, None, None, None, None, None,
                                     0, 1e3, 9.81, 256, None, None) == -7
    assert b"power-of-two" in lib.swense_last_error()
