"""The library's host-side stream-function solve (C ABI, no GPU) against the FP64 oracle's own
solve of the same equations, and its argument checks."""
import numpy as np
import pytest

from oracle import stream as O


@pytest.fixture(scope="module")
def S():
    from paper_2005_12716_gb300 import build
    build.build()
    from paper_2005_12716_gb300 import _swense
    _swense.load()
    return _swense


CASES = [(0.7, 0.058, 0.6, 9, 4),        # the paper's progressive wave (kh 4.7, ka 0.22)
         (1.0, 0.05, 50.0, 16, 4),       # deep water
         (2.0, 0.12, 0.5, 20, 8),        # shallow, kh 0.76
         (0.7, 0.1, 0.6, 9, 4)]          # steep, ka 0.36


@pytest.mark.parametrize("T,H,h,n,steps", CASES)
def test_host_solve_matches_oracle(S, T, H, h, n, steps):
    w = S.swense_stream_solve(T, H, h, 9.81, n, steps)
    o = O.solve(T, H, h, n, steps=steps)
    assert w.n == n
    for key in ("k", "c", "ubar", "Q", "R"):
        assert getattr(w, key) == pytest.approx(o[key], rel=1e-10, abs=1e-13), key
    assert np.max(np.abs(np.array(w.B[:n]) - o["B"])) <= 1e-10 * np.max(np.abs(o["B"]))
    assert np.max(np.abs(np.array(w.E[:n + 1]) - o["E"])) <= 1e-10 * H
    assert np.max(np.abs(np.array(w.eta_m[:n + 1]) - o["eta_m"])) <= 1e-10 * H


def test_host_solve_rejects_bad_requests(S):
    lib = S.load()
    w = S.swense_stream_wave()
    import ctypes
    assert lib.swense_stream_solve(0.7, 0.058, 0.6, 9.81, 0, 4, ctypes.byref(w)) == -2     # n
    assert lib.swense_stream_solve(0.7, 0.058, 0.6, 9.81, 33, 4, ctypes.byref(w)) == -2
    assert lib.swense_stream_solve(-0.7, 0.058, 0.6, 9.81, 9, 4, ctypes.byref(w)) == -1
    assert lib.swense_stream_solve(0.7, 0.058, 0.6, 9.81, 9, 0, ctypes.byref(w)) == -1
    assert lib.swense_stream_solve(0.7, 0.058, 0.6, 9.81, 9, 4, None) == -1
    # far beyond breaking (H / lambda ~ 0.5): no wave exists, the solve must say so
    assert lib.swense_stream_solve(0.7, 0.4, 0.6, 9.81, 9, 2, ctypes.byref(w)) == -8
    assert b"CONVERGENCE" in lib.swense_last_error()
    bad = S.swense_stream_wave()                                                           # unsolved
    assert lib.swense_stream_eval(ctypes.byref(bad), 0.0, 0.0, None, 10, None, None, None, None,
                                  None, 0, 1000.0, None) == -2
