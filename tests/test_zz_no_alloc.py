"""swense_fields_on_grid_noalloc: the allocation-free grid reconstruction for callers that cannot
call cudaMalloc (for example a solver that hands all device memory to its own pool at start-up).

Checked through the C ABI against swense_fields_on_grid, within the parity tolerance of the
other GPU tests (1e-5 of each field's maximum), on consecutive calls whose sizes differ, so that
what one call leaves in the shared scratch array cannot leak into the next. This file is named
to be collected last.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

from tests._util import rel_linf
from wavegen import configs

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12716_gb300 import build
    build.build()
    from paper_2005_12716_gb300 import _swense as S
    from paper_2005_12716_gb300 import api
    return torch, S, api


def _both(env, cfg, pad):
    torch, S, api = env
    sea, z, tl = cfg["sea"], cfg["z_levels"], cfg["t_levels"]
    modes = api.upload_modes(sea)
    ref = api.fields_on_grid(modes, z, pad, tl)                 # existing entry point
    out = api.alloc_grid(modes, z, pad, tl)
    out.nodes.fill_(float("nan"))
    out.eta.fill_(float("nan"))
    desc = S.make_grid_desc(pad, z)
    S.swense_fields_on_grid_noalloc(modes.c_struct(), len(tl), np.asarray(tl, np.float64), desc,
                                    out.nodes, out.eta)
    torch.cuda.synchronize()
    got_n, ref_n = out.nodes.cpu().numpy(), ref.nodes.cpu().numpy()
    for q in range(4):
        assert rel_linf(got_n[..., q], ref_n[..., q]) <= TOL, q
    assert rel_linf(out.eta.cpu().numpy(), ref.eta.cpu().numpy()) <= TOL


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(env):
    small = configs.jonswap3d_small()
    large = configs.jonswap3d(mesh_dims=(4, 8, 4))   # 512 x 256 modes, 64 levels: many chunks
    _both(env, small, 2)
    _both(env, large, 1)
    _both(env, small, 2)                            # after a larger call left its scratch behind


def test_noalloc_2d(env):
    torch, S, api = env
    cfg = configs.stokes2d(n_points=8)
    _both(env, cfg, 4)


def test_noalloc_rejects_requests_beyond_its_scratch(env):
    torch, S, api = env
    nx, ny = 2048, 1024                       # one level needs 32 MiB of scratch
    shape = (ny, nx // 2 + 1, 2)
    A = [torch.zeros(shape, dtype=torch.float32, device="cuda") for _ in range(3)]
    z = np.array([-1.0, -0.5, -0.1, 0.0], np.float32)
    nodes = torch.zeros((1, len(z), ny, nx, 4), dtype=torch.float32, device="cuda")
    eta = torch.zeros((1, ny, nx), dtype=torch.float32, device="cuda")
    m = S.make_modes(nx, ny, 64.0, 32.0, 0.0, A[0], A[1], A[2], n_snap=1)
    lib = S.load()
    launches = S.swense_launches()
    st = lib.swense_fields_on_grid_noalloc(ctypes.byref(m), 1, None,
                                           ctypes.byref(S.make_grid_desc(1, z)),
                                           nodes.data_ptr(), eta.data_ptr(), None)
    assert st == -2
    assert b"SWENSE_NOALLOC_SCRATCH_BYTES" in lib.swense_last_error()
    assert S.swense_launches() == launches


_FRESH = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2005_12716_gb300 import _swense as S, api
from wavegen import configs
torch.cuda.init()
cfg = configs.jonswap3d(mesh_dims=(4, 8, 4))      # 512 x 256 modes, 64 levels: many chunks
sea, z, tl = cfg["sea"], cfg["z_levels"], cfg["t_levels"]
modes = api.upload_modes(sea)
out = api.alloc_grid(modes, z, 1, tl)
for pad in (1, 2):
    if pad == 2:
        out = api.alloc_grid(modes, z, 2, tl)
    S.swense_fields_on_grid_noalloc(modes.c_struct(), len(tl), np.asarray(tl, np.float64),
                                    S.make_grid_desc(pad, z), out.nodes, out.eta)
torch.cuda.synchronize()
assert torch.isfinite(out.nodes).all() and torch.isfinite(out.eta).all()
print("WORKSPACE", S.swense_workspace_bytes())
"""


def test_noalloc_alone_leaves_the_library_workspace_unallocated(env):
    """A fresh process that makes only allocation-free calls (two grid sizes, the larger needing
    several level chunks) ends with no library workspace: nothing went through the allocator."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "WORKSPACE 0" in r.stdout, r.stdout[-500:]
