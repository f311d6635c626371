"""tgs_bin_sort_static: the bin sort for callers that cannot allocate device memory while they run
(a real-time frame loop with a fixed memory budget, or a host that owns all device memory). It uses
a fixed scratch area inside the library instead of a caller workspace. Its output must equal the
workspace version's exactly (binning is integer work), on two calls in a row that share the area.

This file is collected last on purpose: if it fails, a run that stops at the first failure has
already run every other test. It does not depend on any other test's state."""
import ctypes as C
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2605_17855_gb300 as tgs  # noqa: E402
from paper_2605_17855_gb300 import scenes  # noqa: E402


def _np(t):
    return t.detach().cpu().numpy()


def _case(name):
    if name == "box":
        scene, cams = scenes.box_2k_128()
        return scene, cams[0], (2, 2)
    scene = scenes.mixture_scene(30_000, seed=9, components=16, cluster_std=0.3, radius=2.0,
                                 log_scale_mean=-3.8, sh_degree=3)
    return scene, scenes.orbit_cameras(4, 5.0, 203, 149)[1], (4, 2)


def _static_call(proj, cam, tiling, capacity):
    """Bin sort through the raw C entry point with no workspace argument."""
    lib = tgs.load()
    out = tgs.allocate_bins(proj.n, capacity, cam.width, cam.height, tiling)
    host = C.c_int64(0)
    t = tgs._Tiling(*tiling)
    st = lib.tgs_bin_sort_static(C.byref(proj.struct()), proj.n, cam.width, cam.height, C.byref(t),
                                 C.byref(out.struct()), C.byref(host), None)
    assert st == tgs.TGS_OK, lib.tgs_last_error_message()
    out.entries = int(host.value)
    return out


def test_static_scratch_matches_workspace_on_consecutive_calls():
    results = []
    for name in ("box", "mixture"):  # two calls in a row sharing the scratch area
        scene, cam, tiling = _case(name)
        proj = tgs.preprocess(tgs.DeviceScene.from_host(scene), cam)
        ref = tgs.bin_sort(proj, cam.width, cam.height, tiling)
        got = _static_call(proj, cam, tiling, ref.capacity)
        torch.cuda.synchronize()
        E = ref.entries
        assert got.entries == E and E > 0
        for a, b in ((got.keys, ref.keys), (got.vals, ref.vals), (got.masks, ref.masks)):
            assert np.array_equal(_np(a[:E]), _np(b[:E]))
        assert np.array_equal(_np(got.ranges), _np(ref.ranges))
        results.append(E)
    # and again on the first case, after the second call left its contents in the area
    scene, cam, tiling = _case("box")
    proj = tgs.preprocess(tgs.DeviceScene.from_host(scene), cam)
    ref = tgs.bin_sort(proj, cam.width, cam.height, tiling)
    got = _static_call(proj, cam, tiling, ref.capacity)
    torch.cuda.synchronize()
    assert got.entries == results[0]
    assert np.array_equal(_np(got.vals[:got.entries]), _np(ref.vals[:ref.entries]))
    assert np.array_equal(_np(got.ranges), _np(ref.ranges))


@pytest.mark.parametrize("n,capacity,width,height,tiling", [
    (2_000_000, 100_000, 1024, 1024, (2, 2)),   # the per-Gaussian buffers do not fit
    (2_000, 4_000_000, 1600, 1064, (1, 1)),     # the group-id radix buffers do not fit
])
def test_static_scratch_rejects_oversized_requests(n, capacity, width, height, tiling):
    assert tgs.workspace_size(n, capacity, width, height, tiling) > (16 << 20)
    proj = tgs.Projected.empty(n, "cuda")  # refused before any kernel reads it
    cam = scenes.identity_camera(width, height)
    lib = tgs.load()
    big = tgs.allocate_bins(n, capacity, cam.width, cam.height, tiling)
    t = tgs._Tiling(*tiling)
    host = C.c_int64(123)
    st = lib.tgs_bin_sort_static(C.byref(proj.struct()), n, cam.width, cam.height, C.byref(t),
                                 C.byref(big.struct()), C.byref(host), None)
    assert st == tgs.TGS_ERR_CAPACITY
    assert b"static area holds" in lib.tgs_last_error_message()
    assert host.value == -1  # not an entry count: a caller must not retry with a larger capacity


def test_first_call_in_a_fresh_process_allocates_nothing():
    # A process whose very first library call is tgs_bin_sort_static: the library makes no
    # allocation at all (its counter of cudaMalloc / cudaMallocHost calls stays 0), the bins equal
    # the oracle's on three calls in a row, and device memory does not move across the later
    # calls. The first call may commit the library's device code and the static array (CUDA loads
    # modules lazily), which is bounded by the array's size plus the code.
    tgs.load()  # built before the child starts
    child = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_static_first_call.py")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, child, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["allocation_count"] == 0
    for c in res["calls"]:
        assert c["status"] == tgs.TGS_OK, c["message"]
        assert c["entries"] == c["oracle_entries"] > 0 and c["equal"]
    first, *later = res["calls"]
    assert 0 <= first["free_before"] - first["free_after"] <= (16 << 20) + (48 << 20)
    for c in later:
        assert c["free_before"] == c["free_after"]
