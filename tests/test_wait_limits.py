"""GPU test of the bin sort's bounded look-back waits running out: with a limit far below a tile's
run time the waits expire, the device error word reads TGS_ERR_TIMEOUT, the call ends with empty
bins (every range (0, 0), no entries) that rasterize to the background, and the next call with the
default limit is correct again. Nothing faults or hangs: every wait is bounded, and a wait that
runs out only shortens the prefixes every later write position is derived from."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU-only hosts
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2605_17855_gb300 as tgs  # noqa: E402
from paper_2605_17855_gb300 import scenes  # noqa: E402


def _np(t):
    return t.detach().cpu().numpy()


def test_lookback_time_out_leaves_empty_bins_and_the_next_call_succeeds():
    scene, cams = scenes.mixture_1p5m_1600x1064(n=600_000, cams=1)
    cam = cams[0]
    ds = tgs.DeviceScene.from_host(scene)
    proj = tgs.preprocess(ds, cam)
    tgs.last_device_error(reset=True)
    ref = tgs.bin_sort(proj, cam.width, cam.height, (2, 2))
    E = ref.entries
    ref_vals, ref_ranges = _np(ref.vals[:E]).copy(), _np(ref.ranges).copy()
    bins = tgs.allocate_bins(proj.n, ref.capacity, cam.width, cam.height, (2, 2), keys=False)

    # a 1 ns limit: any look-back that finds an earlier tile unpublished gives up at once; with
    # hundreds of tiles per radix pass some wait is all but certain, so a few calls suffice
    timed_out = False
    previous = tgs.set_lookback_limit(1)
    try:
        for _ in range(8):
            try:
                tgs.bin_sort(proj, cam.width, cam.height, (2, 2), bins=bins)
            except tgs.TgsError as e:
                assert e.status == tgs.TGS_ERR_TIMEOUT
                timed_out = True
                break
    finally:
        assert tgs.set_lookback_limit(previous) == 1
    assert timed_out
    assert tgs.last_device_error(reset=True) == tgs.TGS_ERR_TIMEOUT
    assert tgs.last_device_error() == tgs.TGS_OK
    # the failed call's bins are empty and render the background
    assert int(_np(bins.num_entries)[0]) == 0
    assert not _np(bins.ranges).any()
    for prec in ("fp32", "fp16_tc"):
        rgb, T, nc = tgs.rasterize(proj, bins, cam.width, cam.height, prec, bg=(0.25, 0.5, 0.75))
        torch.cuda.synchronize()
        assert np.array_equal(_np(rgb), np.broadcast_to(
            np.array([0.25, 0.5, 0.75], np.float32)[:, None, None], (3, cam.height, cam.width)))
        assert (_np(T) == 1.0).all() and not _np(nc).any()

    # the default limit again: the same bins as before the time-out, no error recorded
    tgs.bin_sort(proj, cam.width, cam.height, (2, 2), bins=bins)
    torch.cuda.synchronize()
    assert bins.entries == E
    assert np.array_equal(_np(bins.vals[:E]), ref_vals)
    assert np.array_equal(_np(bins.ranges), ref_ranges)
    assert tgs.last_device_error() == tgs.TGS_OK
