"""tgs_rasterize_batch: frames of different scenes, resolutions and bins rendered by one persistent
tensor-core launch must equal the frames tgs_rasterize renders one at a time, bit for bit (every
(frame, tile group) item runs the same per-group arithmetic). A frame whose readiness flag is never
set times out on the device (bounded wait), is reported through its status word, and leaves the
other frames and later calls unaffected."""
import ctypes as C

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


@pytest.fixture(scope="module")
def frames_src():
    box, cams = scenes.box_2k_128()
    mix = scenes.mixture_scene(40_000, seed=31, components=32, cluster_std=0.3, radius=2.0,
                               log_scale_mean=-3.8, sh_degree=3, needle_fraction=0.05)
    big = scenes.mixture_scene(150_000, seed=7, components=64, cluster_std=0.3, radius=3.0,
                               log_scale_mean=-4.2, sh_degree=3)
    ds = [tgs.DeviceScene.from_host(x) for x in (box, mix, big)]
    views = [(0, cams[0]), (1, scenes.orbit_cameras(8, 5.0, 320, 240)[3]),
             (1, scenes.orbit_cameras(8, 5.0, 203, 149)[5]), (2, scenes.orbit_cameras(4, 6.0, 640, 480)[1]),
             (0, scenes.identity_camera(70, 33)), (2, scenes.orbit_cameras(4, 6.0, 1280, 720)[2])]
    return ds, views


def _prepare(ds, views, tiling):
    out = []
    for si, cam in views:
        proj = tgs.preprocess(ds[si], cam)
        bins = tgs.bin_sort(proj, cam.width, cam.height, tiling)
        out.append((cam, proj, bins))
    return out


@pytest.mark.parametrize("tiling,precision", [((2, 2), "fp16_tc"), ((1, 1), "fp16_tc"), ((4, 4), "fp16_tc"),
                                              ((2, 2), "bf16_tc"), ((4, 2), "bf16_tc")])
def test_batch_equals_single_frames(frames_src, tiling, precision):
    ds, views = frames_src
    prepared = _prepare(ds, views, tiling)
    frames, refs = [], []
    for cam, proj, bins in prepared:
        rgb = torch.full((3, cam.height, cam.width), -1.0, device="cuda")
        T = torch.full((cam.height, cam.width), -1.0, device="cuda")
        frames.append(tgs.BatchFrame(proj, bins, cam.width, cam.height, rgb, T))
        refs.append(tgs.rasterize(proj, bins, cam.width, cam.height, precision, want_n_contrib=False))
    tgs.rasterize_batch(frames, tiling, precision)
    torch.cuda.synchronize()
    assert tgs.last_device_error() == 0
    for f, (r_rgb, r_T, _) in zip(frames, refs):
        assert np.array_equal(_np(f.out_rgb), _np(r_rgb))
        assert np.array_equal(_np(f.out_T), _np(r_T))


def test_ready_flags_and_device_timeout(frames_src):
    ds, views = frames_src
    prepared = _prepare(ds, views[:3], (2, 2))
    ready = torch.zeros(3, dtype=torch.int32, device="cuda")
    status = torch.zeros(3, dtype=torch.int32, device="cuda")
    done = torch.zeros(3, dtype=torch.int32).pin_memory()  # host words the device writes
    ready[0] = 5
    ready[2] = 5  # frame 1's flag is never set
    frames, refs = [], []
    for k, (cam, proj, bins) in enumerate(prepared):
        rgb = torch.full((3, cam.height, cam.width), -1.0, device="cuda")
        T = torch.full((cam.height, cam.width), -1.0, device="cuda")
        frames.append(tgs.BatchFrame(proj, bins, cam.width, cam.height, rgb, T, ready=ready[k:k + 1],
                                     ready_value=5, status=status[k:k + 1], done=done[k:k + 1],
                                     done_value=10 + k))
        refs.append(tgs.rasterize(proj, bins, cam.width, cam.height, "fp16_tc", want_n_contrib=False))
    ws = tgs.rasterize_batch(frames, (2, 2), "fp16_tc", wait_limit_ns=2_000_000)  # 2 ms
    torch.cuda.synchronize()
    assert _np(status).tolist() == [tgs.TGS_OK, tgs.TGS_ERR_TIMEOUT, tgs.TGS_OK]
    assert done.tolist() == [10, 11, 12]  # every frame completes, the failed one included
    for k in (0, 2):
        assert np.array_equal(_np(frames[k].out_rgb), _np(refs[k][0]))
    assert np.all(_np(frames[1].out_rgb) == -1.0)  # skipped: nothing written
    # the device stays usable: once the flag is set the same batch renders every frame
    ready[1] = 5
    status.zero_()
    done.zero_()
    tgs.rasterize_batch(frames, (2, 2), "fp16_tc", workspace=ws)
    torch.cuda.synchronize()
    assert _np(status).tolist() == [0, 0, 0] and tgs.last_device_error() == 0
    assert done.tolist() == [10, 11, 12]
    for f, r in zip(frames, refs):
        assert np.array_equal(_np(f.out_rgb), _np(r[0]))


def test_batch_argument_checks(frames_src):
    ds, views = frames_src
    cam, proj, bins = _prepare(ds, views[:1], (2, 2))[0]
    rgb = torch.empty((3, cam.height, cam.width), device="cuda")
    T = torch.empty((cam.height, cam.width), device="cuda")
    f = tgs.BatchFrame(proj, bins, cam.width, cam.height, rgb, T)
    with pytest.raises(tgs.TgsError):
        tgs.rasterize_batch([f], (2, 2), "fp32")
    with pytest.raises(tgs.TgsError):
        tgs.rasterize_batch([f] * 33, (2, 2), "fp16_tc")
    lib = tgs.load()
    o = tgs._RasterOpts(1, 0, (C.c_float * 3)(0, 0, 0), None)
    t = tgs._Tiling(2, 2)
    assert lib.tgs_rasterize_batch(None, 1, C.byref(t), C.byref(o), 0, None, None) == tgs.TGS_ERR_INVALID_ARGUMENT
