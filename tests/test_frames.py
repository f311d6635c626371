"""GPU tests of frame sequences from host memory (tgs_frames_*): every image equals the direct
preprocess -> bin sort -> rasterize path bit for bit, across calls that alternate between scenes
(the two device scene copies), more frames than buffer sets, pinned and pageable host arrays and
both precisions; a frame that needs more bin entries than the capacity renders the background and
is reported by wait; bad arguments are refused; render and wait allocate nothing."""
import numpy as np
import pytest
import torch

import paper_2605_17855_gb300 as tgs
from paper_2605_17855_gb300 import scenes

pytestmark = pytest.mark.gpu

BG = (0.1, 0.2, 0.3)


def _host(scene, pin):
    # the scene's arrays as CPU tensors (page-locked or not), plus sh_degree
    class H:
        pass
    h = H()
    for k in ("means", "scales", "quats", "opacities", "sh"):
        t = torch.from_numpy(np.ascontiguousarray(getattr(scene, k), np.float32))
        setattr(h, k, t.pin_memory() if pin else t)
    h.sh_degree = scene.sh_degree
    return h


def _direct(scene, cams, tiling, precision):
    ds = tgs.DeviceScene.from_host(scene)
    out = []
    for cam in cams:
        rgb, T, _, _, _ = tgs.render(ds, cam, tiling, precision, BG)
        out.append((rgb.cpu().numpy(), T.cpu().numpy()))
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("precision,tiling", [("fp16_tc", (2, 2)), ("fp32", (1, 1))])
def test_frames_equal_direct_path(precision, tiling):
    mix = scenes.mixture_scene(40_000, seed=31, components=32, cluster_std=0.3, radius=2.0,
                               log_scale_mean=-3.8, sh_degree=3, needle_fraction=0.05)
    box, _ = scenes.box_2k_128()
    cams = scenes.orbit_cameras(8, 5.0, 320, 240)[:5]
    calls = [(mix, [0, 1, 2, 3, 4], True), (box, [0, 1, 2], False), (mix, [2, 3, 4], True),
             (box, [0, 1, 2, 3, 4], True)]
    ref = {id(mix): _direct(mix, cams, tiling, precision), id(box): _direct(box, cams, tiling, precision)}
    lib = tgs.load()
    with tgs.Frames(60_000, max_size=(320, 240), max_entries=1 << 20, tiling=tiling,
                    precision=precision, bg=BG, sets=3) as fr:
        assert fr.device_bytes > 0
        before = lib.tgs_allocation_count()
        outs = []
        for scene, idx, pin in calls:
            rgb = torch.empty((len(idx), 3, 240, 320)).pin_memory()
            T = torch.empty((len(idx), 240, 320)).pin_memory()
            fr.render(_host(scene, pin), [cams[j] for j in idx], rgb, T)  # stream: the default
            outs.append((scene, idx, rgb, T))
        # the default stream waits for every call: synchronizing it alone completes the images
        torch.cuda.default_stream().synchronize()
        for scene, idx, rgb, T in outs:
            for k, j in enumerate(idx):
                assert np.array_equal(rgb[k].numpy(), ref[id(scene)][j][0])
                assert np.array_equal(T[k].numpy(), ref[id(scene)][j][1])
        fr.wait()
        assert lib.tgs_allocation_count() == before


def test_frames_capacity_and_arguments():
    box, cams = scenes.box_2k_128()
    cam = cams[0]
    host = _host(box, True)
    with tgs.Frames(box.means.shape[0], max_size=(cam.width, cam.height), max_entries=500,
                    precision="fp16_tc", bg=BG, sets=2, max_sh_degree=box.sh_degree) as fr:
        rgb = torch.empty((2, 3, cam.height, cam.width)).pin_memory()
        fr.render(host, [cam, cam], rgb)
        with pytest.raises(tgs.TgsError) as e:
            fr.wait()
        assert e.value.status == tgs.TGS_ERR_CAPACITY
        bg = np.broadcast_to(np.array(BG, np.float32)[:, None, None], (3, cam.height, cam.width))
        assert np.array_equal(rgb[0].numpy(), bg) and np.array_equal(rgb[1].numpy(), bg)
        fr.render(host, [], rgb)  # nothing to do
        fr.wait()                 # the overflow was reported once
        # a frame larger than the object's, cameras of two sizes, a scene larger than it
        big = scenes.identity_camera(cam.width * 2, cam.height)
        with pytest.raises(tgs.TgsError) as e:
            fr.render(host, [big], torch.empty((1, 3, cam.height, cam.width * 2)))
        assert e.value.status == tgs.TGS_ERR_INVALID_ARGUMENT
        small = scenes.identity_camera(cam.width // 2, cam.height // 2)
        with pytest.raises(tgs.TgsError) as e:
            fr.render(host, [cam, small], rgb)
        assert e.value.status == tgs.TGS_ERR_INVALID_ARGUMENT
        mix = scenes.mixture_scene(box.means.shape[0] + 1, seed=3, sh_degree=box.sh_degree)
        with pytest.raises(tgs.TgsError) as e:
            fr.render(_host(mix, False), [cam], rgb)
        assert e.value.status == tgs.TGS_ERR_INVALID_ARGUMENT
    with pytest.raises(tgs.TgsError) as e:
        tgs.Frames(1000, sets=1)
    assert e.value.status == tgs.TGS_ERR_INVALID_ARGUMENT
