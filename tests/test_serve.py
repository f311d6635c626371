"""GPU tests of the rendering service (tgs_serve_*): frames rendered by the server (binned per slot,
rasterized together by batched tensor-core launches) equal the direct preprocess -> bin sort ->
rasterize path bit for bit; admission (BUSY), pause, bounded waits, scene removal while in use, the
fixed slot capacities and the HBM budget, nothing allocated by the worker, and per-resolution
statistics."""
import numpy as np
import pytest
import torch

import paper_2605_17855_gb300 as tgs
from paper_2605_17855_gb300 import scenes

pytestmark = pytest.mark.gpu

GB = 1 << 30


def _scenes():
    box, cams = scenes.box_2k_128()
    mix = scenes.mixture_scene(60_000, seed=7, components=16, cluster_std=0.4, radius=1.5,
                               log_scale_mean=-3.5, sh_degree=3)
    return box, cams[0], mix


def _cameras():
    # three resolutions of an orbit around the mixture scene
    out = []
    for k, (w, h) in enumerate([(320, 240), (256, 256), (200, 136)]):
        out.append(scenes.orbit_cameras(8, 4.0, w, h)[k])
    return out


def _direct(ds, cam, tiling, precision):
    rgb, T, _, _, _ = tgs.render(ds, cam, tiling, precision)
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), T.cpu().numpy()


@pytest.mark.parametrize("precision,tiling", [("fp16_tc", (2, 2)), ("fp32", (1, 1))])
def test_server_frames_equal_direct_path(precision, tiling):
    box, cam1, mix = _scenes()
    cams = _cameras()
    with tgs.Server(8 * GB, max_inflight=32, slots=4, precision=precision, tiling=tiling) as srv:
        s_box = srv.add_scene(tgs.DeviceScene.from_host(box))  # device arrays
        s_mix = srv.add_scene(mix)                            # host arrays
        jobs = []
        for rep in range(3):
            for cam in cams:
                rgb = torch.empty((3, cam.height, cam.width), device="cuda")
                T = torch.empty((cam.height, cam.width), device="cuda")
                jobs.append((srv.submit(s_mix, cam, rgb, T), "mix", cam, rgb, T))
            rgb = torch.empty((3, cam1.height, cam1.width), device="cuda")
            jobs.append((srv.submit(s_box, cam1, rgb, None), "box", cam1, rgb, None))
        for ticket, *_ in jobs:
            assert srv.wait(ticket, 20000) == tgs.TGS_OK
        ds = {"box": tgs.DeviceScene.from_host(box), "mix": tgs.DeviceScene.from_host(mix)}
        for _, name, cam, rgb, T in jobs:
            ref_rgb, ref_T = _direct(ds[name], cam, tiling, precision)
            assert np.array_equal(rgb.cpu().numpy(), ref_rgb)
            if T is not None:
                assert np.array_equal(T.cpu().numpy(), ref_T)
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["failed"] == 0 and st["inflight"] == 0
        res = {(r["width"], r["height"]): r for r in st["resolutions"]}
        assert set(res) == {(c.width, c.height) for c in cams} | {(cam1.width, cam1.height)}
        for r in res.values():
            assert 0 < r["p50_ms"] <= r["p99_ms"]
        assert st["hbm_bytes"] > 0


def test_admission_pause_wait_and_scene_removal():
    box, cam1, _ = _scenes()
    with tgs.Server(2 * GB, max_inflight=3, slots=2) as srv:
        sid = srv.add_scene(box)
        srv.pause(True)
        bufs = [torch.empty((3, cam1.height, cam1.width), device="cuda") for _ in range(4)]
        tickets = [srv.submit(sid, cam1, bufs[k]) for k in range(3)]
        assert srv.try_submit(sid, cam1, bufs[3]) is None        # max_inflight reached
        with pytest.raises(tgs.TgsError) as e:
            srv.wait(tickets[0], 0)                              # paused: not done
        assert e.value.status == tgs.TGS_ERR_TIMEOUT
        assert srv.poll(tickets[0]) is None
        with pytest.raises(tgs.TgsError) as e:
            srv.remove_scene(sid)                                # requests hold the scene
        assert e.value.status == tgs.TGS_ERR_BUSY
        srv.pause(False)
        for t in tickets:
            assert srv.wait(t, 20000) == tgs.TGS_OK
        with pytest.raises(tgs.TgsError) as e:
            srv.poll(tickets[0])                                 # released after completion
        assert e.value.status == tgs.TGS_ERR_NOT_FOUND
        st = srv.stats()
        assert st["rejected"] == 1 and st["completed"] == 3
        srv.remove_scene(sid)
        with pytest.raises(tgs.TgsError) as e:
            srv.submit(sid, cam1, bufs[0])
        assert e.value.status == tgs.TGS_ERR_NOT_FOUND


def test_budget_and_slot_capacities():
    box, cam1, mix = _scenes()
    # slot buffers are allocated at creation: a budget that cannot hold them refuses the server
    with pytest.raises(tgs.TgsError) as e:
        tgs.Server(4 << 20, max_inflight=4, slots=2, max_gaussians=1 << 20, max_size=(2048, 2048))
    assert e.value.status == tgs.TGS_ERR_CAPACITY
    with tgs.Server(16 << 20, max_inflight=4, slots=1, max_gaussians=4096, max_size=(256, 256),
                    max_entries=20000) as srv:
        with pytest.raises(tgs.TgsError) as e:
            srv.add_scene(mix)  # 60k Gaussians: more than a slot renders
        assert e.value.status == tgs.TGS_ERR_CAPACITY
        sid = srv.add_scene(box)
        big = scenes.identity_camera(512, 512)  # larger than a slot's frame
        rgb = torch.empty((3, 512, 512), device="cuda")
        assert srv.wait(srv.submit(sid, big, rgb), 20000) == tgs.TGS_ERR_CAPACITY
        rgb = torch.empty((3, cam1.height, cam1.width), device="cuda")
        assert srv.wait(srv.submit(sid, cam1, rgb), 20000) == tgs.TGS_OK
        assert srv.stats()["failed"] == 1


def test_entry_capacity_and_no_allocation_in_the_worker():
    # a frame that needs more bin entries than the slot holds completes with CAPACITY; the server
    # allocates nothing while it renders (every buffer comes from tgs_serve_create / add_scene)
    box, cam1, _ = _scenes()
    lib = tgs.load()
    with tgs.Server(1 << 30, max_inflight=8, slots=2, max_gaussians=4096, max_size=(128, 128),
                    max_entries=500) as srv:
        sid = srv.add_scene(box)
        before = lib.tgs_allocation_count()
        rgb = torch.empty((3, cam1.height, cam1.width), device="cuda")
        assert srv.wait(srv.submit(sid, cam1, rgb), 20000) == tgs.TGS_ERR_CAPACITY
        assert lib.tgs_allocation_count() == before
    with tgs.Server(1 << 30, max_inflight=8, slots=2, max_gaussians=4096, max_size=(128, 128),
                    max_entries=20000) as srv:
        sid = srv.add_scene(box)
        before = lib.tgs_allocation_count()
        bufs = [torch.empty((3, cam1.height, cam1.width), device="cuda") for _ in range(6)]
        for t in [srv.submit(sid, cam1, b) for b in bufs]:
            assert srv.wait(t, 20000) == tgs.TGS_OK
        assert lib.tgs_allocation_count() == before
        ref, _ = _direct(tgs.DeviceScene.from_host(box), cam1, (2, 2), "fp16_tc")
        for b in bufs:
            assert np.array_equal(b.cpu().numpy(), ref)
