"""Edge cases of the CUDA path against the FP64 oracle: the widest image the ABI accepts with a
ragged height, one splat covering the whole image, a stack of near-opaque splats (early
termination), the 0.99 alpha cap, a minimal splat on a tile corner, and the large-group binning path (more groups
than fit the per-tile count arrays in shared memory). Same bars as the parity tests."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU-only hosts
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_2605_17855_gb300 as tgs  # noqa: E402
from paper_2605_17855_gb300 import scenes  # noqa: E402

from parity_bars import check  # noqa: E402


def _np(t):
    return t.detach().cpu().numpy()


def _scene(means, scales, opac, colour, quats=None):
    n = len(means)
    means = np.asarray(means, np.float32).reshape(n, 3)
    scales = np.asarray(scales, np.float32).reshape(n, 3)
    q = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)) if quats is None else np.asarray(quats, np.float32)
    sh = ((np.asarray(colour, np.float32).reshape(n, 1, 3) - 0.5) / (0.5 / np.sqrt(np.pi))).astype(np.float32)
    return scenes.Scene(means, scales, q, np.asarray(opac, np.float32).reshape(n), sh, 0)


def _check(scene, cam, tiling, precisions=("fp32", "fp16_tc", "bf16_tc")):
    """Bins bit-exact and every precision's image against the oracle; returns the oracle image."""
    ds = tgs.DeviceScene.from_host(scene)
    proj = tgs.preprocess(ds, cam)
    bins = tgs.bin_sort(proj, cam.width, cam.height, tiling)
    torch.cuda.synchronize()
    co = _np(proj.conic_opacity).astype(np.float64)
    p = dict(mean2d=_np(proj.mean2d).astype(np.float64), conic=co[:, :3], opacity=co[:, 3],
             rgb=_np(proj.rgb).astype(np.float64), depth=_np(proj.depth), radius=_np(proj.radius))
    ob = oracle.bin_sort(p["mean2d"], p["radius"], p["depth"], cam.width, cam.height, *tiling,
                         conic=p["conic"], opacity=p["opacity"])
    E = bins.entries
    assert E == ob.num_entries
    assert np.array_equal(_np(bins.vals[:E]).view(np.uint32), ob.vals)
    assert np.array_equal(_np(bins.masks[:E]).view(np.uint16), ob.masks)
    assert np.array_equal(_np(bins.ranges).view(np.uint32), ob.ranges)
    assert np.array_equal(_np(bins.keys[:E]).view(np.uint64), ob.keys)
    img = oracle.blend(cam.width, cam.height, p["mean2d"], p["conic"], p["opacity"], p["rgb"], ob)
    ref = img.rgb.transpose(2, 0, 1)
    for prec in precisions:
        rgb, T, nc = tgs.rasterize(proj, bins, cam.width, cam.height, prec)
        torch.cuda.synchronize()
        assert tgs.last_device_error() == 0
        rgb, T, nc = _np(rgb), _np(T), _np(nc)
        check(prec, rgb, T, nc, ref, img.T, img.n_contrib, img.margin, (prec, tiling))
    return img


def test_widest_image_with_ragged_height():
    # 16384 x 40: the largest width the ABI accepts; 40 rows cut the last tile row at 8 pixels
    cam = scenes.identity_camera(16384, 40, 60.0)
    scene = scenes.box_scene(4000, seed=12, sh_degree=1, log_scale_mean=-4.0)
    scene.means[:, 1] *= 0.005  # squeeze into the thin horizontal band the camera sees
    img = _check(scene, cam, (2, 2))
    assert (img.T < 1.0).mean() > 0.05  # the band is actually covered


@pytest.mark.parametrize("tiling", [(1, 1), (4, 4)])
def test_one_splat_covers_the_image(tiling):
    # a single large splat in front of the camera: an entry in every group, lists of length one
    cam = scenes.identity_camera(200, 120, 60.0)
    scene = _scene([[0.02, -0.01, 3.0]], [[2.0, 1.5, 0.5]], [0.8], [[0.2, 0.6, 0.9]])
    img = _check(scene, cam, tiling)
    assert (img.n_contrib == 1).all()


def test_near_opaque_stack_terminates():
    # 64 broad splats of opacity 0.97 stacked in depth: a central pixel blends a few of them until
    # the next would drop T below 1e-4, and stops
    rng = np.random.default_rng(5)
    n = 64
    means = np.stack([rng.uniform(-0.05, 0.05, n), rng.uniform(-0.05, 0.05, n),
                      np.linspace(2.0, 5.0, n)], 1)
    scene = _scene(means, np.full((n, 3), 0.4), np.full(n, 0.97), rng.uniform(0, 1, (n, 3)))
    cam = scenes.identity_camera(96, 80, 60.0)
    img = _check(scene, cam, (2, 2))
    # n_contrib is the list position of the last blended entry: the pixels stop early in the list,
    # with T between the termination bound and a few layers above it
    T = img.T[30:50, 38:58]
    assert img.n_contrib[30:50, 38:58].max() <= 12 and (T >= 1e-4).all() and (T < 1e-2).all()


def test_alpha_cap():
    # opacity 0.999 in front of a 0.5 splat: alpha is capped at 0.99 around the centre, so T = 0.01
    # there before the second splat
    scene = _scene([[0.0, 0.0, 2.0], [0.0, 0.0, 4.0]], [[0.3, 0.3, 0.3], [1.0, 1.0, 1.0]], [0.999, 0.5],
                   [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    cam = scenes.identity_camera(64, 64, 60.0)
    img = _check(scene, cam, (2, 2))
    c = img.T[31:33, 31:33]
    assert np.allclose(c, 0.01 * (1 - 0.5 * np.exp(-0.5 * 0.0)), rtol=0.02)


def test_minimal_splat_on_a_tile_corner():
    # a tiny splat centred where four tiles meet: it belongs to all four (and to up to four groups)
    cam = scenes.identity_camera(64, 64, 60.0)
    fx = cam.fx
    z = 2.0
    x = (15.5 - cam.cx) * z / fx
    y = (15.5 - cam.cy) * z / fx
    scene = _scene([[x, y, z]], [[1e-4, 1e-4, 1e-4]], [0.9], [[1.0, 0.5, 0.25]])
    for tiling in ((1, 1), (2, 2)):
        img = _check(scene, cam, tiling)
        assert img.n_contrib.sum() > 0


@pytest.mark.parametrize("width,height", [(4096, 3000), (4608, 4096)])
def test_many_groups(width, height):
    # 1x1 tiles: 256 x 188 groups (16 group-id bits, two radix passes) and 288 x 256 groups (17
    # bits, three passes: the sorted indices and masks reach the output after an odd number)
    cam = scenes.identity_camera(width, height, 60.0)
    scene = scenes.box_scene(20000, seed=9, sh_degree=0, log_scale_mean=-4.5)
    ds = tgs.DeviceScene.from_host(scene)
    proj = tgs.preprocess(ds, cam)
    bins = tgs.bin_sort(proj, cam.width, cam.height, (1, 1))
    torch.cuda.synchronize()
    co = _np(proj.conic_opacity).astype(np.float64)
    ob = oracle.bin_sort(_np(proj.mean2d).astype(np.float64), _np(proj.radius), _np(proj.depth),
                         cam.width, cam.height, 1, 1, conic=co[:, :3], opacity=co[:, 3])
    E = bins.entries
    assert E == ob.num_entries and E > 20000
    assert np.array_equal(_np(bins.vals[:E]).view(np.uint32), ob.vals)
    assert np.array_equal(_np(bins.masks[:E]).view(np.uint16), ob.masks)
    assert np.array_equal(_np(bins.ranges).view(np.uint32), ob.ranges)


@pytest.mark.parametrize("tiling", [(1, 1), (2, 2), (4, 4)])
def test_deep_stack_spans_many_jobs(tiling):
    # 150 translucent splats over the same tiles: a tile's packed rows overflow the 32 rows of a
    # tensor-core job several times, so its entries are spread over many jobs (and super-chunks);
    # the list order, the image and the list positions (n_contrib) must survive the split
    rng = np.random.default_rng(11)
    n = 150
    means = np.stack([rng.uniform(-0.02, 0.02, n), rng.uniform(-0.02, 0.02, n),
                      np.linspace(2.0, 6.0, n)], 1)
    scene = _scene(means, np.full((n, 3), 0.5), np.full(n, 0.04), rng.uniform(0, 1, (n, 3)))
    cam = scenes.identity_camera(96, 80, 60.0)
    img = _check(scene, cam, tiling)
    # no pixel terminates (0.96^150 > 1e-4), so central pixels blend every splat
    assert img.n_contrib[38:42, 46:50].min() == n
    ds = tgs.DeviceScene.from_host(scene)
    proj = tgs.preprocess(ds, cam)
    bins = tgs.bin_sort(proj, cam.width, cam.height, tiling)
    for prec in ("fp16_tc", "bf16_tc"):
        _, _, nc = tgs.rasterize(proj, bins, cam.width, cam.height, prec)
        torch.cuda.synchronize()
        assert np.array_equal(_np(nc)[38:42, 46:50], img.n_contrib[38:42, 46:50]), prec
