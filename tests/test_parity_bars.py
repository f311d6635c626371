"""The GPU parity bars themselves (tests/parity_bars.py), on synthetic images with planted errors:
each bar fails when it should and the 0.01% budget admits no more than it states. CPU only."""
import numpy as np
import pytest

import parity_bars as pb

H, W = 40, 50  # 2000 pixels: the budget allows ceil(0.2) = 1 pixel


def _ref(seed=0):
    rng = np.random.default_rng(seed)
    rgb = rng.uniform(0, 1, (3, H, W))
    T = rng.uniform(0, 1, (H, W))
    nc = rng.integers(0, 50, (H, W)).astype(np.int32)
    margin = np.full((H, W), 1.0)  # every decision far from its threshold
    return rgb, T, nc, margin


@pytest.mark.parametrize("precision", ["fp32", "fp16_tc"])
def test_exact_images_pass(precision):
    rgb, T, nc, margin = _ref()
    pb.check(precision, rgb, T, nc, rgb, T, nc, margin)


def test_fp32_bar_on_unambiguous_pixels():
    rgb, T, nc, margin = _ref()
    bad = rgb.copy()
    bad[1, 3, 4] += 2e-4  # one pixel beyond 1e-4, its decisions far from any threshold
    with pytest.raises(AssertionError):
        pb.check("fp32", bad, T, nc, rgb, T, nc, margin)
    # the same pixel with an ambiguous decision uses the one-pixel budget
    m = margin.copy()
    m[3, 4] = 1e-7
    pb.check("fp32", bad, T, nc, rgb, T, nc, m)
    # two ambiguous pixels beyond the bar exceed the 0.01% budget
    bad[0, 5, 6] += 2e-4
    m[5, 6] = 1e-7
    with pytest.raises(AssertionError):
        pb.check("fp32", bad, T, nc, rgb, T, nc, m)


def test_fp32_n_contrib_and_T():
    rgb, T, nc, margin = _ref()
    nc2 = nc.copy()
    nc2[0, 0] += 1
    with pytest.raises(AssertionError):
        pb.check("fp32", rgb, T, nc2, rgb, T, nc, margin)
    T2 = T.copy()
    T2[7, 7] += 2e-4
    with pytest.raises(AssertionError):
        pb.check("fp32", rgb, T2, nc, rgb, T, nc, margin)


def test_tensor_core_bars():
    rgb, T, nc, margin = _ref()
    # inside 2/255 everywhere and PSNR far above 45 dB: passes
    ok = rgb + 1e-4
    pb.check("fp16_tc", ok, T, nc, rgb, T, nc, margin)
    # one pixel beyond 2/255 fails, however ambiguous (no exclusion from max abs)
    bad = rgb.copy()
    bad[2, 1, 1] += 3.0 / 255.0
    m = np.full_like(margin, 1e-9)
    with pytest.raises(AssertionError):
        pb.check("fp16_tc", bad, T, nc, rgb, T, nc, m)
    # a uniform error of 1/255 keeps every pixel inside 2/255 but costs PSNR (48 dB): passes;
    # 1.9/255 (42.5 dB) fails the PSNR bar
    pb.check("fp16_tc", np.clip(rgb + 1.0 / 255.0, 0, None), T, nc, np.clip(rgb, 0, None), T, nc, margin)
    with pytest.raises(AssertionError):
        pb.check("fp16_tc", rgb + 1.9 / 255.0, T, nc, rgb, T, nc, margin)
    # T off by more than 1e-4 on an unambiguous pixel fails; on an ambiguous one it passes
    T2 = T.copy()
    T2[4, 4] += 5e-4
    with pytest.raises(AssertionError):
        pb.check("fp16_tc", rgb, T2, nc, rgb, T, nc, margin)
    m2 = margin.copy()
    m2[4, 4] = 1e-5
    pb.check("fp16_tc", rgb, T2, nc, rgb, T, nc, m2)
    # n_contrib: one ambiguous flip is within the budget, two are not
    nc2 = nc.copy()
    nc2[9, 9] += 1
    m3 = margin.copy()
    m3[9, 9] = 1e-5
    pb.check("fp16_tc", rgb, T, nc2, rgb, T, nc, m3)
    nc2[10, 10] += 1
    m3[10, 10] = 1e-5
    with pytest.raises(AssertionError):
        pb.check("fp16_tc", rgb, T, nc2, rgb, T, nc, m3)
