"""The oracle's blend against single-pixel cases worked out by hand (tests/golden/*.txt): exact
fractions from the paper's blending equations (Section 2), read from text fixtures, so the
expected values share nothing with the oracle's code. Every case runs with 1x1 and 2x2 groups,
on the AABB lists (the paper's organisation) and on the tile-membership lists."""
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
W = H = 16
PIXEL = (8, 8)
CONIC = (0.25, 0.0, 0.25)
RADIUS = 6


def _cases(name):
    cases, cur = [], None
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            word, *rest = line.split()
            if word == "case":
                cur = {"name": rest[0], "splats": []}
                cases.append(cur)
            elif word == "splat":
                cur["splats"].append([Fraction(v) for v in rest])
            elif word in ("bg", "expect_rgb"):
                cur[word] = [Fraction(v) for v in rest]
            elif word == "expect_T":
                cur[word] = Fraction(rest[0])
            elif word == "expect_n_contrib":
                cur[word] = int(rest[0])
            else:
                raise ValueError(f"unknown fixture line: {raw!r}")
    return cases


CASES = _cases("blend_single_pixel.txt")


def test_fixture_is_complete():
    assert len(CASES) >= 7
    for c in CASES:
        assert {"bg", "expect_rgb", "expect_T", "expect_n_contrib"} <= set(c), c["name"]
        # the hand derivation: with every splat on the pixel, the weights and T add up to 1
        assert all(0 <= v for v in c["expect_rgb"]) and 0 < c["expect_T"] <= 1


@pytest.mark.parametrize("membership", [False, True], ids=["aabb", "membership"])
@pytest.mark.parametrize("gw,gh", [(1, 1), (2, 2)])
@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_blend_matches_hand_derivation(orc, case, gw, gh, membership):
    n = len(case["splats"])
    s = np.array([[float(v) for v in sp] for sp in case["splats"]], np.float64).reshape(n, 5)
    mean2d = np.tile(np.array([PIXEL], np.float64), (n, 1))
    conic = np.tile(np.array([CONIC], np.float64), (n, 1))
    depth, opacity, rgb = s[:, 0], s[:, 1], s[:, 2:5]
    radius = np.full(n, RADIUS, np.int32)
    extra = {"conic": conic, "opacity": opacity} if membership else {}
    bins = orc.bin_sort(mean2d, radius, depth, W, H, gw, gh, **extra)
    bg = [float(v) for v in case["bg"]]
    img = orc.blend(W, H, mean2d, conic, opacity, rgb, bins, bg=bg, pixels=[PIXEL])
    want_rgb = [float(v) for v in case["expect_rgb"]]
    np.testing.assert_allclose(img.rgb[0], want_rgb, rtol=1e-12, atol=1e-15)
    assert img.T[0] == pytest.approx(float(case["expect_T"]), rel=1e-12)
    if not membership:  # membership drops entries that cannot pass 1/255, shifting positions
        assert int(img.n_contrib[0]) == case["expect_n_contrib"]
