"""Pins of the FP64 oracle against things other than itself: closed forms, invariants, library
routines (scipy's complex spherical harmonics and rotations) and brute force on tiny inputs.

Each test names the part of the paper it pins. A plausible mistake in the oracle (a dropped term,
a wrong sign, a transposed operand, a wrong bit order) fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

from paper_2605_17855_gb300 import scenes

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


# ------------------------------------------------------------------------------------------------
# Section 2, feature computation: SH colour.

def _real_sh_scipy(l, m, d):
    """Real SH from scipy's complex Y_l^m (Condon-Shortley phase included)."""
    x, y, z = d
    theta = math.acos(max(-1.0, min(1.0, z)))
    phi = math.atan2(y, x)
    if m == 0:
        return sph_harm_y(l, 0, theta, phi).real
    Y = sph_harm_y(l, abs(m), theta, phi)
    return math.sqrt(2.0) * (Y.imag if m < 0 else Y.real)


def test_sh_basis_matches_scipy(orc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        got = orc.sh_basis(d)
        for l in range(4):
            for m in range(-l, l + 1):
                assert got[l * l + m + l] == pytest.approx(_real_sh_scipy(l, m, d), abs=1e-12)


def test_sh_orthonormal_by_quadrature(orc):
    # Gauss-Legendre in cos(theta) x uniform in phi integrates degree <= 6 products exactly.
    xs, ws = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros((16, 16))
    for ct, w in zip(xs, ws):
        st = math.sqrt(1 - ct * ct)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            Y = orc.sh_basis([st * math.cos(ph), st * math.sin(ph), ct])
            G += np.outer(Y, Y) * w * (2 * math.pi / nphi)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def _single(mean, scale, quat, opacity=0.5, sh=None, deg=0):
    sh = np.zeros((1, (deg + 1) ** 2, 3), np.float32) if sh is None else np.asarray(sh, np.float32)
    return scenes.Scene(np.asarray([mean], np.float32), np.asarray([scale], np.float32),
                        np.asarray([quat], np.float32), np.asarray([opacity], np.float32), sh, deg)


def test_sh_colour_degree0_and_clamp(orc):
    cam = scenes.identity_camera(64, 64)
    y00 = sph_harm_y(0, 0, 0.0, 0.0).real
    for dc, expect in ((1.0, 0.5 + y00), (-3.0, 0.0), (0.0, 0.5)):
        s = _single([0, 0, 3], [0.05] * 3, [1, 0, 0, 0], sh=[[[dc, dc, dc]]])
        pr = orc.preprocess(s, cam)
        np.testing.assert_allclose(pr.rgb[0], [max(expect, 0.0)] * 3, atol=1e-12)


def test_sh_colour_view_dependent(orc):
    # degree 1 with only the m=0 (z) band set: colour = 0.5 + k * Y_1^0(dir)
    cam = scenes.identity_camera(64, 64)
    sh = np.zeros((1, 4, 3), np.float32)
    sh[0, 2, :] = [0.5, -0.25, 0.125]
    s = _single([0.3, -0.2, 3.0], [0.05] * 3, [1, 0, 0, 0], sh=sh, deg=1)
    pr = orc.preprocess(s, cam)
    d = np.array([0.3, -0.2, 3.0], np.float32).astype(np.float64)
    d /= np.linalg.norm(d)
    y10 = _real_sh_scipy(1, 0, d)
    np.testing.assert_allclose(pr.rgb[0], 0.5 + sh[0, 2].astype(np.float64) * y10, atol=1e-12)


# ------------------------------------------------------------------------------------------------
# Section 2, feature computation: EWA projection, conic (Section 4.2.1), radius.

def test_projection_on_axis_closed_form(orc):
    cam = scenes.identity_camera(128, 96)
    z, s = 3.0, 0.02
    sc = _single([0, 0, z], [s] * 3, [0.3, 0.5, -0.1, 0.8])  # isotropic: rotation irrelevant
    pr = orc.preprocess(sc, cam)
    fx = cam.fx
    var = (fx * np.float32(s) / z) ** 2
    np.testing.assert_allclose(pr.mean2d[0], [cam.cx, cam.cy], atol=1e-12)
    assert pr.depth[0] == pytest.approx(z)
    np.testing.assert_allclose(pr.conic[0], [1 / (var + 0.3), 0.0, 1 / (var + 0.3)], rtol=1e-6, atol=1e-12)
    # isotropic: discriminant is 0, floored to 0.1 -> lambda_max = var + 0.3 + sqrt(0.1)
    assert pr.radius[0] == math.ceil(3 * math.sqrt(var + 0.3 + math.sqrt(0.1)))


def _mc_projected_cov(mean, scale, quat_wxyz, cam, n=2_000_000, seed=0):
    """Empirical covariance of 3D samples pushed through the pinhole map. The 3D covariance is built
    with scipy's Rotation (quaternion order x, y, z, w)."""
    rng = np.random.default_rng(seed)
    w, x, y, z = quat_wxyz
    Rq = Rotation.from_quat([x, y, z, w]).as_matrix()
    S3 = Rq @ np.diag(np.asarray(scale, np.float64) ** 2) @ Rq.T
    L = np.linalg.cholesky(S3)
    pts = np.asarray(mean, np.float64) + rng.standard_normal((n, 3)) @ L.T
    R = np.asarray(cam.R, np.float64)
    pc = pts @ R.T + np.asarray(cam.t, np.float64)
    u = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
    v = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
    return np.cov(np.stack([u, v]))


def _with_focal(cam, fx, fy):
    """The camera with its focal lengths replaced (fx != fy exercises the two axes separately)."""
    import dataclasses
    return dataclasses.replace(cam, fx=float(np.float32(fx)), fy=float(np.float32(fy)))


@pytest.mark.parametrize("cam_kind", ["identity", "look_at"])
def test_projection_off_axis_from_back_projection(orc, cam_kind):
    # The inverse route: start from a pixel (u, v) and a depth z, walk from the camera centre along
    # its right / down / forward axes by ((u - cx) z / fx, (v - cy) z / fy, z), and put a splat
    # there. Its projected mean must land back on (u, v) and its depth must be z. x != y, fx != fy
    # and an off-centre principal point (W != H) make a swapped axis or focal length visible.
    if cam_kind == "identity":
        cam = _with_focal(scenes.identity_camera(240, 130), 150.0, 95.0)
        eye = np.zeros(3)
        right, down, fwd = np.eye(3)
    else:
        base = scenes.look_at_camera([2.0, 1.0, -3.0], [0.0, 0.2, 0.0], 200, 150)
        cam = _with_focal(base, 180.0, 120.0)
        eye = np.asarray(base.cam_pos, np.float64)
        fwd = np.array([0.0, 0.2, 0.0]) - np.array([2.0, 1.0, -3.0])
        fwd /= np.linalg.norm(fwd)
        down = -(np.array([0.0, 1.0, 0.0]) - fwd[1] * fwd)
        down /= np.linalg.norm(down)
        right = np.cross(down, fwd)
    for (u, v, z) in ((37.25, 101.5, 2.5), (cam.width - 20.75, 12.125, 4.0), (150.5, 20.0, 1.7)):
        X = (u - cam.cx) * z / cam.fx
        Y = (v - cam.cy) * z / cam.fy
        p = eye + X * right + Y * down + z * fwd
        pr = orc.preprocess(_single(p, [0.01] * 3, [1, 0, 0, 0]), cam)
        assert pr.radius[0] > 0
        # float32 rounding of the world-space mean moves the projection by ~1e-4 px
        np.testing.assert_allclose(pr.mean2d[0], [u, v], atol=2e-3)
        assert pr.depth[0] == pytest.approx(z, rel=1e-5)


@pytest.mark.parametrize("cam_kind", ["identity", "look_at"])
def test_ewa_covariance_matches_monte_carlo(orc, cam_kind):
    if cam_kind == "identity":
        cam = scenes.identity_camera(200, 150)
        mean = [0.4, -0.3, 3.0]
    else:
        cam = scenes.look_at_camera([2.0, 1.0, -3.0], [0.0, 0.2, 0.0], 200, 150)
        mean = [0.3, 0.1, 0.4]
    quat = [0.8, 0.3, -0.4, 0.33]
    qn = np.asarray(quat) / np.linalg.norm(quat)
    scale = [0.004, 0.012, 0.002]
    got = orc.project_cov(mean, scale, np.asarray(qn, np.float32), cam)
    want = _mc_projected_cov(mean, np.asarray(scale, np.float32), np.asarray(qn, np.float32).astype(np.float64), cam)
    tol = 0.01 * max(abs(want[0, 0]), abs(want[1, 1]))
    assert abs(got[0] - want[0, 0]) < tol
    assert abs(got[1] - want[0, 1]) < tol
    assert abs(got[2] - want[1, 1]) < tol
    # the off-diagonal must be resolved: the splat is visibly tilted on screen
    assert abs(want[0, 1]) > 5 * tol


def test_ewa_jacobian_clamp_outside_view(orc):
    # Beyond 1.3 tan(half FOV) the Jacobian is taken at the clamped point: moving the mean further out
    # at the same depth leaves the projected covariance unchanged.
    cam = scenes.identity_camera(100, 100)
    lim = 1.3 * 0.5 * cam.width / cam.fx
    z = 2.0
    q = np.asarray([0.9, 0.1, 0.3, -0.2], np.float32)
    c_far = orc.project_cov([3.0 * lim * z, 0.1, z], [0.02, 0.05, 0.01], q, cam)
    c_far2 = orc.project_cov([5.0 * lim * z, 0.1, z], [0.02, 0.05, 0.01], q, cam)
    c_in = orc.project_cov([0.5 * lim * z, 0.1, z], [0.02, 0.05, 0.01], q, cam)
    np.testing.assert_allclose(c_far, c_far2, rtol=1e-12)
    assert not np.allclose(c_far, c_in, rtol=1e-3)


def test_conic_inverts_dilated_covariance(orc):
    scene, cams = scenes.box_2k_128()
    cam = cams[0]
    pr = orc.preprocess(scene, cam)
    for i in range(0, scene.n, 97):
        cov = orc.project_cov(scene.means[i], scene.scales[i], scene.quats[i], cam)
        S = np.array([[cov[0] + 0.3, cov[1]], [cov[1], cov[2] + 0.3]])
        a, b, c = pr.conic[i]
        np.testing.assert_allclose(np.array([[a, b], [b, c]]) @ S, np.eye(2), atol=1e-12)
        lam = np.linalg.eigvalsh(S)
        disc = max(0.1, ((S[0, 0] - S[1, 1]) / 2) ** 2 + S[0, 1] ** 2)
        assert pr.radius[i] == math.ceil(3 * math.sqrt(0.5 * (S[0, 0] + S[1, 1]) + math.sqrt(disc)))
        assert pr.radius[i] >= math.ceil(3 * math.sqrt(lam[1]) - 1e-9)


def test_near_plane_culling(orc):
    cam = scenes.identity_camera(64, 64)
    for z, visible in ((0.19, False), (0.2, False), (0.25, True), (-1.0, False)):
        pr = orc.preprocess(_single([0, 0, z], [0.001] * 3, [1, 0, 0, 0]), cam)
        assert (pr.radius[0] > 0) == visible


# ------------------------------------------------------------------------------------------------
# Section 2, tile intersection (AABB) -- brute force over pixels.

def test_tile_rect_brute_force(orc):
    rng = np.random.default_rng(3)
    for _ in range(400):
        W, H = int(rng.integers(1, 90)), int(rng.integers(1, 90))
        mx, my = rng.uniform(-30, W + 30), rng.uniform(-30, H + 30)
        if rng.random() < 0.2:
            mx = float(np.floor(mx))  # exact integers exercise the closed bounds
        r = int(rng.integers(1, 25))
        ok, rect = orc.tile_rect(mx, my, r, W, H)
        tiles = set()
        for y in range(H):
            for x in range(W):
                if mx - r <= x <= mx + r and my - r <= y <= my + r:
                    tiles.add((x // 16, y // 16))
        assert ok == bool(tiles)
        if tiles:
            want = {(tx, ty) for tx in range(rect[0], rect[2]) for ty in range(rect[1], rect[3])}
            assert tiles == want


# ------------------------------------------------------------------------------------------------
# Section 4.4.2 / Algorithm 1: group entries, masks, sort by (group, depth).

def _tiny_projected(rng, n, W, H):
    mean2d = np.stack([rng.uniform(-10, W + 10, n), rng.uniform(-10, H + 10, n)], 1).astype(np.float32)
    radius = rng.integers(1, 20, n).astype(np.int32)
    radius[rng.random(n) < 0.1] = 0
    depth = rng.uniform(1, 5, n).astype(np.float32)
    depth[: n // 5] = depth[n // 5: 2 * (n // 5)]  # equal depths exercise the index tie-break
    return mean2d, radius, depth


@pytest.mark.parametrize("gw,gh", [(1, 1), (2, 2), (4, 2), (4, 4), (1, 2), (3, 1)])
def test_group_entries_expand_to_tile_entries(orc, gw, gh):
    rng = np.random.default_rng(10 + gw * 7 + gh)
    W, H = 100, 70  # ragged: 7 x 5 tiles
    mean2d, radius, depth = _tiny_projected(rng, 300, W, H)
    b1 = orc.bin_sort(mean2d, radius, depth, W, H, 1, 1)
    bg = orc.bin_sort(mean2d, radius, depth, W, H, gw, gh)
    TX, TY, GX, GY = orc.group_grid(W, H, gw, gh)
    tile_pairs = set()
    for k in range(b1.num_entries):
        t = int(b1.keys[k] >> 32)
        assert b1.masks[k] == 1
        tile_pairs.add((t % TX, t // TX, int(b1.vals[k])))
    grp_pairs = set()
    for k in range(bg.num_entries):
        g = int(bg.keys[k] >> 32)
        gx, gy = g % GX, g // GX
        m = int(bg.masks[k])
        assert m != 0 and m < (1 << (gw * gh))
        for bit in range(gw * gh):
            if m >> bit & 1:
                tx, ty = gx * gw + bit % gw, gy * gh + bit // gw
                assert tx < TX and ty < TY
                grp_pairs.add((tx, ty, int(bg.vals[k])))
    assert grp_pairs == tile_pairs
    # every splat's group entries cover exactly the groups its tiles fall in
    assert bg.num_entries == len({(tx // gw, ty // gh, i) for tx, ty, i in tile_pairs})


@pytest.mark.parametrize("gw,gh", [(1, 1), (2, 2), (4, 2)])
def test_sort_order_and_ranges(orc, gw, gh):
    rng = np.random.default_rng(20 + gw)
    W, H = 77, 61
    mean2d, radius, depth = _tiny_projected(rng, 400, W, H)
    b = orc.bin_sort(mean2d, radius, depth, W, H, gw, gh)
    keys = [(int(k), int(v)) for k, v in zip(b.keys, b.vals)]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    # low 32 bits are the float32 depth bits of the splat
    for k, v in keys:
        assert (k & 0xFFFFFFFF) == int(np.float32(depth[v]).view(np.uint32))
    _, _, GX, GY = orc.group_grid(W, H, gw, gh)
    for g in range(GX * GY):
        s, e = b.ranges[g]
        idx = [k for k, (key, _) in enumerate(keys) if key >> 32 == g]
        if idx:
            assert (s, e) == (idx[0], idx[-1] + 1)
        else:
            assert (s, e) == (0, 0)


# ------------------------------------------------------------------------------------------------
# Section 2, Eqs. power_d, power, alpha, blend; pruning and early termination.

def _bins_for(orc, mean2d, radius, depth, W, H, gw=2, gh=2):
    return orc.bin_sort(np.asarray(mean2d, np.float64), np.asarray(radius, np.int32),
                        np.asarray(depth, np.float64), W, H, gw, gh)


def test_single_isotropic_splat_closed_form(orc):
    W = H = 48
    mu = np.array([[20.3, 25.6]])
    sig2 = 9.0
    conic = np.array([[1 / sig2, 0.0, 1 / sig2]])
    o, c = 0.7, np.array([[0.2, 0.5, 0.9]])
    r = 10
    b = _bins_for(orc, mu, [r], [2.0], W, H)
    img = orc.blend(W, H, mu, conic, [o], c, b)
    for y in range(H):
        for x in range(W):
            d2 = (x - mu[0, 0]) ** 2 + (y - mu[0, 1]) ** 2
            a = min(0.99, o * math.exp(-d2 / (2 * sig2)))
            _, rect = orc.tile_rect(mu[0, 0], mu[0, 1], r, W, H)
            in_rect = rect[0] <= x // 16 < rect[2] and rect[1] <= y // 16 < rect[3]
            if in_rect and a >= 1 / 255:
                np.testing.assert_allclose(img.rgb[y, x], a * c[0], rtol=1e-13, atol=1e-15)
                assert img.T[y, x] == pytest.approx(1 - a, rel=1e-13)
                assert img.n_contrib[y, x] == 1
            else:
                assert np.all(img.rgb[y, x] == 0) and img.T[y, x] == 1.0 and img.n_contrib[y, x] == 0


def test_two_splats_front_to_back(orc):
    W = H = 32
    mu = np.array([[10.0, 10.0], [11.0, 9.5]])
    conic = np.array([[0.1, 0.02, 0.15], [0.2, -0.05, 0.08]])
    o = np.array([0.6, 0.8])
    c = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.5]])
    px = (12, 9)
    a = []
    for i in range(2):
        dx, dy = px[0] - mu[i, 0], px[1] - mu[i, 1]
        pw = -0.5 * (conic[i, 0] * dx * dx + conic[i, 2] * dy * dy) - conic[i, 1] * dx * dy
        a.append(min(0.99, o[i] * math.exp(pw)))
    for depth, order in (([1.0, 2.0], (0, 1)), ([3.0, 2.0], (1, 0))):
        b = _bins_for(orc, mu, [8, 8], depth, W, H)
        img = orc.blend(W, H, mu, conic, o, c, b)
        i, j = order
        want = a[i] * c[i] + (1 - a[i]) * a[j] * c[j]
        np.testing.assert_allclose(img.rgb[px[1], px[0]], want, rtol=1e-12)
        assert img.T[px[1], px[0]] == pytest.approx((1 - a[i]) * (1 - a[j]), rel=1e-12)


def test_early_termination_does_not_blend_the_stopping_entry(orc):
    W = H = 16
    n = 4
    mu = np.tile([[8.0, 8.0]], (n, 1))
    conic = np.tile([[0.5, 0.0, 0.5]], (n, 1))
    o = np.full(n, 0.98)
    c = np.eye(3)[[0, 1, 2, 0]] * 1.0
    b = _bins_for(orc, mu, [3] * n, [1.0, 2.0, 3.0, 4.0], W, H, 1, 1)
    img = orc.blend(W, H, mu, conic, o, c, b)
    # at the centre: alpha = 0.98 each; T: 1 -> 0.02 -> 4e-4 -> 8e-6 (< 1e-4: stop, not blended)
    np.testing.assert_allclose(img.rgb[8, 8], [0.98, 0.02 * 0.98, 0.0], rtol=1e-12)
    assert img.T[8, 8] == pytest.approx(0.02 * 0.02, rel=1e-12)
    assert img.n_contrib[8, 8] == 2


def test_pruning_of_negligible_alpha(orc):
    W = H = 16
    mu = np.array([[8.0, 8.0]])
    for o, blended in ((0.9 / 255, False), (1.1 / 255, True)):
        img = orc.blend(W, H, mu, [[0.5, 0.0, 0.5]], [o], [[1.0, 1.0, 1.0]], _bins_for(orc, mu, [3], [1.0], W, H))
        assert (img.n_contrib[8, 8] == 1) == blended


def test_blend_weights_sum_to_one(orc):
    # with every colour 1 and a black background, C = sum_i T_i alpha_i = 1 - T_final
    scene, cams = scenes.box_2k_128()
    pr = orc.preprocess(scene, cams[0])
    b = orc.bin_sort(pr.mean2d, pr.radius, pr.depth, 128, 128, 2, 2)
    img = orc.blend(128, 128, pr.mean2d, pr.conic, pr.opacity, np.ones_like(pr.rgb), b)
    np.testing.assert_allclose(img.rgb[..., 0] + img.T, 1.0, atol=1e-12)
    assert img.T.min() >= 1e-4  # stop-before-blend keeps T >= 1e-4
    assert img.guard == 0


def _brute_force_pixel(orc, x, y, pr, W, H):
    """Blend one pixel over ALL splats globally sorted by (float32 depth, index) whose tile range
    holds the pixel's tile -- no group lists, no masks."""
    order = sorted((int(np.float32(pr.depth[i]).view(np.uint32)), i)
                   for i in range(len(pr.radius)) if pr.radius[i] > 0)
    T, C, last = 1.0, np.zeros(3), 0
    pos = 0
    for _, i in order:
        ok, rect = orc.tile_rect(pr.mean2d[i, 0], pr.mean2d[i, 1], int(pr.radius[i]), W, H)
        if not (ok and rect[0] <= x // 16 < rect[2] and rect[1] <= y // 16 < rect[3]):
            continue
        pos += 1
        dx, dy = x - pr.mean2d[i, 0], y - pr.mean2d[i, 1]
        a, b, c = pr.conic[i]
        power = -0.5 * a * dx * dx - b * dx * dy - 0.5 * c * dy * dy
        if power > 0:
            continue
        alpha = min(0.99, pr.opacity[i] * math.exp(power))
        if alpha < 1 / 255:
            continue
        Tn = T * (1 - alpha)
        if Tn < 1e-4:
            break
        C = C + alpha * T * pr.rgb[i]
        T = Tn
        last = pos
    return C, T, last


def test_group_lists_equal_brute_force_per_pixel(orc):
    scene = scenes.box_scene(60, seed=11, log_scale_mean=-2.5)
    cam = scenes.identity_camera(40, 36)
    pr = orc.preprocess(scene, cam)
    b = orc.bin_sort(pr.mean2d, pr.radius, pr.depth, 40, 36, 1, 1)
    img = orc.blend(40, 36, pr.mean2d, pr.conic, pr.opacity, pr.rgb, b)
    for y in range(0, 36, 3):
        for x in range(0, 40, 3):
            C, T, last = _brute_force_pixel(orc, x, y, pr, 40, 36)
            assert np.array_equal(img.rgb[y, x], C) and img.T[y, x] == T and img.n_contrib[y, x] == last


@pytest.mark.parametrize("gw,gh", [(2, 2), (4, 2), (4, 4), (1, 2), (3, 3)])
def test_grouping_is_exact(orc, gw, gh):
    # Section 4.4.2: filtering a group list by the mask keeps every tile's order, so the image is
    # identical to the per-tile rasterization.
    scene = scenes.box_scene(1500, seed=5, log_scale_mean=-3.0)
    cam = scenes.identity_camera(150, 110)
    pr = orc.preprocess(scene, cam)
    i1 = orc.blend(150, 110, pr.mean2d, pr.conic, pr.opacity, pr.rgb,
                   orc.bin_sort(pr.mean2d, pr.radius, pr.depth, 150, 110, 1, 1))
    ig = orc.blend(150, 110, pr.mean2d, pr.conic, pr.opacity, pr.rgb,
                   orc.bin_sort(pr.mean2d, pr.radius, pr.depth, 150, 110, gw, gh))
    assert np.array_equal(i1.rgb, ig.rgb) and np.array_equal(i1.T, ig.T)
    assert i1.evaluated == ig.evaluated


def test_pixel_list_matches_full_frame(orc):
    scene, cams = scenes.box_2k_128()
    pr, b, img = orc.render(scene, cams[0])
    rng = np.random.default_rng(0)
    pix = np.stack([rng.integers(0, 128, 200), rng.integers(0, 128, 200)], 1)
    sub = orc.blend(128, 128, pr.mean2d, pr.conic, pr.opacity, pr.rgb, b, pixels=pix)
    assert np.array_equal(sub.rgb, img.rgb[pix[:, 1], pix[:, 0]])
    assert np.array_equal(sub.n_contrib, img.n_contrib[pix[:, 1], pix[:, 0]])


# ------------------------------------------------------------------------------------------------
# Backward of the blend: analytic chain rule vs FP64 central differences of the forward.

def _fd_check(orc, W, H, mu, conic, opac, rgb, depth, pix, G, bg=(0.0, 0.0, 0.0), radius=16,
              tiling=(2, 2)):
    """Analytic gradient of L = sum(image[pix] * G) against FP64 central differences of the
    forward. Returns the analytic gradients."""
    b = _bins_for(orc, mu, [radius] * len(opac), depth, W, H, *tiling)

    def loss(m, cn, o, c):
        img = orc.blend(W, H, m, cn, o, c, b, bg=bg, pixels=pix)
        return float(np.sum(img.rgb * G)), img

    _, base = loss(mu, conic, opac, rgb)
    assert base.margin.min() > 1e-3  # FD steps stay on one side of every threshold
    g = orc.blend_backward(W, H, mu, conic, opac, rgb, b, G, bg=bg, pixels=pix)
    names = ["mean2d", "conic", "opacity", "rgb"]
    for name, arr, grad in (("mean2d", mu, g.mean2d), ("conic", conic, g.conic),
                            ("opacity", opac, g.opacity), ("rgb", rgb, g.rgb)):
        flat = arr.reshape(-1)
        fd = np.zeros_like(flat)
        for k in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[k]))
            args = [mu.copy(), conic.copy(), opac.copy(), rgb.copy()]
            idx = names.index(name)
            args[idx].reshape(-1)[k] += h
            lp, _ = loss(*args)
            args[idx].reshape(-1)[k] -= 2 * h
            lm, _ = loss(*args)
            fd[k] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(grad.reshape(-1), fd, rtol=1e-5, atol=1e-7 * max(np.abs(fd).max(), 1e-3),
                                   err_msg=name)
    return g, base


@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.3, 0.6, 0.9)])
def test_backward_matches_central_differences(orc, bg):
    # a random stack; with a non-zero background the colour behind each entry includes bg T_final
    rng = np.random.default_rng(7)
    W, H, n = 32, 32, 12
    mu = np.stack([rng.uniform(6, 26, n), rng.uniform(6, 26, n)], 1)
    s2 = rng.uniform(4, 16, n)
    conic = np.stack([1 / s2, rng.uniform(-0.02, 0.02, n), 1 / (s2 * rng.uniform(0.7, 1.3, n))], 1)
    opac = rng.uniform(0.2, 0.7, n)
    rgb = rng.uniform(0, 1, (n, 3))
    depth = rng.uniform(1, 3, n)
    pix = np.array([(x, y) for y in range(10, 22, 2) for x in range(10, 22, 2)])
    G = rng.standard_normal((len(pix), 3))
    g, base = _fd_check(orc, W, H, mu, conic, opac, rgb, depth, pix, G, bg)
    if any(bg):  # the background term is live: T_final < 1 at the pixels and non-zero gradients
        assert base.T.max() < 1.0 and np.abs(g.opacity).max() > 0


def test_backward_alpha_cap_passes_no_gradient(orc):
    # Splat 1 reaches o e^power > 0.99 at the test pixel: its alpha is the constant 0.99 there, so
    # neither its opacity nor its power inputs (mean, conic) receive a gradient from that pixel;
    # its colour still does. Splats 0 (in front) and 2 (behind) are below the cap.
    W = H = 32
    mu = np.array([[11.0, 8.5], [10.1, 9.85], [12.0, 11.0]])
    conic = np.array([[0.08, 0.01, 0.1], [1 / 9, 0.0, 1 / 9], [0.05, -0.01, 0.06]])
    opac = np.array([0.4, 0.998, 0.7])
    rgb = np.array([[0.9, 0.1, 0.2], [0.3, 0.8, 0.4], [0.2, 0.3, 0.95]])
    depth = np.array([1.0, 2.0, 3.0])
    pix = np.array([(10, 10)])
    d = pix[0] - mu[1]
    oe = opac[1] * math.exp(-0.5 * (conic[1, 0] * d[0] ** 2 + conic[1, 2] * d[1] ** 2)
                            - conic[1, 1] * d[0] * d[1])
    assert oe - 0.99 > 1e-3  # the cap holds on both sides of every FD step
    G = np.array([[0.7, -1.1, 0.4]])
    g, base = _fd_check(orc, W, H, mu, conic, opac, rgb, depth, pix, G, bg=(0.1, 0.2, 0.3))
    assert g.opacity[1] == 0.0 and np.all(g.conic[1] == 0.0) and np.all(g.mean2d[1] == 0.0)
    assert np.all(g.rgb[1] != 0.0)
    assert g.opacity[0] != 0.0 and g.opacity[2] != 0.0


def test_backward_early_termination(orc):
    # Four nearly opaque splats and a faint one over the test pixels: T falls 1 -> ~0.05 -> ~2.5e-3 -> ~1.3e-4,
    # the fourth would take it below 1e-4 and ends the pixel unblended. The fourth and fifth
    # splats therefore get no gradient at all (their parameters do not change the image), and the
    # first three get the gradient of a stack that stops there.
    W = H = 32
    n = 5
    mu = np.array([[16.2, 15.9], [15.8, 16.1], [16.1, 16.3], [15.9, 15.7], [16.3, 16.2]])
    conic = np.tile([[0.02, 0.002, 0.025]], (n, 1))
    opac = np.array([0.96, 0.95, 0.95, 0.97, 0.1])  # a faint fifth splat would still blend
    rgb = np.random.default_rng(5).uniform(0.1, 0.9, (n, 3))
    depth = np.arange(1.0, n + 1.0)
    pix = np.array([(16, 16), (17, 15), (15, 17)])
    G = np.random.default_rng(6).standard_normal((len(pix), 3))
    g, base = _fd_check(orc, W, H, mu, conic, opac, rgb, depth, pix, G, bg=(0.5, 0.25, 0.75))
    assert np.all(base.n_contrib == 3)
    assert np.all(base.T < 1e-3) and np.all(base.T >= 1e-4)
    assert base.evaluated == 4 * len(pix)  # the fourth splat is evaluated and stops the pixel
    for k in (3, 4):
        assert g.opacity[k] == 0.0 and np.all(g.conic[k] == 0.0) and np.all(g.mean2d[k] == 0.0)
        assert np.all(g.rgb[k] == 0.0)
    assert np.all(g.opacity[:3] != 0.0)


# ------------------------------------------------------------------------------------------------
# Tile membership at binning time (beyond the paper): a tile stays in a splat's entry only if the
# splat can reach alpha >= 1/255 there.

def _membership_case(seed, n=400, W=150, H=110):
    """Projected splats of every shape: round and needle-like conics at every orientation, tiny
    and large, opacities from just above 1/255 to 0.99, centres on and off screen."""
    rng = np.random.default_rng(seed)
    mean2d = np.stack([rng.uniform(-20, W + 20, n), rng.uniform(-20, H + 20, n)], 1).astype(np.float32)
    s_major = np.exp(rng.uniform(np.log(0.6), np.log(40.0), n))
    ratio = np.where(rng.random(n) < 0.3, rng.uniform(20, 400, n), rng.uniform(1, 3, n))
    s_minor = np.maximum(s_major / ratio, 0.55)
    th = rng.uniform(0, np.pi, n)
    cth, sth = np.cos(th), np.sin(th)
    # covariance = Rot diag(s_major^2, s_minor^2) Rot^T; conic = its inverse
    cxx = cth ** 2 * s_major ** 2 + sth ** 2 * s_minor ** 2
    cyy = sth ** 2 * s_major ** 2 + cth ** 2 * s_minor ** 2
    cxy = cth * sth * (s_major ** 2 - s_minor ** 2)
    det = cxx * cyy - cxy ** 2
    conic = np.stack([cyy / det, -cxy / det, cxx / det], 1).astype(np.float32)
    opac = np.where(rng.random(n) < 0.15, rng.uniform(1.0 / 255, 0.02, n), rng.uniform(0.02, 0.99, n))
    opac = opac.astype(np.float32)
    radius = np.ceil(3 * np.sqrt(0.5 * (cxx + cyy) + np.sqrt(np.maximum(0.1, (0.5 * (cxx - cyy)) ** 2
                                                                         + cxy ** 2)))).astype(np.int32)
    depth = rng.uniform(1, 5, n).astype(np.float32)
    return mean2d, conic, opac, radius, depth, W, H


def _pairs(orc, b, W, H):
    """(splat, tx, ty) of every set mask bit."""
    TX, TY, GX, GY = orc.group_grid(W, H, b.gw, b.gh)
    out = set()
    for k in range(b.num_entries):
        g = int(b.keys[k] >> 32)
        gx, gy = g % GX, g // GX
        for bit in range(b.gw * b.gh):
            if int(b.masks[k]) >> bit & 1:
                out.add((int(b.vals[k]), gx * b.gw + bit % b.gw, gy * b.gh + bit // b.gw))
    return out


def _max_alpha_in_tile(mean2d, conic, opac, i, tx, ty, W, H):
    xs = np.arange(tx * 16, min(tx * 16 + 16, W), dtype=np.float64)
    ys = np.arange(ty * 16, min(ty * 16 + 16, H), dtype=np.float64)
    X, Y = np.meshgrid(xs, ys)
    a, b, c = conic[i].astype(np.float64)
    dx, dy = X - float(mean2d[i, 0]), Y - float(mean2d[i, 1])
    power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
    return float(opac[i]) * float(np.exp(power.max()))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_membership_drops_only_pairs_below_the_pruning_threshold(orc, seed):
    mean2d, conic, opac, radius, depth, W, H = _membership_case(seed)
    rect_only = orc.bin_sort(mean2d, radius, depth, W, H, 1, 1)
    member = orc.bin_sort(mean2d, radius, depth, W, H, 1, 1, conic=conic, opacity=opac)
    all_pairs, kept = _pairs(orc, rect_only, W, H), _pairs(orc, member, W, H)
    assert kept <= all_pairs
    dropped = all_pairs - kept
    assert len(dropped) > 0.3 * len(all_pairs)  # the rule does cull
    # conservative: every dropped pair is pruned at every pixel centre of its tile (FP64 brute force)
    for (i, tx, ty) in dropped:
        assert _max_alpha_in_tile(mean2d, conic, opac, i, tx, ty, W, H) < 1.0 / 255.0, (i, tx, ty)
    # tight: the pairs kept although no pixel of the tile reaches 1/255 are a small minority
    dead_kept = sum(1 for (i, tx, ty) in kept
                    if _max_alpha_in_tile(mean2d, conic, opac, i, tx, ty, W, H) < 1.0 / 255.0)
    dead = dead_kept + len(dropped)
    assert dead_kept < 0.15 * dead, (dead_kept, dead)


@pytest.mark.parametrize("gw,gh", [(2, 2), (4, 2), (4, 4), (3, 1)])
def test_membership_does_not_depend_on_grouping(orc, gw, gh):
    # the kept (splat, tile) pairs are a property of the splat and the tile alone
    mean2d, conic, opac, radius, depth, W, H = _membership_case(9)
    one = orc.bin_sort(mean2d, radius, depth, W, H, 1, 1, conic=conic, opacity=opac)
    grp = orc.bin_sort(mean2d, radius, depth, W, H, gw, gh, conic=conic, opacity=opac)
    assert _pairs(orc, grp, W, H) == _pairs(orc, one, W, H)
    assert np.all(grp.masks != 0)


def test_membership_leaves_the_image_unchanged(orc):
    # dropped pairs would be pruned at every pixel: colour and transmittance are bit-identical, the
    # passing pairs are the same, only pairs that fail the 1/255 test disappear from the lists
    scene = scenes.mixture_scene(6000, seed=4, components=8, cluster_std=0.3, radius=1.5,
                                 log_scale_mean=-3.2, sh_degree=1, needle_fraction=0.2)
    cam = scenes.orbit_cameras(4, 4.0, 200, 150)[1]
    pr = orc.preprocess(scene, cam)
    for gw, gh in ((1, 1), (2, 2)):
        plain = orc.bin_sort(pr.mean2d, pr.radius, pr.depth, 200, 150, gw, gh)
        memb = orc.bin_sort(pr.mean2d, pr.radius, pr.depth, 200, 150, gw, gh, conic=pr.conic,
                            opacity=pr.opacity)
        assert memb.num_entries < plain.num_entries
        i0 = orc.blend(200, 150, pr.mean2d, pr.conic, pr.opacity, pr.rgb, plain, bg=(0.1, 0.2, 0.3))
        i1 = orc.blend(200, 150, pr.mean2d, pr.conic, pr.opacity, pr.rgb, memb, bg=(0.1, 0.2, 0.3))
        assert np.array_equal(i0.rgb, i1.rgb) and np.array_equal(i0.T, i1.T)
        assert i0.passing == i1.passing and i1.evaluated < i0.evaluated
        # n_contrib counts list positions: the last blended splat is the same one
        _, _, GX, _ = orc.group_grid(200, 150, gw, gh)
        for y in range(0, 150, 7):
            for x in range(0, 200, 7):
                g = ((y // 16) // gh) * GX + (x // 16) // gw
                n0, n1 = int(i0.n_contrib[y, x]), int(i1.n_contrib[y, x])
                assert (n0 == 0) == (n1 == 0)
                if n0:
                    assert plain.vals[plain.ranges[g][0] + n0 - 1] == memb.vals[memb.ranges[g][0] + n1 - 1]
