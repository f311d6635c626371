"""The parity bars of the rasterizers against the FP64 oracle, shared by the GPU test files.

Threshold decisions (alpha >= 1/255, T' < 1e-4, the 0.99 cap) can go either way when the exact
value sits within the arithmetic's error of the threshold; the oracle records, per pixel, the
smallest relative distance of any of its decisions from its threshold (`margin`). Reading of the
tolerance statement: a pixel whose margin is below the path's error bound is "ambiguous"; at most
0.01% of the pixels (rounded up to a whole pixel) may break a bar, and a pixel that does must be
ambiguous.

  FP32 CUDA-core path: max abs <= 1e-4 on rgb and T, n_contrib equal, on every pixel with margin
    > 1e-5 (FP32 alpha is accurate to ~1e-6 relative); over all pixels, at most 0.01% outside
    1e-4 or with a different n_contrib.
  Tensor-core paths (FP16, BF16): PSNR >= 45 dB and max abs <= 2/255 on rgb and T over ALL pixels
    (no exclusion: a single flipped decision moves a pixel by about alpha T c, inside the bar in
    practice, and the measured maximum is ~3e-5); n_contrib equal and |dT| <= 1e-4 on every pixel
    with margin > 1e-3 (the worst-case exponent error of an FP16 row, 2^-22 times the weighted
    coefficient bound 4096, is 2^-10 in log2 units, 7e-4 relative in alpha); over all pixels, at
    most 0.01% with a different n_contrib.
"""
import numpy as np

FP32_TOL = 1e-4
FP32_MARGIN = 1e-5
TC_MAXABS = 2.0 / 255.0
TC_PSNR = 45.0
TC_T_TOL = 1e-4
TC_MARGIN = 1e-3
BUDGET = 1e-4  # fraction of pixels that may break a bar (each must be ambiguous)


def psnr(a, b):
    a = np.clip(np.asarray(a, np.float64), 0.0, 1.0)
    b = np.clip(np.asarray(b, np.float64), 0.0, 1.0)
    mse = float(np.mean((a - b) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(1.0 / mse)


def check(precision, rgb, T, nc, ref_rgb, ref_T, ref_nc, margin, what=""):
    """rgb / ref_rgb: [3, ...] or [..., 3] matching; T, nc, margin: per pixel (same shape)."""
    rgb, ref_rgb = np.asarray(rgb, np.float64), np.asarray(ref_rgb, np.float64)
    ch_axis = 0 if rgb.shape[0] == 3 and rgb.shape != T.shape + (3,) else -1
    err = np.abs(rgb - ref_rgb).max(axis=ch_axis)
    terr = np.abs(np.asarray(T, np.float64) - ref_T)
    px = err.size
    allowed = int(np.ceil(BUDGET * px))  # 0.01% of the pixels, at least one
    if precision == "fp32":
        ok = margin > FP32_MARGIN
        assert err[ok].max(initial=0.0) <= FP32_TOL, (what, err[ok].max())
        assert terr[ok].max(initial=0.0) <= FP32_TOL, (what, terr[ok].max())
        assert ((err > FP32_TOL) | (terr > FP32_TOL)).sum() <= allowed, what
        if nc is not None:
            assert np.array_equal(nc[ok], ref_nc[ok]), what
            assert (nc != ref_nc).sum() <= allowed, what
    else:
        assert psnr(rgb, ref_rgb) >= TC_PSNR, (what, psnr(rgb, ref_rgb))
        assert err.max() <= TC_MAXABS, (what, err.max())
        assert terr.max() <= TC_MAXABS, (what, terr.max())
        ok = margin > TC_MARGIN
        assert terr[ok].max(initial=0.0) <= TC_T_TOL, (what, terr[ok].max())
        if nc is not None:
            assert np.array_equal(nc[ok], ref_nc[ok]), what
            assert (nc != ref_nc).sum() <= allowed, (what, int((nc != ref_nc).sum()))
    return err
