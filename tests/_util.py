"""Shared helpers of the test-suite (comparison statistics, GPU availability)."""
import numpy as np

# Image tolerance (normalised [0, 1] RGBA units): <= 2e-3 max abs on >= 99.9% of pixels,
# <= 2e-2 on every pixel.
TOL_BULK = 2e-3
TOL_ALL = 2e-2
BULK_FRACTION = 0.999


def image_error(gpu_img, ref_img):
    """Per-pixel max-abs error over RGBA; returns (fraction within TOL_BULK, max error)."""
    e = np.abs(np.asarray(gpu_img, np.float64) - np.asarray(ref_img, np.float64)).max(axis=-1)
    return float((e <= TOL_BULK).mean()), float(e.max()), e


def assert_image_parity(gpu_img, ref_img, what=""):
    frac, emax, _ = image_error(gpu_img, ref_img)
    assert frac >= BULK_FRACTION and emax <= TOL_ALL, (
        f"{what}: {100 * frac:.4f}% of pixels within {TOL_BULK}, max error {emax:.3e}")
    return frac, emax


def gpu_available():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False
