"""Sensor intrinsic lookup tables (elevation per row, azimuth offset per row).

Row 0 is the top beam (largest elevation), as on a spinning LiDAR whose range
image is stored with the sky at the top.  All angles are radians, float64.
"""
import numpy as np


def uniform_phi(H, top_deg, bottom_deg):
    """H elevations evenly spaced from ``top_deg`` (row 0) to ``bottom_deg`` (row H-1)."""
    return np.deg2rad(np.linspace(top_deg, bottom_deg, H, dtype=np.float64))


def hdl64_like_phi():
    """64 rows in two blocks, like a Velodyne HDL-64: rows 0-31 start at +2 deg in
    -1/3 deg steps (to -8.333 deg); rows 32-63 run linearly from -8.833 deg to
    -24.8 deg.  The exact block layout is an assumption (no datasheet is used)."""
    upper = 2.0 - np.arange(32, dtype=np.float64) / 3.0
    lower = np.linspace(-8.833, -24.8, 32, dtype=np.float64)
    return np.deg2rad(np.concatenate([upper, lower]))


def zero_theta(H):
    """Azimuth offsets of a sensor without interlacing (all zero)."""
    return np.zeros(H, dtype=np.float64)


def random_theta(H, rng, max_deg=2.0):
    """Seeded per-row azimuth offsets, uniform in [-max_deg, +max_deg] degrees."""
    return np.deg2rad(rng.uniform(-max_deg, max_deg, size=H)).astype(np.float64)
