"""FP64 CPU reference of projective SDF integration (Section 4.2, Eq. 8-10).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
benchmark's CPU-baseline leg may import this module; the library never does,
and it shares no code with the CUDA path.

For a query point x and a scan j with range image Omega_j and pose
(R_j, t_j) (mapping world points into the scan's sensor frame), Eq. 8 gives
the pixel and the range of the transformed point, [u v r] = Pi(R_j x + t_j),
and Eq. 9 the signed distance along that ray, d_j(x) = Omega_j(u, v) - r
(positive in front of the measured surface).  Eq. 10 fuses the scans by
least squares: d(x) = sum_j d_j / N over the N scans that observe x, which
the running mean d <- d + (d_j - d) / (N + 1) reproduces incrementally.

Readings (the paper leaves these open):
  * a scan observes x when Pi puts it inside the vertical field of view and
    the measured range Omega_j(u, v) is valid (finite, > 0);
  * truncation (the classical practice the paper builds on): with tau > 0 a
    scan whose d_j < -tau (x hidden behind the surface) does not observe x,
    and d_j is clipped to at most tau; tau <= 0 keeps Eq. 10 as printed;
  * query points are voxel centres origin + voxel * (i + 1/2, j + 1/2, k + 1/2)
    of a dense grid stored [k][j][i] (x fastest).
"""
import numpy as np

from .rimg_oracle import project, level_tables, row_margin, NEAR_TIE_PX, NEAR_TIE_ROW

NEAR_TIE_TRUNC = 1e-4      # m: |d_j + tau| below this is a truncation near-tie


def voxel_centres(dims, origin, voxel):
    """Centres of a dense grid, shape (nz, ny, nx, 3), x fastest."""
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    o = np.asarray(origin, np.float64)
    return np.stack([o[0] + voxel * (i + 0.5), o[1] + voxel * (j + 0.5), o[2] + voxel * (k + 0.5)], axis=-1)


def signed_distance(X, rng, T, phi_lut, theta_lut, r0, level=0):
    """Eq. 8-9 for query points X (n, 3) against one scan: returns d (n,),
    observed (n,) and a near-tie flag (n,) for points whose pixel choice lies
    within the near-tie distance of a decision boundary."""
    X = np.asarray(X, np.float64).reshape(-1, 3)
    T = np.asarray(T, np.float64).reshape(4, 4)
    ph, th = level_tables(phi_lut, theta_lut, level)
    rng_l = np.asarray(rng, np.float64)[::1 << level, ::1 << level]
    H, W = rng_l.shape
    Xs = X @ T[:3, :3].T + T[:3, 3]
    u, v, r, fov, det = project(Xs, ph, th, r0, W, return_detail=True)
    meas = rng_l[v, u]
    ok = fov & np.isfinite(meas) & (meas > 0)
    d = np.where(ok, np.where(ok, meas, 0.0) - r, 0.0)
    uc = det["u_c"]
    m_u = np.abs(np.mod(uc, 1.0) - 0.5)
    m_v = row_margin(np.where(np.isfinite(det["phi"]), det["phi"], 0.0), ph)
    near = (m_u < NEAR_TIE_PX) | (m_v < NEAR_TIE_ROW)
    return d, ok, near


def integrate(X, scans, poses, phi_lut, theta_lut, r0, trunc=0.0, level=0, sdf0=None, weight0=None):
    """Eq. 10 over scans (a list of range images) with poses (world -> sensor),
    starting from (sdf0, weight0) (zero by default).  Returns sdf, weight
    (number of observing scans, float) and a near-tie flag per point (any scan
    whose pixel or truncation decision is a near-tie)."""
    X = np.asarray(X, np.float64).reshape(-1, 3)
    n = X.shape[0]
    total = np.zeros(n) if sdf0 is None else np.asarray(sdf0, np.float64).ravel() * np.asarray(weight0).ravel()
    count = np.zeros(n) if weight0 is None else np.asarray(weight0, np.float64).ravel().copy()
    near = np.zeros(n, bool)
    for rng, T in zip(scans, poses):
        d, ok, nt = signed_distance(X, rng, T, phi_lut, theta_lut, r0, level)
        if trunc > 0:
            near |= ok & (np.abs(d + trunc) < NEAR_TIE_TRUNC)
            ok = ok & (d >= -trunc)
            d = np.minimum(d, trunc)
        near |= nt
        total += np.where(ok, d, 0.0)
        count += ok
    sdf = np.where(count > 0, total / np.maximum(count, 1), 0.0)
    return sdf, count, near
