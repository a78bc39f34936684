"""Pins of the oracle's PCA normals (the eigen-decomposition alternative of
Section 4.1): exact on analytic planes, equal to the smallest right singular
vector of each window's centred points (an independent LAPACK routine), and
the window rules (range jumps leave the window, too few points invalidate)."""
import numpy as np

from oracle import rimg_oracle as O
from synth import CONFIGS, Sensor, make_pair, uniform_phi, random_theta


def _sensor(r0=0.0, theta=False):
    H, W = 16, 128
    phi = uniform_phi(H, 10.0, -20.0)
    th = random_theta(H, np.random.default_rng(4), 2.0) if theta else np.zeros(H)
    return Sensor(H, W, phi, th, r0)


def _plane_image(s, n, c):
    """Range image of the plane n . p = c along the sensor's rays."""
    o, d = s.rays()
    den = d @ n
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(den > 1e-6, (c - o @ n) / den, 0.0)
    return np.where(t > 0, t, 0.0).reshape(s.H, s.W)


def test_exact_on_planes():
    for r0, theta in ((0.0, False), (0.02, True)):
        s = _sensor(r0, theta)
        for nvec, c in (((1.0, 0.0, 0.0), 10.0), ((0.6, 0.0, 0.8), 6.0), ((0.3, -0.5, 0.1), 4.0)):
            nv = np.asarray(nvec) / np.linalg.norm(nvec)
            img = _plane_image(s, nv, c)
            n, ok = O.normals_pca(img, s.phi_lut, s.theta_lut, s.r0, 0.1)
            assert ok.sum() > 50
            np.testing.assert_allclose(n[ok], np.broadcast_to(-nv, n[ok].shape), atol=1e-9)


def test_matches_svd_of_each_window():
    cfg = CONFIGS["pair32x512"]
    p = make_pair(cfg, 1)
    s = p["sensor"]
    rng_img = p["dst_range"]
    n, ok, det = O.normals_pca(rng_img, s.phi_lut, s.theta_lut, s.r0, 0.1, return_detail=True)
    P, valid = O.unproject(rng_img.astype(np.float64), s.phi_lut, s.theta_lut, s.r0)
    r = np.where(valid, rng_img.astype(np.float64), 0.0)
    rng = np.random.default_rng(0)
    vs, us = np.nonzero(ok)
    pick = rng.choice(len(vs), size=300, replace=False)
    for v, u in zip(vs[pick], us[pick]):
        pts = []
        for dv in (-1, 0, 1):
            for du in (-1, 0, 1):
                vv, uu = v + dv, (u + du) % s.W
                if valid[vv, uu] and abs(r[vv, uu] - r[v, u]) <= 0.1 * r[v, u]:
                    pts.append(P[vv, uu])
        Q = np.asarray(pts) - np.mean(pts, axis=0)
        _, sv, Vt = np.linalg.svd(Q)
        assert len(pts) == det["count"][v, u]
        assert abs(abs(np.dot(Vt[-1], n[v, u])) - 1.0) < 1e-9
        np.testing.assert_allclose(np.sort(sv ** 2), det["lam"][v, u], rtol=1e-9, atol=1e-12)


def test_window_rules():
    s = _sensor()
    # two walls at 10 m and 12 m meeting at a step in azimuth
    a = _plane_image(s, np.array([1.0, 0.0, 0.0]), 10.0)
    b = _plane_image(s, np.array([1.0, 0.0, 0.0]), 12.0)
    img = np.where(np.arange(s.W)[None, :] < 4, a, b)
    n, ok = O.normals_pca(img, s.phi_lut, s.theta_lut, s.r0, 0.1)
    n_x, ok_x = O.normals(img, s.phi_lut, s.theta_lut, s.r0, 0.1)
    # at the step the cross product is invalid; the window drops the other
    # wall's points and still fits the pixel's own wall
    v = 8
    for u in (3, 4):
        assert not ok_x[v, u] and ok[v, u]
        np.testing.assert_allclose(n[v, u], [-1.0, 0.0, 0.0], atol=1e-9)
    # a single valid row leaves three points per window: invalid
    one = np.zeros_like(a)
    one[8] = a[8]
    _, ok1 = O.normals_pca(one, s.phi_lut, s.theta_lut, s.r0, 0.1)
    assert not ok1.any()
