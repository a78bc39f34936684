"""Pins of the oracle's point-cloud projection (Section 3.2, last paragraph:
clouds without scan structure enter the same path through Pi): a scan turned
into points along the simulator's own rays projects back onto itself (the
lossless round trip of Section 3), the nearest point wins a pixel, and point
order and non-finite points do not matter."""
import numpy as np

from oracle import rimg_oracle as O
from synth import Sensor, outdoor_scene, raycast, uniform_phi, random_theta


def _scan(r0, theta, seed=0):
    H, W = 32, 256
    phi = uniform_phi(H, 10.0, -20.0)
    th = random_theta(H, np.random.default_rng(seed), 2.0) if theta else np.zeros(H)
    s = Sensor(H, W, phi, th, r0)
    rng = np.random.default_rng(seed)
    scene = outdoor_scene(rng, 30, 40.0)
    img = raycast(scene, s, np.diag([1.0, 1.0, 1.0, 1.0]) + np.array([[0, 0, 0, 0], [0, 0, 0, 0], [0, 0, 0, 1.7],
                                                                         [0, 0, 0, 0]]), 0.5, 40.0)
    o, d = s.rays()
    t = img.ravel().astype(np.float64)
    ok = t > 0
    X = o[ok] + t[ok, None] * d[ok]
    return s, img, X, ok


def test_scan_points_project_back_onto_the_scan():
    for r0, theta in ((0.0, False), (0.02, True)):
        s, img, X, ok = _scan(r0, theta)
        got, near = O.points_to_range(X, s.phi_lut, s.theta_lut, s.r0, s.W)
        want = np.where(img > 0, img.astype(np.float64), np.inf)
        assert not near.any()
        fin = np.isfinite(want)
        assert np.array_equal(np.isfinite(got), fin)
        np.testing.assert_allclose(got[fin], want[fin], rtol=1e-12)


def test_nearest_point_wins_and_order_and_nan_do_not_matter():
    s, img, X, ok = _scan(0.0, False, seed=3)
    rng = np.random.default_rng(1)
    far = X * 1.5                                   # the same rays, farther away (hidden)
    junk = np.full((10, 3), np.nan)
    Y = np.concatenate([far, X, junk])
    Y = Y[rng.permutation(len(Y))]
    got, _ = O.points_to_range(Y, s.phi_lut, s.theta_lut, s.r0, s.W)
    ref, _ = O.points_to_range(X, s.phi_lut, s.theta_lut, s.r0, s.W)
    assert np.array_equal(got, ref)
