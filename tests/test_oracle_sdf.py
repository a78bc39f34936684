"""Pins of the FP64 projective-SDF oracle (Section 4.2, Eq. 8-10) against
closed forms: points placed on a pixel's own ray in front of / behind an
analytic wall, whose signed distance along the ray is (c - n.x) / (n.dir);
the least-squares fusion of two scans; the world -> sensor pose convention;
truncation; invalid and out-of-view pixels; the voxel-centre ordering."""
import numpy as np

from oracle import sdf_oracle as S
from synth import Sensor, uniform_phi, random_theta


def _sensor(r0, theta=False):
    H, W = 16, 64
    phi = uniform_phi(H, 10.0, -20.0)
    th = random_theta(H, np.random.default_rng(1), 2.0) if theta else np.zeros(H)
    return Sensor(H, W, phi, th, r0)


def _wall_image(sensor, c, pos=np.zeros(3)):
    """Range image of the plane x = c seen from a sensor at `pos` (identity
    orientation): t = (c - o_x) / d_x along each pixel ray."""
    o, d = sensor.rays()
    o = o + pos
    with np.errstate(divide="ignore"):
        t = np.where(d[:, 0] > 1e-9, (c - o[:, 0]) / d[:, 0], 0.0)
    return t.reshape(sensor.H, sensor.W)


def _on_ray_points(sensor, rng, n):
    """n (pixel, rho) samples and the points o + rho * dir on those pixel rays
    (pixels facing +x so that the wall is in view)."""
    o, d = sensor.rays()
    idx = np.nonzero(d[:, 0] > 0.5)[0]
    pick = rng.choice(idx, size=n, replace=False)
    rho = rng.uniform(2.0, 20.0, size=n)
    return pick, rho, o[pick] + rho[:, None] * d[pick], d[pick]


def test_signed_distance_along_the_ray_closed_form():
    rng = np.random.default_rng(0)
    for r0, theta in ((0.0, False), (0.03, True)):
        s = _sensor(r0, theta)
        c = 10.0
        img = _wall_image(s, c)
        pick, rho, X, dirs = _on_ray_points(s, rng, 200)
        d, ok, near = S.signed_distance(X, img, np.eye(4), s.phi_lut, s.theta_lut, s.r0)
        assert ok.all() and not near.any()
        np.testing.assert_allclose(d, (c - X[:, 0]) / dirs[:, 0], rtol=0, atol=1e-9)


def test_least_squares_fusion_of_two_scans():
    rng = np.random.default_rng(1)
    s = _sensor(0.0)
    a, b = _wall_image(s, 10.0), _wall_image(s, 10.5)
    pick, rho, X, dirs = _on_ray_points(s, rng, 100)
    sdf, w, near = S.integrate(X, [a, b], [np.eye(4)] * 2, s.phi_lut, s.theta_lut, s.r0)
    assert np.all(w == 2) and not near.any()
    want = 0.5 * (a.ravel()[pick] + b.ravel()[pick]) - rho
    np.testing.assert_allclose(sdf, want, atol=1e-9)
    # incremental form: integrating b on top of (sdf, w) after a gives the same
    s1, w1, _ = S.integrate(X, [a], [np.eye(4)], s.phi_lut, s.theta_lut, s.r0)
    s2, w2, _ = S.integrate(X, [b], [np.eye(4)], s.phi_lut, s.theta_lut, s.r0, sdf0=s1, weight0=w1)
    np.testing.assert_allclose(s2, sdf, atol=1e-12)
    assert np.array_equal(w2, w)


def test_pose_maps_world_points_into_the_sensor_frame():
    rng = np.random.default_rng(2)
    s = _sensor(0.0)
    p = np.array([3.0, -1.0, 0.5])                   # sensor position in the world
    img = _wall_image(s, 10.0, pos=p)                # the wall x = 10 in the world
    pick, rho, Xs, dirs = _on_ray_points(s, rng, 100)
    Xw = Xs + p
    T = np.eye(4)
    T[:3, 3] = -p                                    # world -> sensor
    d, ok, _ = S.signed_distance(Xw, img, T, s.phi_lut, s.theta_lut, s.r0)
    assert ok.all()
    np.testing.assert_allclose(d, (10.0 - Xw[:, 0]) / dirs[:, 0], atol=1e-9)


def test_truncation_invalid_pixels_and_field_of_view():
    rng = np.random.default_rng(3)
    s = _sensor(0.0)
    img = _wall_image(s, 10.0)
    pick, rho, X, dirs = _on_ray_points(s, rng, 200)
    tau = 0.3
    sdf, w, _ = S.integrate(X, [img], [np.eye(4)], s.phi_lut, s.theta_lut, s.r0, trunc=tau)
    d = img.ravel()[pick] - rho
    assert np.all(w[d < -tau] == 0)
    seen = d >= -tau
    np.testing.assert_allclose(sdf[seen], np.minimum(d[seen], tau), atol=1e-9)
    # an invalid measured range hides the pixel
    bad = img.copy()
    bad.ravel()[pick[:50]] = 0.0
    _, w2, _ = S.integrate(X[:50], [bad], [np.eye(4)], s.phi_lut, s.theta_lut, s.r0)
    assert np.all(w2 == 0)
    # a point far above the vertical field of view (+10 deg) is not observed
    _, w3, _ = S.integrate(np.array([[5.0, 0.0, 5.0]]), [img], [np.eye(4)], s.phi_lut, s.theta_lut, s.r0)
    assert w3[0] == 0


def test_voxel_centres_are_x_fastest():
    C = S.voxel_centres((3, 2, 4), (1.0, -2.0, 0.5), 0.25)
    assert C.shape == (4, 2, 3, 3)
    np.testing.assert_allclose(C[0, 0, 0], [1.125, -1.875, 0.625])
    np.testing.assert_allclose(C[3, 1, 2], [1.0 + 0.25 * 2.5, -2.0 + 0.25 * 1.5, 0.5 + 0.25 * 3.5])
    flat = C.reshape(-1, 3)
    np.testing.assert_allclose(flat[1] - flat[0], [0.25, 0, 0])
