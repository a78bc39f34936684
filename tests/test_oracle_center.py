"""Pins of the oracle's initial pose by centre alignment (Section 4.1: the
rotation starts at the identity, the translation aligns the centres of the two
point sets).  Checked against a translated copy of a scan, a closed form for
constant-range images, and the simulated sensor's own rays."""
import numpy as np

from oracle import rimg_oracle as O
from synth import CONFIGS, Sensor, make_pair, uniform_phi, hdl64_like_phi, random_theta


def test_translated_copy_is_recovered():
    """A scan's point set and the same set moved by -t and shuffled: the
    alignment returns [I | t]."""
    cfg = CONFIGS["pair64x1024"]
    s = cfg.sensor()
    dst = make_pair(cfg, 3)["dst_range"]
    P, valid = O.unproject(dst, s.phi_lut, s.theta_lut, s.r0)
    P = P[valid]
    t = np.array([0.7, -1.3, 0.25])
    rng = np.random.default_rng(0)
    P_src = (P - t)[rng.permutation(len(P))]
    T = O.center_align(P_src, P)
    np.testing.assert_array_equal(T[:3, :3], np.eye(3))
    np.testing.assert_allclose(T[:3, 3], t, atol=1e-12)
    np.testing.assert_array_equal(T[3], [0, 0, 0, 1])


def test_constant_range_closed_form():
    """Constant ranges r_s (source) and r_d (target) on a full 360-degree sensor
    with theta_lut = 0: the columns' cos / sin sum to zero (receiver offset
    included), so t = (0, 0, (r_d - r_s) mean_v sin(phi_v))."""
    for r0 in (0.0, 0.02):
        s = Sensor(16, 64, uniform_phi(16, 10.0, -20.0), np.zeros(16), r0)
        rs, rd = 7.0, 11.5
        T, ok = O.center_init(np.full((16, 64), rs), np.full((16, 64), rd), (s.phi_lut, s.theta_lut, r0),
                              (s.phi_lut, s.theta_lut, r0))
        assert ok
        np.testing.assert_allclose(T[:3, 3], [0.0, 0.0, (rd - rs) * np.mean(np.sin(s.phi_lut))], atol=1e-12)


def test_matches_simulated_rays_with_invalid_pixels_and_levels():
    """Against the mean of receiver origin + range * direction over the valid
    pixels, from the simulator's rays (an independent ray model), with
    invalid pixels (0, NaN, inf, negative) excluded and at pyramid levels
    0-2 (strided images and tables)."""
    rng = np.random.default_rng(4)
    for sensor in (Sensor(16, 64, uniform_phi(16, 10.0, -20.0), random_theta(16, rng, 2.0), 0.015),
                   Sensor(64, 256, hdl64_like_phi(), np.zeros(64), 0.0)):
        H, W = sensor.H, sensor.W
        imgs = []
        for _ in range(2):
            r = rng.uniform(0.5, 90.0, (H, W))
            bad = rng.random((H, W))
            r[bad < 0.05] = 0.0
            r[(bad >= 0.05) & (bad < 0.07)] = np.nan
            r[(bad >= 0.07) & (bad < 0.08)] = np.inf
            r[(bad >= 0.08) & (bad < 0.09)] = -3.0
            imgs.append(r)
        sens = (sensor.phi_lut, sensor.theta_lut, sensor.r0)
        for level in (0, 1, 2):
            T, ok = O.center_init(imgs[0], imgs[1], sens, sens, level)
            assert ok
            s = 1 << level
            sub = Sensor(H // s, W // s, sensor.phi_lut[::s], sensor.theta_lut[::s], sensor.r0)
            o, d = sub.rays()
            cents = []
            for r in imgs:
                rl = r[::s, ::s].reshape(-1)
                keep = np.isfinite(rl) & (rl > 0)
                cents.append((o[keep] + rl[keep, None] * d[keep]).mean(axis=0))
            np.testing.assert_allclose(T[:3, 3], cents[1] - cents[0], atol=1e-10)
            np.testing.assert_array_equal(T[:3, :3], np.eye(3))


def test_empty_image_gives_identity():
    s = Sensor(8, 32, uniform_phi(8, 10.0, -20.0), np.zeros(8), 0.0)
    sens = (s.phi_lut, s.theta_lut, s.r0)
    T, ok = O.center_init(np.zeros((8, 32)), np.full((8, 32), 5.0), sens, sens)
    assert not ok and np.array_equal(T, np.eye(4))
