"""Pins of the oracle's near-tie classifier.

Every GPU parity test excuses a GPU/oracle disagreement only where the oracle
flags a near-tie: a source point whose projection (Section 3.2, Eq. 3-4 and
the column rounding of its footnote) or whose association test (Section 4.1,
Eq. 5-6) lies within a small distance of a decision boundary.  These tests
place points at a KNOWN distance from each boundary -- built from the
simulated sensor's own rays, not from the oracle's projection -- and check the
distance the oracle reports and the flag it raises:

* the column boundary u_c = k + 1/2 + delta (pixels), with and without
  azimuth offsets and receiver offset;
* a mid-elevation row boundary of the non-uniform HDL-64-like table, at
  +-delta times the local gap (the gaps on either side differ by 3/2);
* both edges of the vertical field of view;
* the normal-degeneracy threshold |a x b| = 1e-4 |a| |b| (1 +- delta);
* the correspondence-distance gate |x - q| = d_max (1 +- delta);
* the same column / row / edge decisions in the point-cloud imaging and the
  SDF integration, whose truncation test has its own near-tie distance.

A margin off by a factor of two, measured in radians instead of row spacings,
taken from the wrong neighbouring gap, or shifted by half a pixel fails at
least one assertion below."""
import numpy as np
import pytest

from oracle import rimg_oracle as O
from oracle import sdf_oracle as S
from synth import Sensor, hdl64_like_phi, uniform_phi, random_theta

DELTAS = (0.3, -0.3, 0.2, 5e-4, -5e-4, 2e-3, -2e-3, 0.49)


def _point_on_ray(sensor, col, v, r, dphi=0.0):
    """The point at range r along the ray of continuous column `col` (pixels)
    and row v of the simulated sensor, elevation shifted by dphi: the receiver
    sits at column angle 2 pi col / W, the ray leaves at that angle plus
    theta_lut[v] (the physical model the simulator casts rays with)."""
    a = 2.0 * np.pi * col / sensor.W
    el = sensor.phi_lut[v] + dphi
    az = a + sensor.theta_lut[v]
    o = sensor.r0 * np.array([np.cos(a), np.sin(a), 0.0])
    return o + r * np.array([np.cos(az) * np.cos(el), np.sin(az) * np.cos(el), np.sin(el)])


def _flat_target(sensor, r=20.0):
    """A valid target: constant range, every normal valid (pointing back along -x;
    only validity matters for the decisions tested here)."""
    rng = np.full((sensor.H, sensor.W), r)
    n = np.zeros((sensor.H, sensor.W, 3))
    n[..., 0] = -1.0
    return rng, n, np.ones((sensor.H, sensor.W), bool)


def _terms(sensor, X, gate=0.0, target=None):
    rng, n, nv = target if target is not None else _flat_target(sensor)
    return O.icp_terms(np.asarray(X, np.float64).reshape(-1, 3), np.ones(len(np.atleast_2d(X)), bool), np.eye(4),
                       rng, n, nv, sensor.phi_lut, sensor.theta_lut, sensor.r0, 0.5, max_corr_dist=gate)


def _sensors():
    rng = np.random.default_rng(11)
    yield "uniform", Sensor(16, 64, uniform_phi(16, 10.0, -20.0), np.zeros(16), 0.0)
    yield "interlaced_r0", Sensor(16, 64, uniform_phi(16, 10.0, -20.0), random_theta(16, rng, 2.0), 0.015)
    yield "hdl64_like", Sensor(64, 256, hdl64_like_phi(), np.zeros(64), 0.0)


@pytest.mark.parametrize("name,sensor", list(_sensors()))
def test_column_margin_is_distance_to_half_integer(name, sensor):
    """u_c = k + 1/2 + delta: the oracle's column margin is |delta| pixels
    (not radians, not measured from the integer k), the flag is raised exactly
    below NEAR_TIE_PX, and the column is k + 1 for delta >= 0, else k."""
    v = sensor.H // 2
    for k in (0, 5, sensor.W - 1):
        for d in DELTAS:
            X = _point_on_ray(sensor, k + 0.5 + d, v, 17.0, dphi=0.1 * (sensor.phi_lut[v - 1] - sensor.phi_lut[v]))
            t = _terms(sensor, X)
            assert abs(t["margin_u"][0] - abs(d)) < 1e-8, (k, d, t["margin_u"][0])
            assert t["margin_row"][0] > 0.35            # the point sits well inside row v
            assert bool(t["near_tie"][0]) == (abs(d) < O.NEAR_TIE_PX), (k, d)
            u_exp = (k + 1) % sensor.W if d >= 0 else k
            assert t["assoc"][0] == v * sensor.W + u_exp, (k, d, t["assoc"][0])


def test_row_margin_in_local_spacings_on_uneven_table():
    """HDL-64-like table: rows 30 / 31 are 1/3 deg apart, rows 31 / 32 about
    half a degree.  A point delta spacings from either midpoint has margin |delta|
    (in units of that gap, not radians, not the other gap's), and a point on
    a row's own elevation has margin exactly 1/2."""
    s = Sensor(64, 256, hdl64_like_phi(), np.zeros(64), 0.0)
    p = s.phi_lut
    for lo in (30, 31):
        mid = 0.5 * (p[lo] + p[lo + 1])
        gap = p[lo] - p[lo + 1]                       # elevation decreases with the row index
        assert abs(gap - np.deg2rad(1 / 3 if lo == 30 else 0.5)) < np.deg2rad(1e-3)
        for d in DELTAS:
            el = mid - d * gap                        # d > 0: towards row lo + 1
            X = _point_on_ray(s, 7.0, lo, 30.0, dphi=el - p[lo])
            t = _terms(s, X)
            assert abs(t["margin_row"][0] - abs(d)) < 1e-8, (lo, d, t["margin_row"][0])
            assert bool(t["near_tie"][0]) == (abs(d) < O.NEAR_TIE_ROW), (lo, d)
            v_exp = lo + 1 if d > 0 else lo
            assert t["assoc"][0] == v_exp * s.W + 7, (lo, d, t["assoc"][0])
    # on a row's own elevation the nearest boundary is half a gap away on either side
    for v in (1, 20, 31, 32, 50):
        t = _terms(s, _point_on_ray(s, 3.0, v, 30.0))
        assert abs(t["margin_row"][0] - 0.5) < 1e-9, (v, t["margin_row"][0])
    # a factor-of-two or unit mistake would move these values: the direct formula
    m = O.row_margin(np.array([0.5 * (p[30] + p[31]) - 0.25 * (p[30] - p[31])]), p)
    assert abs(m[0] - 0.25) < 1e-12


@pytest.mark.parametrize("edge", ["top", "bottom"])
def test_fov_edge_margin(edge):
    """Half an edge spacing beyond the first / last row is the field-of-view
    edge: a point delta edge-spacings inside is associated, one outside is not,
    and both report margin |delta| (flagged below NEAR_TIE_ROW)."""
    s = Sensor(64, 256, hdl64_like_phi(), np.zeros(64), 0.0)
    p = s.phi_lut
    if edge == "top":
        v, g = 0, p[0] - p[1]
        boundary = p[0] + 0.5 * g
        outward = +1.0
    else:
        v, g = 63, p[62] - p[63]
        boundary = p[63] - 0.5 * g
        outward = -1.0
    for d in DELTAS:
        if abs(d) >= 0.49:
            continue
        el = boundary - outward * d * g               # d > 0: inside the field of view
        X = _point_on_ray(s, 11.0, v, 25.0, dphi=el - p[v])
        t = _terms(s, X)
        assert abs(t["margin_row"][0] - abs(d)) < 1e-8, (d, t["margin_row"][0])
        assert bool(t["near_tie"][0]) == (abs(d) < O.NEAR_TIE_ROW)
        assert (t["assoc"][0] >= 0) == (d > 0), (d, t["assoc"][0])
        lo, hi = O.fov_limits(p)
        assert abs((lo if edge == "bottom" else hi) - boundary) < 1e-15


def _nearly_parallel_setup():
    """A 5 x 16 sensor whose rows 1 and 3 have azimuth offsets that let the
    vertical difference b = P(u, v+1) - P(u, v-1) line up with the horizontal
    one a = P(u+1, v) - P(u-1, v) at pixel (4, 2) for positive ranges.  Returns
    the sensor and the ranges (rL, rR, rU, rD) that make a parallel to b,
    computed from the simulator's rays."""
    phi = np.deg2rad(np.array([17.0, 11.5, 10.0, 9.0, 4.0]))
    th = np.deg2rad(np.array([-3.0, -16.0, -27.0, 10.0, 15.5]))
    s = Sensor(5, 16, phi, th, 0.0)
    _, d = s.rays()
    d = d.reshape(5, 16, 3)
    u, v = 4, 2
    dL, dR, dU, dD = d[v, u - 1], d[v, u + 1], d[v - 1, u], d[v + 1, u]
    m = np.cross(np.cross(dL, dR), np.cross(dU, dD))
    best = None
    for sa in (1.0, -1.0):
        ca = np.linalg.lstsq(np.stack([dR, -dL], 1), sa * m, rcond=None)[0]
        for sb in (1.0, -1.0):
            cb = np.linalg.lstsq(np.stack([dD, -dU], 1), sb * m, rcond=None)[0]
            if np.all(ca > 0) and np.all(cb > 0):
                best = (ca, cb)
    assert best is not None
    ca, cb = best
    ca = 10.0 * ca / ca.max()
    cb = 10.0 * cb / cb.max()
    return s, d, (ca[1], ca[0], cb[1], cb[0])


def _sine(d, rL, rR, rU, rD):
    a = rR * d[2, 5] - rL * d[2, 3]
    b = rD * d[3, 4] - rU * d[1, 4]
    return np.linalg.norm(np.cross(a, b)) / (np.linalg.norm(a) * np.linalg.norm(b))


def test_normal_degeneracy_margin():
    """The cross-product normal is invalid when |a x b| <= 1e-4 |a| |b|.  With
    the lower neighbour's range tuned (bisection on the simulator's rays) so
    that the sine of the angle between a and b is 1e-4 (1 + delta), the
    oracle's relative margin is |delta| and validity is delta > 0."""
    s, d, (rL, rR, rU, rD0) = _nearly_parallel_setup()
    assert _sine(d, rL, rR, rU, rD0) < 1e-12
    for delta in (0.5, -0.5, 0.1, -0.1, 2e-3, -2e-3, 5e-4):
        target = O.NORMAL_SIN_EPS * (1.0 + delta)
        lo, hi = rD0, rD0 * 1.2
        assert _sine(d, rL, rR, rU, hi) > target
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if _sine(d, rL, rR, rU, mid) < target:
                lo = mid
            else:
                hi = mid
        rD = 0.5 * (lo + hi)
        img = np.full((5, 16), 10.0)
        img[2, 3], img[2, 5], img[1, 4], img[3, 4] = rL, rR, rU, rD
        n, ok, margin = O.normals(img, s.phi_lut, s.theta_lut, s.r0, rel_jump=100.0, return_margin=True)
        assert abs(margin[2, 4] - abs(delta)) < 1e-6, (delta, margin[2, 4])
        assert bool(ok[2, 4]) == (delta > 0), delta


def test_gate_margin():
    """With the distance gate on, a source point on the target pixel's own ray
    at |x - q| = d_max (1 + delta) is kept for delta <= 0, and flagged a
    near-tie below a relative distance of 1e-5."""
    s = Sensor(16, 64, uniform_phi(16, 10.0, -20.0), np.zeros(16), 0.0)
    gate = 0.5
    tgt = _flat_target(s, r=20.0)
    for delta in (0.3, -0.3, 2e-5, -2e-5, 5e-6, -5e-6):
        X = _point_on_ray(s, 9.0, 7, 20.0 + gate * (1.0 + delta))
        t = _terms(s, X, gate=gate, target=tgt)
        assert abs(np.linalg.norm(X - O.unproject_pixels(9, 7, 20.0, s.phi_lut, s.theta_lut, 0.0, s.W)) -
                   gate * (1 + delta)) < 1e-12
        assert (t["assoc"][0] >= 0) == (delta <= 0), delta
        assert bool(t["near_tie"][0]) == (abs(delta) < 1e-5), delta


def test_points_to_range_near_mask():
    """Point-cloud imaging: a point delta from a column boundary (or a row
    boundary) marks its pixel and the 8 around it as near-tie pixels exactly
    when |delta| is below the near-tie distance; elsewhere the mask is clear."""
    s = Sensor(16, 64, uniform_phi(16, 10.0, -20.0), random_theta(16, np.random.default_rng(5), 2.0), 0.015)
    v = 6
    for d in DELTAS:
        X = _point_on_ray(s, 20.5 + d, v, 12.0)[None]
        img, near = O.points_to_range(X, s.phi_lut, s.theta_lut, s.r0, s.W)
        u = 21 if d >= 0 else 20
        assert np.isfinite(img[v, u]) and np.isfinite(img).sum() == 1, d
        if abs(d) < O.NEAR_TIE_PX:
            assert near.sum() == 9 and near[v - 1:v + 2, u - 1:u + 2].all(), d
        else:
            assert not near.any(), d
    gap = s.phi_lut[v] - s.phi_lut[v + 1]
    for d in (5e-4, 2e-3):
        X = _point_on_ray(s, 30.0, v, 12.0, dphi=-(0.5 - d) * gap)[None]
        _, near = O.points_to_range(X, s.phi_lut, s.theta_lut, s.r0, s.W)
        assert near.any() == (d < O.NEAR_TIE_ROW), d


def test_sdf_near_flags():
    """SDF integration: a voxel centre delta from a column boundary of the
    scan is flagged iff |delta| < NEAR_TIE_PX; with truncation tau a voxel
    whose signed distance is -tau -+ eps is flagged iff eps < 1e-4 m, and
    observed iff d >= -tau."""
    s = Sensor(16, 64, uniform_phi(16, 10.0, -20.0), np.zeros(16), 0.0)
    scan = np.full((16, 64), 15.0)
    v = 8
    for d in DELTAS:
        X = _point_on_ray(s, 40.5 + d, v, 10.0)[None]
        _, ok, near = S.signed_distance(X, scan, np.eye(4), s.phi_lut, s.theta_lut, s.r0)
        assert ok[0] and bool(near[0]) == (abs(d) < O.NEAR_TIE_PX), d
    tau = 0.3
    for eps in (5e-5, -5e-5, 2e-4, -2e-4):
        r = 15.0 + tau + eps                          # d = 15 - r = -tau - eps
        X = _point_on_ray(s, 40.0, v, r)[None]
        sdf, w, near = S.integrate(X, [scan], [np.eye(4)], s.phi_lut, s.theta_lut, s.r0, trunc=tau)
        assert bool(near[0]) == (abs(eps) < S.NEAR_TIE_TRUNC), eps
        assert (w[0] == 1) == (eps <= 0), eps
