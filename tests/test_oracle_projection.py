"""Pins of the oracle's unprojection / projection (Section 3, Eq. 1-4).

Each check compares the oracle with something other than itself: the
simulated sensor's rays (an independent implementation of the ray model),
closed forms, and brute-force searches."""
import numpy as np
import pytest

from oracle import rimg_oracle as O
from synth import Sensor, hdl64_like_phi, uniform_phi, random_theta


def _sensors():
    rng = np.random.default_rng(7)
    yield "uniform_r0=0", Sensor(16, 64, uniform_phi(16, 10.0, -20.0), np.zeros(16), 0.0)
    yield "interlaced_r0", Sensor(16, 64, uniform_phi(16, 10.0, -20.0), random_theta(16, rng, 2.0), 0.015)
    yield "hdl64_like", Sensor(64, 256, hdl64_like_phi(), np.zeros(64), 0.0)
    yield "hdl64_interlaced_r0", Sensor(64, 256, hdl64_like_phi(), random_theta(64, rng, 2.0), 0.03)


@pytest.mark.parametrize("name,sensor", list(_sensors()))
def test_round_trip_lossless(name, sensor):
    """Section 1/3: the LUT model maps pixels to points and back without loss:
    Pi(Pi^-1(u, v, r)) returns the same pixel exactly and the same range."""
    rng = np.random.default_rng(1)
    H, W = sensor.H, sensor.W
    r = rng.uniform(0.5, 100.0, size=(H, W))
    P, valid = O.unproject(r, sensor.phi_lut, sensor.theta_lut, sensor.r0)
    assert valid.all()
    u, v, rr, in_fov = O.project(P, sensor.phi_lut, sensor.theta_lut, sensor.r0, W)
    vv, uu = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    assert in_fov.all()
    assert np.array_equal(v, vv)
    assert np.array_equal(u, uu)
    np.testing.assert_allclose(rr, r, rtol=1e-12)


@pytest.mark.parametrize("name,sensor", list(_sensors()))
def test_unproject_matches_simulated_rays(name, sensor):
    """Eq. 1-2 against the ray model written independently in the simulator:
    point = receiver origin + r * direction."""
    rng = np.random.default_rng(2)
    r = rng.uniform(0.5, 100.0, size=(sensor.H, sensor.W))
    P, _ = O.unproject(r, sensor.phi_lut, sensor.theta_lut, sensor.r0)
    o, d = sensor.rays()
    ref = (o + r.reshape(-1, 1) * d).reshape(sensor.H, sensor.W, 3)
    np.testing.assert_allclose(P, ref, rtol=0, atol=1e-12 * 100)


def _brute_pixel(X, sensor):
    """Brute force over all H x W pixels (r0 = 0): the row whose elevation is
    nearest to the point's (Eq. 4), then within that row the column whose ray
    azimuth is nearest on the circle.  Ray angles come from the simulator."""
    _, d = sensor.rays()
    el = np.arcsin(d[:, 2]).reshape(sensor.H, sensor.W)
    az = np.arctan2(d[:, 1], d[:, 0]).reshape(sensor.H, sensor.W)
    out = []
    for x in X:
        rr = np.linalg.norm(x)
        phi = np.arcsin(x[2] / rr)
        th = np.arctan2(x[1], x[0])
        best = None
        for v in range(sensor.H):
            for u in range(sensor.W):
                dv = abs(el[v, u] - phi)
                dth = abs((az[v, u] - th + np.pi) % (2 * np.pi) - np.pi)
                key = (round(dv, 12), dth, v)
                if best is None or key < best[0]:
                    best = (key, u, v)
        out.append((best[1], best[2]))
    return np.array(out)


def test_projection_equals_brute_force_nearest_pixel():
    """Eq. 3-4 plus the column recovery on a tiny image equal the brute-force
    nearest pixel over all H x W rays (interlaced azimuth table, r0 = 0)."""
    rng = np.random.default_rng(3)
    sensor = Sensor(8, 32, uniform_phi(8, 10.0, -20.0), random_theta(8, rng, 2.0), 0.0)
    pts = []
    while len(pts) < 300:
        th = rng.uniform(-np.pi, np.pi)
        ph = np.deg2rad(rng.uniform(-21.0, 11.0))
        rr = rng.uniform(1.0, 50.0)
        x = rr * np.array([np.cos(th) * np.cos(ph), np.sin(th) * np.cos(ph), np.sin(ph)])
        u, v, _, fov, det = O.project(x[None], sensor.phi_lut, sensor.theta_lut, 0.0, sensor.W,
                                      return_detail=True)
        # stay off decision boundaries so float64 rounding in the brute force
        # cannot flip a choice
        if abs(det["u_c"][0] - np.floor(det["u_c"][0]) - 0.5) < 1e-6:
            continue
        if O.row_margin(det["phi"], sensor.phi_lut)[0] < 1e-6:
            continue
        pts.append(x)
    X = np.array(pts)
    u, v, _, _ = O.project(X, sensor.phi_lut, sensor.theta_lut, 0.0, sensor.W)
    ref = _brute_pixel(X, sensor)
    assert np.array_equal(u, ref[:, 0])
    assert np.array_equal(v, ref[:, 1])


def test_synthetic_intrinsics_closed_form():
    """Section 3.2, last paragraph: with theta_lut = 0 and evenly spaced
    elevations the model reduces to the linear synthetic projection: the row is
    (phi_max - phi) / spacing rounded, the column W theta / 2 pi rounded."""
    H, W = 64, 2048
    top, bot = np.deg2rad(2.0), np.deg2rad(-24.8)
    phi_lut = np.linspace(top, bot, H)
    rng = np.random.default_rng(4)
    n = 20000
    th = rng.uniform(0, 2 * np.pi, n)
    ph = rng.uniform(bot, top, n)
    rr = rng.uniform(1, 80, n)
    X = np.stack([rr * np.cos(th) * np.cos(ph), rr * np.sin(th) * np.cos(ph), rr * np.sin(ph)], -1)
    u, v, r, fov = O.project(X, phi_lut, np.zeros(H), 0.0, W)
    spacing = (top - bot) / (H - 1)
    v_ref = np.clip(np.floor((top - ph) / spacing + 0.5), 0, H - 1).astype(int)
    u_ref = np.mod(np.floor(W * th / (2 * np.pi) + 0.5).astype(int), W)
    away = (np.abs((top - ph) / spacing - np.floor((top - ph) / spacing) - 0.5) > 1e-7) & \
           (np.abs(W * th / (2 * np.pi) - np.floor(W * th / (2 * np.pi)) - 0.5) > 1e-7)
    assert fov.all()
    assert np.array_equal(v[away], v_ref[away])
    assert np.array_equal(u[away], u_ref[away])
    np.testing.assert_allclose(r, rr, rtol=1e-13)


def test_field_of_view_edges():
    """Points more than half an edge spacing above the top row or below the
    bottom row fall outside the image; points just inside land on the edge rows."""
    H, W = 16, 64
    phi_lut = np.deg2rad(np.linspace(10.0, -20.0, H))
    step = np.deg2rad(2.0)
    for ph, expect, row in [(np.deg2rad(10.0) + 0.49 * step, True, 0),
                            (np.deg2rad(10.0) + 0.51 * step, False, None),
                            (np.deg2rad(-20.0) - 0.49 * step, True, H - 1),
                            (np.deg2rad(-20.0) - 0.51 * step, False, None)]:
        x = 10 * np.array([np.cos(ph), 0.0, np.sin(ph)])
        u, v, _, fov = O.project(x[None], phi_lut, np.zeros(H), 0.0, W)
        assert bool(fov[0]) == expect
        if expect:
            assert v[0] == row and u[0] == 0


def _random_monotone_lut(rng, H):
    gaps = rng.uniform(1.0, 1.9, size=H - 1)
    phi = np.concatenate([[0.0], np.cumsum(gaps)])
    phi = np.deg2rad(10.0) - phi / phi[-1] * np.deg2rad(30.0)
    return phi


@pytest.mark.parametrize("seed", range(5))
def test_inverse_lut_2h_within_one_row(seed):
    """Section 3.2: an inverse table with 2H entries bounds the elevation index
    error by +-1 (for tables whose gaps vary by less than 2x); refining the
    candidate over its neighbours gives exactly the Eq. 4 argmin."""
    rng = np.random.default_rng(seed)
    H = int(rng.integers(8, 130))
    phi_lut = _random_monotone_lut(rng, H)
    table, phi0, width = O.inverse_lut_build(phi_lut)
    assert table.shape[0] == 2 * H
    ph = rng.uniform(phi_lut.min(), phi_lut.max(), size=20000)
    exact = O.row_argmin(ph, phi_lut)
    cand = O.inverse_lut_row(ph, table, phi0, width)
    assert np.max(np.abs(cand - exact)) <= 1
    assert np.array_equal(O.inverse_lut_refined(ph, phi_lut, table, phi0, width), exact)


def test_inverse_lut_too_coarse_detected():
    """The +-1 bound is a property of the table size: with too few bins for a
    very uneven table the candidate can be two rows off (so the check above is
    able to fail)."""
    H = 16
    gaps = np.array([1.0] * 8 + [20.0] * 7)
    phi = np.concatenate([[0.0], np.cumsum(gaps)])
    phi_lut = np.deg2rad(10.0) - phi / phi[-1] * np.deg2rad(30.0)
    table, phi0, width = O.inverse_lut_build(phi_lut, n_bins=H // 2)
    ph = np.linspace(phi_lut.min(), phi_lut.max(), 20000)
    cand = O.inverse_lut_row(ph, table, phi0, width)
    assert np.max(np.abs(cand - O.row_argmin(ph, phi_lut))) >= 2


def test_pyramid_keeps_intrinsics_bit_exact():
    """Section 4.1: a pyramid level is the strided image with the original
    intrinsics; its unprojection equals the finest unprojection at
    (2^l u, 2^l v) bit for bit."""
    rng = np.random.default_rng(5)
    H, W = 64, 256
    phi = hdl64_like_phi()
    th = random_theta(H, rng, 2.0)
    r = rng.uniform(0.5, 100, size=(H, W)).astype(np.float32)
    P0, _ = O.unproject(r, phi, th, 0.02)
    for l in range(1, 4):
        Pl, _ = O.source_points(r, phi, th, 0.02, l)
        s = 1 << l
        assert np.array_equal(Pl, P0[::s, ::s])
        pyr = O.pyramid(r, l + 1)
        assert np.array_equal(pyr[l], r[::s, ::s])


def test_pose_error_metric():
    """Section 6.1's metric (trace reading): a z-rotation by a and a shift by d
    give errors (a, |d|)."""
    a = 0.0123
    T = np.eye(4)
    T[:3, :3] = [[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]]
    T[:3, 3] = [0.3, -0.4, 0.0]
    eR, et = O.pose_error(T, np.eye(4))
    assert abs(eR - a) < 1e-9
    assert abs(et - 0.5) < 1e-15
