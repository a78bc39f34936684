"""Pins of the oracle's normals, normal equations, solve, SE(3) update and
registration (Section 4.1, Eq. 5-7)."""
import numpy as np
import pytest
import scipy.linalg

from oracle import rimg_oracle as O
from synth import CONFIGS, Sensor, make_pair, uniform_phi, random_theta, hdl64_like_phi
from tests.conftest import f32


def _plane_ranges(sensor, n, c):
    """Float64 ranges of the plane n.x = c from the simulator's rays (inf/neg -> 0)."""
    o, d = sensor.rays()
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (c - o @ n) / (d @ n)
    t = np.where(np.isfinite(t) & (t > 0) & (t < 500), t, 0.0)
    return t.reshape(sensor.H, sensor.W)


@pytest.mark.parametrize("r0", [0.0, 0.015])
def test_normals_exact_on_plane(r0):
    """On an analytic plane the neighbour cross product is the plane normal (up
    to rounding), oriented towards the sensor."""
    rng = np.random.default_rng(11)
    sensor = Sensor(32, 128, uniform_phi(32, 5.0, -25.0), random_theta(32, rng, 1.0), r0)
    n_pl = np.array([0.2, -0.1, 1.0])
    n_pl /= np.linalg.norm(n_pl)
    r = _plane_ranges(sensor, n_pl, -1.7)
    n, ok = O.normals(r, sensor.phi_lut, sensor.theta_lut, r0, 0.5)
    assert ok.sum() > 500
    # the sensor (origin) lies on the positive side: n_pl . 0 = 0 > -1.7, so the
    # normal facing it is +n_pl
    err = np.abs(n[ok] - n_pl[None, :]).max()
    assert err < 1e-9


def test_normals_cylinder_second_order():
    """Inside a vertical cylinder whose axis is off the sensor centre the normal
    is -(p_xy - c)/Rc; central differences make the error second order in the
    angular step, so halving the step cuts it about 4x."""
    errs = []
    c = np.array([2.5, -1.0])
    Rc = 8.0
    for W in (256, 512):
        sensor = Sensor(32, W, uniform_phi(32, 10.0, -10.0), np.zeros(32), 0.0)
        o, d = sensor.rays()
        # |o_xy + t d_xy - c| = Rc, far root
        px, py = o[:, 0] - c[0], o[:, 1] - c[1]
        a = d[:, 0] ** 2 + d[:, 1] ** 2
        b = 2 * (px * d[:, 0] + py * d[:, 1])
        cc = px * px + py * py - Rc * Rc
        t = (-b + np.sqrt(b * b - 4 * a * cc)) / (2 * a)
        r = t.reshape(sensor.H, sensor.W)
        n, ok = O.normals(r, sensor.phi_lut, sensor.theta_lut, 0.0, 0.5)
        P, _ = O.unproject(r, sensor.phi_lut, sensor.theta_lut, 0.0)
        ref = -np.stack([P[..., 0] - c[0], P[..., 1] - c[1], 0 * P[..., 2]], -1) / Rc
        errs.append(np.abs(n[ok] - ref[ok]).max())
    assert errs[0] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_normals_agree_with_window_pca_on_plane():
    """The smallest-eigenvalue eigenvector of the 3x3-window covariance (the
    paper's alternative normal estimator) agrees with the cross product on a
    plane.  Eigenvectors come from numpy's symmetric eigensolver."""
    sensor = Sensor(16, 64, uniform_phi(16, 5.0, -25.0), np.zeros(16), 0.0)
    n_pl = np.array([0.1, 0.3, 1.0])
    n_pl /= np.linalg.norm(n_pl)
    r = _plane_ranges(sensor, n_pl, -2.0)
    n, ok = O.normals(r, sensor.phi_lut, sensor.theta_lut, 0.0, 0.5)
    P, _ = O.unproject(r, sensor.phi_lut, sensor.theta_lut, 0.0)
    checked = 0
    for v in range(1, 15):
        for u in range(64):
            if not ok[v, u]:
                continue
            win = np.array([P[v + dv, (u + du) % 64] for dv in (-1, 0, 1) for du in (-1, 0, 1)])
            C = np.cov(win.T)
            w, V = np.linalg.eigh(C)
            e = V[:, 0]
            assert min(np.abs(e - n[v, u]).max(), np.abs(e + n[v, u]).max()) < 1e-9
            checked += 1
    assert checked > 100


def test_normals_validity_rules():
    """Rows 0 and H-1 are invalid; a depth jump above rel_jump * r_c or an
    invalid neighbour invalidates the pixel; the jump test is inclusive."""
    sensor = Sensor(8, 64, uniform_phi(8, 5.0, -25.0), np.zeros(8), 0.0)
    r = _plane_ranges(sensor, np.array([1.0, 0.0, 0.0]), 10.0)     # wall x = 10
    n, ok = O.normals(r, sensor.phi_lut, sensor.theta_lut, 0.0, 0.1)
    assert not ok[0].any() and not ok[-1].any()
    v, u = 5, 1
    assert ok[v, u]
    np.testing.assert_allclose(n[v, u], [-1.0, 0.0, 0.0], atol=1e-12)
    r2 = r.copy()
    r2[v, u + 1] = 0.0                    # invalid right neighbour
    _, ok2 = O.normals(r2, sensor.phi_lut, sensor.theta_lut, 0.0, 0.1)
    assert not ok2[v, u] and not ok2[v, u + 2] and not ok2[v, u + 1]
    r3 = r.copy()
    r3[v + 1, u] = r[v, u] * 1.25         # depth jump of 25 %
    _, ok3 = O.normals(r3, sensor.phi_lut, sensor.theta_lut, 0.0, 0.1)
    assert not ok3[v, u]
    r4 = r.astype(np.float32)
    rc = np.float32(r4[v, u])
    jump = np.float32(0.125)
    r4[v, u + 1] = rc + jump * rc          # exactly at the threshold: kept
    _, ok4 = O.normals(r4, sensor.phi_lut, sensor.theta_lut, 0.0, float(jump))
    assert ok4[v, u]
    r4[v, u + 1] = np.nextafter(rc + jump * rc, np.float32(np.inf))   # one ulp above
    _, ok5 = O.normals(r4, sensor.phi_lut, sensor.theta_lut, 0.0, float(jump))
    assert not ok5[v, u]


def test_se3_exp_matches_matrix_exponential():
    """Exp of a twist equals scipy's matrix exponential of [[hat(w), tau], [0, 0]],
    including the small-angle branch."""
    rng = np.random.default_rng(12)
    for scale in (1.0, 1e-3, 1e-9, 0.0):
        xi = rng.normal(size=6) * scale
        M = np.zeros((4, 4))
        M[:3, :3] = O.hat(xi[:3])
        M[:3, 3] = xi[3:]
        np.testing.assert_allclose(O.se3_exp(xi), scipy.linalg.expm(M), atol=1e-14, rtol=1e-12)


def test_cholesky_solve_matches_lapack_and_flags_degenerate():
    rng = np.random.default_rng(13)
    A = rng.normal(size=(6, 6))
    Hm = A @ A.T + 0.1 * np.eye(6)
    g = rng.normal(size=6)
    x, ok = O.cholesky_solve(Hm, g)
    assert ok
    np.testing.assert_allclose(x, np.linalg.solve(Hm, -g), rtol=1e-10)
    Hd = np.zeros((6, 6))
    Hd[:5, :5] = np.eye(5)
    x, ok = O.cholesky_solve(Hd, g)
    assert not ok and not x.any()


def test_pseudo_huber_weight_is_irls_of_the_kernel():
    """The oracle's per-point weight times residual equals the derivative of
    rho(e) = d^2 (sqrt(1 + (e/d)^2) - 1) (central differences), i.e. it is the
    IRLS weight of the pseudo-Huber kernel of size d."""
    p, s, tgt = _scene_target()
    d = f32(0.5)
    rng_l, n_l, nv_l, ph, th = tgt.level(1)
    P, sv = O.source_points(p["src_range"], s.phi_lut, s.theta_lut, s.r0, 1)
    terms = O.icp_terms(P, sv, np.eye(4), rng_l, n_l, nv_l, ph, th, s.r0, d)
    ok = terms["w"] > 0
    e, w = terms["e"][ok], terms["w"][ok]
    assert np.abs(e).max() > d          # residuals on both sides of the kernel size
    rho = lambda x: d * d * (np.sqrt(1 + (x / d) ** 2) - 1)
    h = 1e-6
    np.testing.assert_allclose(w * e, (rho(e + h) - rho(e - h)) / (2 * h), atol=1e-8)
    assert np.isclose(terms["sum_wr2"], np.sum(w * e * e))


def _scene_target(cfg_name="pair32x512", idx=0, levels=3):
    cfg = CONFIGS[cfg_name]
    p = make_pair(cfg, idx)
    s = p["sensor"]
    tgt = O.Target(p["dst_range"], s.phi_lut, s.theta_lut, s.r0, levels, f32(0.1))
    return p, s, tgt


def _objective(xi, X, n, q, w):
    T = O.se3_exp(xi)
    Xp = X @ T[:3, :3].T + T[:3, 3]
    e = np.sum(n * (Xp - q), axis=-1)
    return 0.5 * np.sum(w * e * e)


def test_gradient_and_hessian_match_finite_differences():
    """J^T W e is the gradient of F(xi) = 1/2 sum w (n.(Exp(xi) x - q))^2 at a
    fixed association (central differences, FP64); at zero residual J^T W J is
    its Hessian.  A dropped term, wrong sign or transposed operand in J, H or
    g fails here."""
    p, s, tgt = _scene_target()
    rng_l, n_l, nv_l, ph, th = tgt.level(0)
    P, sv = O.source_points(p["src_range"], s.phi_lut, s.theta_lut, s.r0, 0)
    T = np.eye(4)
    terms = O.icp_terms(P, sv, T, rng_l, n_l, nv_l, ph, th, s.r0, 0.5)
    ok = terms["w"] > 0
    X = terms["X"][ok]
    assoc = terms["assoc"][ok]
    v, u = assoc // rng_l.shape[1], assoc % rng_l.shape[1]
    q = O.unproject_pixels(u, v, rng_l[v, u], ph, th, s.r0, rng_l.shape[1])
    n = n_l[v, u]
    w = terms["w"][ok]
    h = 1e-6
    g_fd = np.array([(_objective(h * np.eye(6)[k], X, n, q, w) - _objective(-h * np.eye(6)[k], X, n, q, w)) / (2 * h)
                     for k in range(6)])
    np.testing.assert_allclose(terms["g"], g_fd, rtol=1e-6, atol=1e-6 * np.abs(terms["g"]).max())
    # zero-residual configuration: move the targets onto the source points' planes
    q0 = q + (np.sum(n * (X - q), axis=-1))[:, None] * n
    e0 = np.sum(n * (X - q0), axis=-1)
    assert np.abs(e0).max() < 1e-9
    J = np.concatenate([np.cross(X, n), n], axis=-1)
    H_ref = (J * w[:, None]).T @ J
    Hfd = np.zeros((6, 6))
    hh = 1e-4
    f0 = _objective(np.zeros(6), X, n, q0, w)
    for i in range(6):
        for j in range(6):
            ei, ej = hh * np.eye(6)[i], hh * np.eye(6)[j]
            Hfd[i, j] = (_objective(ei + ej, X, n, q0, w) - _objective(ei - ej, X, n, q0, w)
                         - _objective(-ei + ej, X, n, q0, w) + _objective(-ei - ej, X, n, q0, w)) / (4 * hh * hh)
    np.testing.assert_allclose(Hfd, H_ref, rtol=2e-3, atol=2e-3 * np.abs(H_ref).max())
    # and the oracle's H is that same J^T W J
    np.testing.assert_allclose(terms["H"], H_ref, rtol=1e-12, atol=1e-9)


def test_pack29_layout():
    Hm = np.arange(36, dtype=float).reshape(6, 6)
    Hm = Hm + Hm.T
    t = dict(H=Hm, g=np.arange(6.0), sum_wr2=7.5, count=42)
    v = O.pack29(t)
    assert v.shape == (29,)
    assert v[0] == Hm[0, 0] and v[5] == Hm[0, 5] and v[6] == Hm[1, 1] and v[20] == Hm[5, 5]
    assert np.array_equal(v[21:27], np.arange(6.0)) and v[27] == 7.5 and v[28] == 42


def _rz(a):
    T = np.eye(4)
    T[:2, :2] = [[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]]
    return T


def test_recovers_known_transform_point_set():
    """Source points = T_gt^-1 applied to the target's own points: every residual
    vanishes at T_gt, so Gauss-Newton must land on T_gt (to 1e-6)."""
    rng = np.random.default_rng(14)
    from synth.scenes import random_delta_pose
    p, s, tgt = _scene_target("pair32x512", 3, levels=3)
    T_gt = random_delta_pose(rng, 3.0, 0.3)
    Tinv = np.linalg.inv(T_gt)
    T = np.eye(4)
    for l, iters in ((2, 10), (1, 10), (0, 15)):
        rng_l, n_l, nv_l, ph, th = tgt.level(l)
        Q, qv = O.unproject(rng_l, ph, th, s.r0)
        P = Q.reshape(-1, 3) @ Tinv[:3, :3].T + Tinv[:3, 3]
        for _ in range(iters):
            terms = O.icp_terms(P, qv.reshape(-1), T, rng_l, n_l, nv_l, ph, th, s.r0, 0.5)
            T, ok = O.gn_update(T, terms)
            assert ok
    eR, et = O.pose_error(T, T_gt)
    assert eR < 1e-6 and et < 1e-6


def test_recovers_column_shift_as_yaw():
    """The target image with its columns rolled by k is the same scene seen
    after a yaw of 2 pi k / W (theta_lut = 0, r0 = 0): multi-scale registration
    of the pair returns exactly that rotation."""
    cfg = CONFIGS["pair32x512"]
    p = make_pair(cfg, 5)
    s = p["sensor"]
    k = 4
    dst = p["dst_range"]
    src = np.roll(dst, -k, axis=1)        # src(u, v) = dst(u + k, v)
    T_gt = _rz(2 * np.pi * k / s.W)
    sens = (s.phi_lut, s.theta_lut, s.r0)
    T, deg = O.register(src, dst, sens, sens, np.eye(4), 3, (10, 10, 10),
                        dict(huber_delta=f32(0.5), normal_rel_jump=f32(0.1)))
    assert not deg
    eR, et = O.pose_error(T, T_gt)
    assert eR < 1e-6 and et < 1e-6


@pytest.mark.parametrize("idx", [0, 1])
def test_register_noisy_pair_lands_near_ground_truth(idx):
    """End-to-end poses on noisy pairs have no closed form; the oracle must at
    least land within the noise level of the generator's T_gt."""
    cfg = CONFIGS["pair32x512"]
    p = make_pair(cfg, idx)
    s = p["sensor"]
    sens = (s.phi_lut, s.theta_lut, s.r0)
    T, deg = O.register(p["src_range"], p["dst_range"], sens, sens, np.eye(4), cfg.levels, cfg.iters,
                        dict(huber_delta=f32(cfg.huber_delta), normal_rel_jump=f32(0.1)))
    e0 = O.pose_error(np.eye(4), p["T_gt"])
    eR, et = O.pose_error(T, p["T_gt"])
    assert eR < 0.2 * e0[0] + 2e-3 and et < 0.2 * e0[1] + 1e-2


def test_degenerate_system_leaves_pose_unchanged():
    """Fewer than 6 correspondences: the update is skipped."""
    sensor = Sensor(8, 32, uniform_phi(8, 5.0, -25.0), np.zeros(8), 0.0)
    r = np.zeros((8, 32), np.float32)
    tgt = O.Target(r, sensor.phi_lut, sensor.theta_lut, 0.0, 1, f32(0.1))
    P, sv = O.source_points(r, sensor.phi_lut, sensor.theta_lut, 0.0, 0)
    T0 = _rz(0.1)
    T, ok, terms = O.icp_step(P, sv, tgt, 0, T0, dict(huber_delta=0.5))
    assert not ok and terms["count"] == 0
    assert np.array_equal(T, T0)


def test_gauss_newton_step_is_left_update_quadratic():
    """Far from the identity the update must compose on the left (the Jacobian
    is that of a left perturbation): from 1e-3 rad / 1e-3 m off a large T_gt
    one step lands within 1e-5 of it (quadratic convergence); composing on the
    wrong side would leave an error of the order of the rotation times the
    large translation."""
    p, s, tgt = _scene_target("pair32x512", 2, levels=1)
    T_gt = _rz(1.3)
    T_gt[:3, 3] = [3.0, -2.0, 0.4]
    Tinv = np.linalg.inv(T_gt)
    rng_l, n_l, nv_l, ph, th = tgt.level(0)
    Q, qv = O.unproject(rng_l, ph, th, s.r0)
    P = Q.reshape(-1, 3) @ Tinv[:3, :3].T + Tinv[:3, 3]
    T = O.se3_exp(np.array([1e-3, -1e-3, 5e-4, 1e-3, 1e-3, -1e-3])) @ T_gt
    e0 = O.pose_error(T, T_gt)
    terms = O.icp_terms(P, qv.reshape(-1), T, rng_l, n_l, nv_l, ph, th, s.r0, 0.5)
    T1, ok = O.gn_update(T, terms)
    e1 = O.pose_error(T1, T_gt)
    assert ok and e0[0] > 1e-3
    assert e1[0] < 1e-5 and e1[1] < 1e-5
