"""Projective SDF integration on the GPU (rimg_sdf_integrate) against the FP64
oracle (Section 4.2, Eq. 8-10).

Bars.  The observation count of a voxel is integer work: bit-exact wherever
no scan's pixel or truncation decision is a near-tie (reading 17), and
different by at most the number of near-tie scans elsewhere.  The SDF value
is an FP32 mean of FP32 signed distances: the voxel centre, the rigid
transform and r = |x - o| each carry a few float32 roundings of coordinates
of size |x| + |t| (world) and r, so |d_gpu - d_oracle| <= 32 u (|x| + |t| + r_max)
+ 1e-6 m with u = 2^-24; the bar below uses r_max = 120 m for every voxel."""
import numpy as np
import pytest

from oracle import sdf_oracle as S
from synth import CONFIGS, outdoor_scene, raycast

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_02779_b300.rimg as R
    return R


def _sequence(cfg_name, n_scans, seed):
    """n_scans range images of one outdoor scene from a sensor moving along x
    with small yaw changes; returns (sensor, images [n,H,W], world poses).
    cfg_name: a workload name or a PairConfig."""
    cfg = CONFIGS[cfg_name] if isinstance(cfg_name, str) else cfg_name
    sensor = cfg.sensor()
    rng = np.random.default_rng(seed)
    poses = []
    for k in range(n_scans):
        W = np.eye(4)
        yaw = 0.05 * k
        W[:3, :3] = [[np.cos(yaw), -np.sin(yaw), 0], [np.sin(yaw), np.cos(yaw), 0], [0, 0, 1]]
        W[:3, 3] = [0.8 * k, 0.3 * np.sin(k), 1.7]
        poses.append(W)
    scene = outdoor_scene(rng, 60, 40.0, keep_clear=[p[:3, 3] for p in poses])
    imgs = np.stack([raycast(scene, sensor, W, cfg.r_min, 40.0, cfg.sigma, cfg.dropout, rng) for W in poses])
    return sensor, imgs, poses


def _check(sdf_g, w_g, sdf_o, w_o, near, X, T_ws, n_scans):
    w_g, sdf_g = w_g.ravel(), sdf_g.ravel()
    far = ~near
    assert np.array_equal(w_g[far], w_o[far])
    assert np.all(np.abs(w_g[near] - w_o[near]) <= n_scans)
    both = far & (w_o > 0)
    tmax = max(np.linalg.norm(T[:3, 3]) for T in T_ws)
    bar = 32 * U32 * (np.linalg.norm(X, axis=1) + tmax + 120.0) + 1e-6
    err = np.abs(sdf_g[both] - sdf_o[both])
    assert np.all(err <= bar[both]), (err.max(), np.argmax(err / bar[both]))
    assert both.sum() > 1000


def _r0_fast_config():
    """The 32 x 512 sensor (uniform elevations, theta_lut = 0, power-of-two
    width, so an exact inverse table) with a receiver offset r0 = 1.5 cm: the
    branch-free projection inside the receiver-offset fixed point."""
    import dataclasses
    return dataclasses.replace(CONFIGS["pair32x512"], name="pair32x512_r0", config_id=91, r0=0.015)


@pytest.mark.parametrize("cfg_name,level,trunc", [("pair64x1024", 0, 0.5), ("pair64x1024", 1, 0.0),
                                                   ("lut64x512", 0, 0.3), ("r0_fast", 0, 0.3),
                                                   ("r0_fast", 1, 0.0)])
def test_sdf_matches_oracle(R, cfg_name, level, trunc):
    n = 6
    if cfg_name == "r0_fast":
        cfg_name = _r0_fast_config()
        s0 = cfg_name.sensor()
        sens0 = R.rimg_sensor_build(s0.H, s0.W, 2, s0.phi_lut, s0.theta_lut, s0.r0)
        L = sens0.struct.level[level]
        # the launch takes the branch-free form: exact table, no azimuth offsets, power-of-two width
        assert L.bins_exact and not L.has_theta and (L.W & (L.W - 1)) == 0 and s0.r0 > 0
    sensor, imgs, poses = _sequence(cfg_name, n, seed=11)
    T_ws = [np.linalg.inv(W) for W in poses]
    dims, origin, voxel = (64, 48, 16), (-6.0, -6.0, -0.5), 0.25
    X = S.voxel_centres(dims, origin, voxel).reshape(-1, 3)
    lv = imgs[:, ::1 << level, ::1 << level]
    sdf_o, w_o, near = S.integrate(X, list(imgs), T_ws, sensor.phi_lut, sensor.theta_lut, sensor.r0, trunc=trunc,
                                   level=level)
    sens = R.rimg_sensor_build(sensor.H, sensor.W, 2, sensor.phi_lut, sensor.theta_lut, sensor.r0)
    rng_d = torch.from_numpy(np.ascontiguousarray(lv)).cuda()
    T_d = torch.from_numpy(np.stack(T_ws).reshape(n, 16)).cuda()
    sdf = torch.zeros((dims[2], dims[1], dims[0]), device="cuda")
    w = torch.zeros_like(sdf)
    # two calls (scans 0-2, then 3-5): the state carries the running mean
    R.rimg_sdf_integrate(sens, level, rng_d[:3], T_d[:3], dims, origin, voxel, sdf, w, trunc=trunc)
    R.rimg_sdf_integrate(sens, level, rng_d[3:], T_d[3:], dims, origin, voxel, sdf, w, trunc=trunc)
    torch.cuda.synchronize()
    _check(sdf.cpu().numpy(), w.cpu().numpy(), sdf_o, w_o, near, X, T_ws, n)


def test_sdf_one_call_equals_oracle_and_empty_calls_are_noops(R):
    n = 4
    sensor, imgs, poses = _sequence("pair64x1024", n, seed=5)
    T_ws = [np.linalg.inv(W) for W in poses]
    dims, origin, voxel = (40, 40, 12), (-4.0, -5.0, -0.2), 0.2
    X = S.voxel_centres(dims, origin, voxel).reshape(-1, 3)
    sdf_o, w_o, near = S.integrate(X, list(imgs), T_ws, sensor.phi_lut, sensor.theta_lut, sensor.r0, trunc=0.4)
    sens = R.rimg_sensor_build(sensor.H, sensor.W, 1, sensor.phi_lut, sensor.theta_lut, sensor.r0)
    rng_d = torch.from_numpy(imgs).cuda()
    T_d = torch.from_numpy(np.stack(T_ws).reshape(n, 16)).cuda()
    sdf = torch.zeros((dims[2], dims[1], dims[0]), device="cuda")
    w = torch.zeros_like(sdf)
    R.rimg_sdf_integrate(sens, 0, rng_d, T_d, dims, origin, voxel, sdf, w, trunc=0.4)
    R.rimg_sdf_integrate(sens, 0, rng_d, T_d, dims, origin, voxel, sdf, w, trunc=0.4, n_scans=0)
    R.rimg_sdf_integrate(sens, 0, rng_d, T_d, (0, 40, 12), origin, voxel, sdf, w, trunc=0.4)
    torch.cuda.synchronize()
    _check(sdf.cpu().numpy(), w.cpu().numpy(), sdf_o, w_o, near, X, T_ws, n)
    # surface consistency: voxels the scans see on both sides of the ground
    # plane z = 0 change sign across it
    s = sdf.cpu().numpy()
    wv = w.cpu().numpy()
    col = (wv[0] > 0) & (wv[3] > 0)                  # z = -0.1 m and z = +0.5 m
    assert np.mean(s[0][col] < 0) > 0.9 and np.mean(s[3][col] > 0) > 0.9
