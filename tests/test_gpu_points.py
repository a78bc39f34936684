"""Point clouds without scan structure (rimg_points_to_range) against the
oracle's nearest-point projection, on the scan's own sensor and on a
synthetic-intrinsics sensor (theta_lut = 0, rows evenly spread: the mode of
Section 3.2's last paragraph), followed by registration of two such images.

Bars.  Which pixel a point lands on is integer work: the set of filled pixels
is bit-exact away from pixels a near-tie point could reach.  The kept range
is one float32 evaluation of |x - o| (a few roundings): within 8 u r."""
import numpy as np
import pytest

from oracle import rimg_oracle as O
from synth import CONFIGS, Sensor, make_pair, outdoor_scene, raycast, uniform_phi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_02779_b300.rimg as R
    return R


def _cloud(seed, n_extra=20000):
    """Points of a 64x1024 scan (along the simulator's rays), hidden copies
    farther along the same rays, random points and NaNs, shuffled; float32."""
    cfg = CONFIGS["pair64x1024"]
    s = cfg.sensor()
    rng = np.random.default_rng(seed)
    scene = outdoor_scene(rng, 80, 60.0)
    W = np.eye(4)
    W[2, 3] = 1.7
    img = raycast(scene, s, W, 1.0, 60.0, 0.0, 0.1, rng)
    o, d = s.rays()
    t = img.ravel().astype(np.float64)
    ok = t > 0
    X = o[ok] + t[ok, None] * d[ok]
    extra = rng.uniform(-40, 40, size=(n_extra, 3))
    Y = np.concatenate([X, 1.3 * X, extra, np.full((7, 3), np.nan)])
    return Y[rng.permutation(len(Y))].astype(np.float32), s, img


def _compare(got, ref, near):
    far = ~near
    assert np.array_equal(np.isfinite(got[far]), np.isfinite(ref[far]))
    fin = far & np.isfinite(ref)
    assert np.all(np.abs(got[fin] - ref[fin]) <= 8 * U32 * ref[fin])
    assert fin.sum() > 1000


def _synthetic_sensor():
    # 64 rows evenly spread over +2 .. -24.8 deg, theta_lut = 0
    return Sensor(64, 1024, uniform_phi(64, 2.0, -24.8), np.zeros(64), 0.0)


@pytest.mark.parametrize("kind", ["own", "synthetic", "synthetic_posed"])
def test_points_to_range_matches_oracle(R, kind):
    Y, s_own, img = _cloud(1)
    s = s_own if kind == "own" else _synthetic_sensor()
    T = np.eye(4)
    if kind == "synthetic_posed":
        c, sn = np.cos(0.3), np.sin(0.3)
        T[:3, :3] = [[c, -sn, 0], [sn, c, 0], [0, 0, 1]]
        T[:3, 3] = [1.0, -2.0, 0.3]
    sens = R.rimg_sensor_build(s.H, s.W, 1, s.phi_lut, s.theta_lut, s.r0)
    n = Y.shape[0]
    xyz = torch.from_numpy(Y.reshape(1, n, 3)).cuda()
    out = torch.zeros((1, s.H, s.W), device="cuda")
    Td = torch.from_numpy(T.reshape(1, 16)).cuda() if kind == "synthetic_posed" else None
    R.rimg_points_to_range(sens, 0, xyz, out, T_cloud_to_sensor=Td)
    torch.cuda.synchronize()
    Xs = Y.astype(np.float64) @ T[:3, :3].T + T[:3, 3]
    ref, near = O.points_to_range(Xs, s.phi_lut, s.theta_lut, s.r0, s.W)
    got = out[0].cpu().numpy().astype(np.float64)
    _compare(got, ref, near)
    if kind == "own":
        # the scan's points give the scan back wherever no random point is nearer
        scan = np.where(img > 0, img.astype(np.float64), np.inf)
        with np.errstate(invalid="ignore"):
            same = np.isfinite(scan) & ~near & (np.abs(ref - scan) <= 8 * U32 * scan)
        assert same.sum() > 1000
        assert np.all(np.abs(got[same] - scan[same]) <= 16 * U32 * scan[same])


def test_counts_and_batches(R):
    Y, s, _ = _cloud(2, n_extra=0)
    sens = R.rimg_sensor_build(s.H, s.W, 1, s.phi_lut, s.theta_lut, s.r0)
    n = Y.shape[0]
    half = n // 2
    xyz = torch.from_numpy(np.stack([Y, Y])).cuda()
    counts = torch.tensor([n, half], dtype=torch.int32, device="cuda")
    out = torch.zeros((2, s.H, s.W), device="cuda")
    R.rimg_points_to_range(sens, 0, xyz, out, counts=counts)
    torch.cuda.synchronize()
    a, near_a = O.points_to_range(Y[:].astype(np.float64), s.phi_lut, s.theta_lut, s.r0, s.W)
    b, near_b = O.points_to_range(Y[:half].astype(np.float64), s.phi_lut, s.theta_lut, s.r0, s.W)
    _compare(out[0].cpu().numpy().astype(np.float64), a, near_a)
    _compare(out[1].cpu().numpy().astype(np.float64), b, near_b)


def test_registration_of_clouds_through_synthetic_intrinsics(R):
    """Two scans handed over as unordered clouds, imaged through the synthetic
    sensor on the GPU and registered by the same path: the ground-truth motion
    is recovered to a few milliradians / centimetres (re-gridding the 64
    HDL-like beams onto evenly spread rows costs some accuracy -- the data
    loss of synthetic projection that Section 3 describes)."""
    cfg = CONFIGS["pair64x1024"]
    pair = make_pair(cfg, 5)
    s_own = pair["sensor"]
    o, d = s_own.rays()
    clouds = []
    for img in (pair["src_range"], pair["dst_range"]):
        t = img.ravel().astype(np.float64)
        ok = t > 0
        clouds.append((o[ok] + t[ok, None] * d[ok]).astype(np.float32))
    m = max(len(c) for c in clouds)
    xyz = np.full((2, m, 3), np.nan, np.float32)
    for i, c in enumerate(clouds):
        xyz[i, :len(c)] = c
    s = _synthetic_sensor()
    sens = R.rimg_sensor_build(s.H, s.W, 4, s.phi_lut, s.theta_lut, s.r0)
    imgs = torch.zeros((2, s.H, s.W), device="cuda")
    R.rimg_points_to_range(sens, 0, torch.from_numpy(xyz).cuda(), imgs)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    T0 = torch.eye(4, dtype=torch.float64, device="cuda").reshape(1, 16).contiguous()
    T1 = torch.empty_like(T0)
    ws = torch.empty(R.rimg_register_workspace_bytes(sens, sens, 1, 4), dtype=torch.uint8, device="cuda")
    R.rimg_register(sens, sens, 1, imgs[0:1].contiguous(), imgs[1:2].contiguous(), T0, T1, 4, cfg.iters, params,
                    None, ws)
    torch.cuda.synchronize()
    eR, et = O.pose_error(T1.cpu().numpy().reshape(4, 4), pair["T_gt"])
    assert eR < 5e-3 and et < 3e-2, (eR, et)
