"""GPU parity of the initial pose by centre alignment (Section 4.1: identity
rotation, translation aligning the centres of the two point sets) against the
FP64 oracle, and registrations started from it.

Bar: the rotation is the identity bit for bit; the translation is a pose
component, so it is held to the pose tolerance, 1e-4 m.  (Each GPU point is
within 16 u (r + r0) + 1e-7 m of the oracle's and the FP32 sums run over four
points only, so the centres' errors average these per-point errors; the
observed differences are printed.)"""
import numpy as np
import pytest

from oracle import rimg_oracle as O
from synth import CONFIGS, make_pairs
from tests.gpu_common import gpu_sensor, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_02779_b300.rimg as R
    return R


def _gpu_center(R, sens, level, src, dst):
    n = src.shape[0]
    s = 1 << level
    sl = torch.from_numpy(np.ascontiguousarray(src[:, ::s, ::s])).cuda()
    dl = torch.from_numpy(np.ascontiguousarray(dst[:, ::s, ::s])).cuda()
    T = torch.full((n, 16), 7.0, dtype=torch.float64, device="cuda")
    st = torch.zeros(n, dtype=torch.int32, device="cuda")
    R.rimg_center_init(sens, sens, level, sl, dl, T, st)
    torch.cuda.synchronize()
    return T.cpu().numpy().reshape(n, 4, 4), st.cpu().numpy()


@pytest.mark.parametrize("name,levels", [("pair64x1024", 4), ("lut64x512", 3), ("indoor128x2048", 4)])
def test_center_init_matches_oracle(R, name, levels):
    cfg = CONFIGS[name]
    n = 6
    src, dst, _ = make_pairs(cfg, range(n), processes=4)
    # invalid encodings and one image without a single valid pixel
    src[0, 0, :7] = np.nan
    src[0, 1, :7] = np.inf
    src[0, 2, :7] = -2.0
    dst[n - 1] = 0.0
    s = cfg.sensor()
    sens = gpu_sensor(R, s, levels)
    so = (s.phi_lut, s.theta_lut, s.r0)
    worst = 0.0
    for level in range(levels):
        Tg, st = _gpu_center(R, sens, level, src, dst)
        for i in range(n):
            To, ok = O.center_init(src[i], dst[i], so, so, level)
            assert np.array_equal(Tg[i][:3, :3], np.eye(3)) and np.array_equal(Tg[i][3], [0, 0, 0, 1])
            assert bool(st[i] & R.RIMG_FLAG_DEGENERATE) == (not ok), (level, i, st[i])
            d = np.abs(Tg[i][:3, 3] - To[:3, 3]).max()
            worst = max(worst, d)
            assert d <= 1e-4, (name, level, i, d)
        assert np.array_equal(Tg[n - 1], np.eye(4))
    print(f"{name}: max |t_gpu - t_oracle| = {worst:.3g} m")


def test_center_init_feeds_register(R):
    """The helper's poses are a registration's T_init: the GPU registration
    started from them matches the oracle's registration started from the
    oracle's centre alignment (32 x 512 workload, 3 levels x 10)."""
    cfg = CONFIGS["pair32x512"]
    n = 4
    src, dst, _ = make_pairs(cfg, range(n), processes=4)
    s = cfg.sensor()
    sens = gpu_sensor(R, s, cfg.levels)
    so = (s.phi_lut, s.theta_lut, s.r0)
    ts, td = torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()
    T0 = torch.empty((n, 16), dtype=torch.float64, device="cuda")
    R.rimg_center_init(sens, sens, 0, ts, td, T0)
    T1 = torch.empty_like(T0)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    ws = torch.empty(R.rimg_register_workspace_bytes(sens, sens, n, cfg.levels), dtype=torch.uint8, device="cuda")
    R.rimg_register(sens, sens, n, ts, td, T0, T1, cfg.levels, cfg.iters, params, None, ws)
    torch.cuda.synchronize()
    Tg = T1.cpu().numpy().reshape(n, 4, 4)
    for i in range(n):
        Ti, _ = O.center_init(src[i], dst[i], so, so)
        To, _ = O.register(src[i], dst[i], so, so, Ti, cfg.levels, cfg.iters, oracle_params(cfg))
        eR, et = O.pose_error(Tg[i], To)
        assert eR <= 1e-4 and et <= 1e-4, (i, eR, et)
