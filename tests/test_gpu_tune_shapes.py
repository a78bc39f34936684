"""Every launch shape the autotuner can pick, pinned by rimg_autotune_set,
against the untuned shape: the association step's 29 sums over the same
pixels at the same pose.  The association count is an exact integer and must
match exactly (a shape that dropped or repeated a chunk would change it); the
other sums, summed in another order, within FP32 rounding.

Shapes: 128 and 256 threads per block, 1, 2, 4, ... H_l blocks per pair (the
tuner's candidates), on every level of the 32 x 512 workload (branch-free
projection, row-stride cursors where the thread stride is whole rows), of
the interlaced 64 x 512 sensor (general projection) and of the 64 x 1024
headline sensor, for batches of one pair and of 40 pairs, at the identity and
at a perturbed pose."""
import numpy as np
import pytest

from synth import CONFIGS, make_pairs
from tests.gpu_common import gpu_sensor, planes_for, src_pyramid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_02779_b300.rimg as R
    return R


def _pose(n, perturb):
    T = np.tile(np.eye(4), (n, 1, 1))
    if perturb:
        a = 0.01
        c, s = np.cos(a), np.sin(a)
        T[:, :2, :2] = [[c, -s], [s, c]]
        T[:, :3, 3] = [0.05, -0.03, 0.01]
    return torch.from_numpy(T.reshape(n, 16).copy()).cuda()


def _sums(R, sens, level, n, src_l, planes_l, pose, params):
    out = torch.zeros((n, 29), dtype=torch.float64, device="cuda")
    ws = torch.empty(R.rimg_icp_workspace_bytes(sens, n), dtype=torch.uint8, device="cuda")
    R.rimg_icp_step(sens, sens, level, n, src_l, planes_l, None, pose.clone(), params, 0, out, None, None, ws)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("cfg_name", ["pair32x512", "lut64x512", "pair64x1024"])
@pytest.mark.parametrize("n", [1, 40])
def test_every_tuner_shape_gives_the_same_sums(R, cfg_name, n):
    cfg = CONFIGS[cfg_name]
    s = cfg.sensor()
    sens = gpu_sensor(R, s, cfg.levels)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    src, dst, _ = make_pairs(cfg, [i % 8 for i in range(n)], processes=4)
    src_t = torch.from_numpy(src).cuda()
    dst_t = torch.from_numpy(dst).cuda()
    planes, _ = planes_for(R, torch, sens, dst_t, params)
    srcl = src_pyramid(R, torch, sens, src_t)
    R.rimg_autotune_clear()
    checked = 0
    try:
        for level in range(cfg.levels):
            Hl, Wl = cfg.H >> level, cfg.W >> level
            for perturb in (False, True):
                pose = _pose(n, perturb)
                R.rimg_autotune_clear()
                ref = _sums(R, sens, level, n, srcl[level], planes[level], pose, params)
                assert np.all(ref[:, 28] > 0)
                scale = np.abs(ref).max(axis=0) + 1.0
                for threads in (128, 256):
                    b = 1
                    while b <= Hl:
                        R.rimg_autotune_set(Hl, Wl, n, threads, b, -1)
                        got = _sums(R, sens, level, n, srcl[level], planes[level], pose, params)
                        where = (cfg_name, n, level, perturb, threads, b)
                        assert np.array_equal(got[:, 28], ref[:, 28]), where
                        err = np.abs(got - ref) / scale
                        assert err.max() <= 2e-5, (where, err.max(axis=0))
                        checked += 1
                        b *= 2
    finally:
        R.rimg_autotune_clear()
    assert checked >= cfg.levels * 2 * 2


def test_autotune_set_rejects_bad_arguments(R):
    for args in [(0, 64, 1, 128, 1, -1), (16, 64, 0, 128, 1, -1), (16, 64, 1, 192, 1, -1), (16, 64, 1, 128, 0, -1),
                 (16, 64, 1, 128, 17, -1), (16, 64, 1, 128, 1, 3), (16, 64, 1, 128, 1, 5), (16, 64, 1, 128, 1, -2)]:
        with pytest.raises(R.RimgError):
            R.rimg_autotune_set(*args)
    for s in (0, 1, 2, 4, 8):
        R.rimg_autotune_set(16, 64, 1, 0, 0, s)
    R.rimg_autotune_clear()
