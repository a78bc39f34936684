"""The GPU ray caster of synth.gpu against the numpy ray caster on the same
scenes and poses (noise off), and its noise and dropout statistics."""
import numpy as np
import pytest

from synth import CONFIGS, raycast
from synth import gpu as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_gpu_cast_matches_numpy_cast(cuda):
    cfg = CONFIGS["learn64x1024"]
    idx = [0, 1, 2]
    src, dst, T = G.make_pairs_gpu(cfg, idx, noise=False)
    torch.cuda.synchronize()
    sensor = cfg.sensor()
    for j, i in enumerate(idx):
        W1, W2, dT, ob = G.draw_pair(cfg, i)
        np.testing.assert_array_equal(T[j], dT)
        scene = G.scene_of(ob)
        for img, Wk in ((dst[j], W1), (src[j], W2)):
            ref = raycast(scene, sensor, Wk, cfg.r_min, cfg.r_max)
            got = img.cpu().numpy()
            both = (ref > 0) & (got > 0)
            # float32 vs float64 decide differently only on rays that graze an edge
            assert np.mean((ref > 0) != (got > 0)) < 2e-3
            bad = np.abs(got - ref) > 1e-3 * np.maximum(1.0, ref)
            assert np.mean(bad & both) < 2e-3
            assert both.mean() > 0.5


def test_gpu_noise_and_dropout_statistics(cuda):
    cfg = CONFIGS["learn64x1024"]
    idx = list(range(4))
    s0, d0, _ = G.make_pairs_gpu(cfg, idx, noise=False)
    s1, d1, _ = G.make_pairs_gpu(cfg, idx, noise=True)
    s2, _, _ = G.make_pairs_gpu(cfg, idx, noise=True)
    torch.cuda.synchronize()
    assert torch.equal(s1, s2)                          # keyed by pair: reproducible
    a, b = s0.cpu().numpy(), s1.cpu().numpy()
    valid0 = a > 0
    dropped = valid0 & (b == 0)
    assert abs(dropped.sum() / valid0.sum() - cfg.dropout) < 0.01
    keep = valid0 & (b > 0)
    e = (b - a)[keep]
    assert abs(e.mean()) < 5e-4 and abs(e.std() - cfg.sigma) < 1e-3
    # the source of pair 1 cast alone equals its cast in the batch
    s_one, _, _ = G.make_pairs_gpu(cfg, [1], noise=True)
    torch.cuda.synchronize()
    assert torch.equal(s_one[0], s1[1])
