"""Levels on thread-block clusters: with schedule C = 2, 4 or 8
(rimg_autotune_set), every iteration of a level runs in one launch with each
pair on a cluster of C blocks, which exchange their FP32 block sums through
distributed shared memory and each run the same FP64 update.  The arithmetic
and its order are those of C blocks per pair in per-iteration launches (one
association launch with the last-block FP64 sum, one solve launch), so the
registrations must agree bit for bit with that schedule -- on every level,
those that fit one block and the finest level of the 64 x 1024 sensor, which
does not -- on every projection form: the branch-free form (32 x 512 and the
headline 64 x 1024 sensor), the general form with azimuth offsets and a
receiver offset (interlaced 64 x 512), and plain FP32 accumulation; for
batches of several pairs and of one pair.  The cluster schedule is also
checked level by level against the FP64 oracle (the shadowed per-level
check)."""
import json

import numpy as np
import pytest

from synth import CONFIGS, make_pairs
from tests.gpu_common import gpu_register, gpu_sensor, oracle_params, shadowed_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_CHUNKS = 4096   # a level fits one block up to this many four-pixel chunks per pair


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_02779_b300.rimg as R
    yield R
    R.rimg_autotune_clear()


def _fitting_levels(cfg):
    return [l for l in range(cfg.levels) if (cfg.H >> l) * ((cfg.W >> l) // 4) <= MAX_CHUNKS]


def _perturbed(n, seed):
    rng = np.random.default_rng(seed)
    T = np.tile(np.eye(4), (n, 1, 1))
    for i in range(n):
        a = rng.uniform(-0.02, 0.02)
        c, s = np.cos(a), np.sin(a)
        T[i, :2, :2] = [[c, -s], [s, c]]
        T[i, :3, 3] = rng.uniform(-0.1, 0.1, 3)
    return T


CASES = {
    "pair32x512": ("pair32x512", 6, {}),
    "pair64x1024": ("pair64x1024", 4, {}),
    "pair64x1024_one_pair": ("pair64x1024", 1, {}),
    "lut64x512_offsets_r0": ("lut64x512", 3, {}),
    "pair32x512_plain_fp32": ("pair32x512", 3, dict(kahan=0)),
}


@pytest.mark.parametrize("C", [2, 4, 8])
@pytest.mark.parametrize("case", list(CASES))
def test_cluster_schedule_equals_per_iteration_launches(R, case, C):
    name, n, kw = CASES[case]
    cfg = CONFIGS[name]
    s = cfg.sensor()
    sens = gpu_sensor(R, s, cfg.levels)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta, **kw)
    src, dst, _ = make_pairs(cfg, range(n), processes=4)
    T0 = _perturbed(n, 5)
    R.rimg_autotune_clear()
    try:
        for l in range(cfg.levels):   # per-iteration launches, 128 threads, C blocks per pair
            R.rimg_autotune_set(cfg.H >> l, cfg.W >> l, n, 128, C, 0)
        Ta, sa = gpu_register(R, torch, sens, src, dst, T0, cfg.levels, cfg.iters, params)
        for l in range(cfg.levels):   # every level on clusters of C blocks
            R.rimg_autotune_set(cfg.H >> l, cfg.W >> l, n, 0, 0, C)
        Tb, sb = gpu_register(R, torch, sens, src, dst, T0, cfg.levels, cfg.iters, params)
        R.rimg_autotune_clear()
        Tc, _ = gpu_register(R, torch, sens, src, dst, T0, cfg.levels, cfg.iters, params)
    finally:
        R.rimg_autotune_clear()
    assert np.array_equal(sa, sb)
    assert np.array_equal(Ta, Tb), np.abs(Ta - Tb).max()
    # against the default schedule (one block per pair): another summation
    # order, the same registrations up to FP32 rounding of the sums
    assert np.abs(Tb - Tc).max() < 1e-3


def test_cluster_schedule_per_level_parity(R):
    """The headline sensor with its three small levels on clusters of four
    blocks and its finest level on clusters of eight, level by level against
    the oracle."""
    cfg = CONFIGS["pair64x1024"]
    n = 4
    s = cfg.sensor()
    sens = gpu_sensor(R, s, cfg.levels)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    src, dst, _ = make_pairs(cfg, range(n), processes=4)
    R.rimg_autotune_clear()
    try:
        fit = _fitting_levels(cfg)
        assert fit == [1, 2, 3]
        for l in range(cfg.levels):
            R.rimg_autotune_set(cfg.H >> l, cfg.W >> l, n, 0, 0, 4 if l in fit else 8)
        rep = shadowed_check(R, torch, sens, s, src, dst, cfg.levels, cfg.iters, params, oracle_params(cfg))
    finally:
        R.rimg_autotune_clear()
    print(json.dumps({k: rep[k] for k in ("pairs", "levels_checked", "max_err", "explained", "by_kind")}))
    assert rep["levels_checked"] == n * cfg.levels
