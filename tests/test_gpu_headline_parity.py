"""The headline workload (64x1024, HDL-64-like table, 4 levels x 10) registered
on the GPU against the oracle's registrations of the same 32 pairs, read with
the oracle's own motion at the end of the fixed schedule.

Many pairs of this workload are still moving when the schedule ends (the
last Gauss-Newton step is 1e-5 .. 1e-3): there both runs stop mid-motion and
a near-tie association decided differently by FP32 and FP64 shifts where.
So: a pair whose oracle last step is below 1e-5 (rad and m) must be within
1e-4 rad / 1e-4 m; a pair still moving within 1e-4 + 3 x the geometric tail
last * rho / (1 - rho), rho = last / previous <= 0.95 (at least the last
step) -- the reading the precision study uses."""
import os

import numpy as np
import pytest

from oracle import rimg_oracle as O
from synth import CONFIGS, make_pairs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
CFG = "pair64x1024"
N = 32


def _oracle_one(args):
    src, dst = args
    cfg = CONFIGS[CFG]
    s = cfg.sensor()
    sens = (s.phi_lut, s.theta_lut, s.r0)
    params = dict(huber_delta=float(np.float32(cfg.huber_delta)), max_corr_dist=0.0,
                  normal_rel_jump=float(np.float32(0.1)))
    T, _, poses = O.register(src, dst, sens, sens, np.eye(4), cfg.levels, cfg.iters, params, return_poses=True)
    return T, O.pose_error(poses[-1], poses[-2]), O.pose_error(poses[-2], poses[-3])


def test_headline_pairs_against_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = CONFIGS[CFG]
    src, dst, _ = make_pairs(cfg, range(N), processes=4)
    import multiprocessing as mp
    env = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env}
    os.environ.update({k: "1" for k in env})
    try:
        with mp.get_context("spawn").Pool(max(1, min(16, (os.cpu_count() or 2) - 1))) as pool:
            out = pool.map(_oracle_one, [(src[i], dst[i]) for i in range(N)], chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    import paper_2112_02779_b300.rimg as R
    s = cfg.sensor()
    sens = R.rimg_sensor_build(cfg.H, cfg.W, cfg.levels, s.phi_lut, s.theta_lut, s.r0)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    T0 = torch.eye(4, dtype=torch.float64, device="cuda").reshape(1, 16).repeat(N, 1).contiguous()
    T1 = torch.empty_like(T0)
    ws = torch.empty(R.rimg_register_workspace_bytes(sens, sens, N, cfg.levels), dtype=torch.uint8, device="cuda")
    R.rimg_register(sens, sens, N, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), T0, T1, cfg.levels,
                    cfg.iters, params, None, ws)
    torch.cuda.synchronize()
    Tg = T1.cpu().numpy().reshape(N, 4, 4)
    err = np.array([O.pose_error(Tg[i], out[i][0]) for i in range(N)])
    last = np.array([o[1] for o in out])
    prev = np.array([o[2] for o in out])
    rho = np.minimum(last / np.maximum(prev, 1e-30), 0.95)
    tail = np.maximum(last, last * rho / (1.0 - rho))
    settled = np.all(last < 1e-5, axis=1)
    assert settled.sum() >= 4, settled.sum()
    assert np.all(err[settled] <= 1e-4), err[settled].max(0)
    bar = 1e-4 + 3.0 * tail
    assert np.all(err <= bar), [(i, err[i], bar[i]) for i in range(N) if np.any(err[i] > bar[i])]
    # the typical pair agrees far inside the bar
    assert np.median(err[:, 0]) < 1e-5 and np.median(err[:, 1]) < 1e-4
