"""The headline workload (64x1024, HDL-64-like table, 4 levels x 10) registered
on the GPU against the FP64 oracle on 32 pairs, level by level.

Per level (the coarse-to-fine schedule of Section 6.1): the oracle runs the
level from the pose the GPU started it from, and the GPU's level-end pose
must lie within 1e-4 rad and 1e-4 m of the oracle's.  A level that does not
is accepted only when the test itself shows why, step by step (see
tests/gpu_common.shadowed_check and oracle/shadow.py): every GPU association
equals the oracle's at the same pose except on near-tie pixels, every GPU
step equals the oracle's step from the same pose and associations within
1e-6, and the level contains a near-tie decided the other way.  The counts
are printed."""
import json

import numpy as np
import pytest

from oracle import rimg_oracle as O
from synth import CONFIGS, make_pairs
from tests.gpu_common import gpu_sensor, oracle_params, shadowed_check, oracle_pool_map

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
CFG = "pair64x1024"
N = 32


def _oracle_full(args):
    src, dst, sens, levels, iters, params = args
    return O.register(src, dst, sens, sens, np.eye(4), levels, iters, params)[0]


def test_headline_pairs_per_level_against_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_02779_b300.rimg as R
    cfg = CONFIGS[CFG]
    src, dst, _ = make_pairs(cfg, range(N), processes=4)
    s = cfg.sensor()
    sens = gpu_sensor(R, s, cfg.levels)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    rep = shadowed_check(R, torch, sens, s, src, dst, cfg.levels, cfg.iters, params, oracle_params(cfg))
    print(json.dumps(rep))
    assert rep["levels_checked"] == N * cfg.levels
    # every level beyond 1e-4 was explained by the step-by-step reading (the
    # check asserts it); they stay a minority
    assert len(rep["beyond"]) <= 0.1 * rep["levels_checked"]
    # context: the whole registration against the oracle's whole registration
    Tg = []
    T0 = torch.eye(4, dtype=torch.float64, device="cuda").reshape(1, 16).repeat(N, 1).contiguous()
    T1 = torch.empty_like(T0)
    ws = torch.empty(R.rimg_register_workspace_bytes(sens, sens, N, cfg.levels), dtype=torch.uint8, device="cuda")
    R.rimg_register(sens, sens, N, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), T0, T1, cfg.levels,
                    cfg.iters, params, None, ws)
    torch.cuda.synchronize()
    Tg = T1.cpu().numpy().reshape(N, 4, 4)
    so = (s.phi_lut, s.theta_lut, s.r0)
    To = oracle_pool_map(_oracle_full, [(src[i], dst[i], so, cfg.levels, cfg.iters, oracle_params(cfg))
                                        for i in range(N)])
    err = np.array([O.pose_error(Tg[i], To[i]) for i in range(N)])
    print("whole registration: median", np.median(err, 0), "max", err.max(0),
          "within 1e-4:", int(np.sum(np.all(err <= 1e-4, axis=1))))
    assert np.median(err[:, 0]) < 1e-5 and np.median(err[:, 1]) < 1e-4
