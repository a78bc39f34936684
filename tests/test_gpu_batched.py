"""Uneven batches (several image sizes in one rimg_register_groups call)
captured once in a CUDA graph and replayed.

* Replays give poses bit-identical to the eager call (the graph re-runs the
  same kernels with the same launch shapes, so even the FP32 summation order
  is the same), twice in a row, with T_init untouched.
* The replayed poses match the FP64 oracle on one pair of every size, per
  pyramid level (the shadowed check of tests/gpu_common.py).
"""
import numpy as np
import pytest

from synth import CONFIGS, make_pairs
from tests.gpu_common import gpu_sensor, oracle_params, shadowed_check, groups_runner

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = ["mixed32x512_out", "mixed64x1024_in", "mixed128x1024_out", "mixed128x2048_in"]


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_02779_b300.rimg as R
    return R


def _groups(R, counts):
    groups, keep = [], []
    for kind, n in zip(KINDS, counts):
        cfg = CONFIGS[kind]
        s = cfg.sensor()
        sens = gpu_sensor(R, s, cfg.levels)
        src, dst, _ = make_pairs(cfg, range(n), processes=4)
        T0 = torch.eye(4, dtype=torch.float64, device="cuda").reshape(1, 16).repeat(n, 1).contiguous()
        groups.append(dict(src=sens, dst=sens, n_pairs=n, levels=cfg.levels, iters=cfg.iters,
                           params=R.rimg_default_params(huber_delta=cfg.huber_delta),
                           src_range=torch.from_numpy(src).cuda(), dst_range=torch.from_numpy(dst).cuda(),
                           T_init=T0, T_out=torch.empty_like(T0),
                           status=torch.full((n,), -3, dtype=torch.int32, device="cuda")))
        keep.append((cfg, s, src, dst))
    return groups, keep


def test_register_groups_graph_replay(R):
    groups, keep = _groups(R, [5, 3, 2, 2])
    G = R.Groups(groups)
    ws = torch.empty(R.rimg_register_groups_workspace_bytes(G), dtype=torch.uint8, device="cuda")
    side = torch.cuda.Stream()
    # the first call on a device creates the library's internal streams and
    # events, so it runs before the capture
    with torch.cuda.stream(side):
        R.rimg_register_groups(G, ws, side)
    torch.cuda.synchronize()
    eager = [g["T_out"].clone() for g in groups]
    eager_status = [g["status"].clone() for g in groups]
    T_init = [g["T_init"].clone() for g in groups]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        R.rimg_register_groups(G, ws, side)
    for _ in range(2):
        for g in groups:
            g["T_out"].fill_(float("nan"))
            g["status"].fill_(-3)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        for g, e, es, t0 in zip(groups, eager, eager_status, T_init):
            assert torch.equal(g["T_out"], e)
            assert torch.equal(g["status"], es)
            assert torch.equal(g["T_init"], t0)
    # the replayed poses against the oracle, level by level, one pair per size
    for g, (cfg, s, src, dst) in zip(groups, keep):
        rep = shadowed_check(R, torch, g["src"], s, src, dst, cfg.levels, cfg.iters, g["params"], oracle_params(cfg),
                             pairs=[0], final=g["T_out"][:1].cpu().numpy(), runner=groups_runner(R, torch, g))
        print(cfg.name, rep)
