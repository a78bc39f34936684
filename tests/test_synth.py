"""The seeded input generator: deterministic, shaped like the workloads."""
import numpy as np

from synth import CONFIGS, make_pair, make_pairs


def test_pairs_are_deterministic_and_distinct():
    cfg = CONFIGS["pair32x512"]
    a, b, c = make_pair(cfg, 3), make_pair(cfg, 3), make_pair(cfg, 4)
    assert np.array_equal(a["src_range"], b["src_range"])
    assert np.array_equal(a["T_gt"], b["T_gt"])
    assert not np.array_equal(a["src_range"], c["src_range"])


def test_workload_statistics():
    for name, lo, hi in (("pair32x512", 0.5, 80.0), ("pair64x1024", 1.0, 120.0)):
        cfg = CONFIGS[name]
        p = make_pair(cfg, 0)
        for img in (p["src_range"], p["dst_range"]):
            assert img.shape == (cfg.H, cfg.W) and img.dtype == np.float32
            v = img[img > 0]
            assert v.min() >= lo - 0.2 and v.max() <= hi + 0.2
            # dropout alone invalidates ~10 % of pixels
            assert 0.05 < (img == 0).mean() < 0.6
        R = p["T_gt"][:3, :3]
        ang = np.degrees(np.arccos(np.clip((np.trace(R) - 1) / 2, -1, 1)))
        assert ang <= cfg.rot_max_deg + 1e-9
        assert np.linalg.norm(p["T_gt"][:3, 3]) <= cfg.trans_max + 1e-9


def test_make_pairs_stacks():
    src, dst, T = make_pairs(CONFIGS["stress16x64"], range(3))
    assert src.shape == (3, 16, 64) and dst.shape == (3, 16, 64) and T.shape == (3, 4, 4)
