"""Seeded scan-pair workloads.

Each pair is two scans of one procedural scene: the *target* from world pose
W1 and the *source* from W2 = W1 * dT.  The ground-truth registration T_gt maps
source-frame points into the target frame, so T_gt = W1^-1 W2 = dT.

Seeds are derived from (config id, pair index, purpose) through numpy's
SeedSequence, so any pair can be regenerated on its own.
"""
from dataclasses import dataclass
import numpy as np

from .luts import uniform_phi, hdl64_like_phi, zero_theta, random_theta
from .scenes import Sensor, outdoor_scene, indoor_scene, raycast, random_delta_pose

_PURPOSE_SCENE, _PURPOSE_POSE, _PURPOSE_NOISE_DST, _PURPOSE_NOISE_SRC, _PURPOSE_LUT = range(5)


@dataclass(frozen=True)
class PairConfig:
    name: str
    config_id: int
    H: int
    W: int
    phi: str                 # "uniform" or "hdl64"
    phi_top_deg: float = 0.0
    phi_bottom_deg: float = 0.0
    theta_max_deg: float = 0.0   # 0: theta_lut == 0
    r0: float = 0.0
    scene: str = "outdoor"       # "outdoor" | "indoor"
    n_objects: int = 20
    r_min: float = 0.5
    r_max: float = 80.0
    rot_max_deg: float = 3.0
    trans_max: float = 0.5
    sigma: float = 0.02
    dropout: float = 0.10
    levels: int = 3
    iters: tuple = (10, 10, 10)  # coarse -> fine
    huber_delta: float = 0.5
    seed_base: int = 0

    def sensor(self):
        if self.phi == "hdl64":
            phi = hdl64_like_phi()
            assert phi.shape[0] == self.H
        else:
            phi = uniform_phi(self.H, self.phi_top_deg, self.phi_bottom_deg)
        if self.theta_max_deg > 0:
            rng = np.random.default_rng(np.random.SeedSequence([self.config_id, 0, _PURPOSE_LUT]))
            theta = random_theta(self.H, rng, self.theta_max_deg)
        else:
            theta = zero_theta(self.H)
        return Sensor(self.H, self.W, phi, theta, self.r0)


CONFIGS = {
    # Small parity case: 32 x 512, uniform +15..-15 deg, 20 objects, 3 levels x 10.
    "pair32x512": PairConfig("pair32x512", 1, 32, 512, "uniform", 15.0, -15.0,
                             n_objects=20, r_min=0.5, r_max=80.0, rot_max_deg=3.0,
                             trans_max=0.5, levels=3, iters=(10, 10, 10), seed_base=1000),
    # Headline workload: 64 x 1024, HDL-64-like elevation table, 200 objects, 4 levels x 10.
    "pair64x1024": PairConfig("pair64x1024", 2, 64, 1024, "hdl64",
                              n_objects=200, r_min=1.0, r_max=120.0, rot_max_deg=5.0,
                              trans_max=1.0, levels=4, iters=(10, 10, 10, 10), seed_base=2000),
    # Precision study: 128 x 2048 indoor rooms, sigma 1 cm, delta 0.2 m.
    "indoor128x2048": PairConfig("indoor128x2048", 3, 128, 2048, "uniform", 22.5, -22.5,
                                 scene="indoor", n_objects=12, r_min=0.3, r_max=40.0,
                                 rot_max_deg=5.0, trans_max=1.0, sigma=0.01, levels=4,
                                 iters=(10, 10, 10, 10), huber_delta=0.2, seed_base=3000),
    # Sizes of the mixed batched workload (rot <= 5 deg, trans <= 1 m), outdoor and indoor.
    "mixed32x512_out": PairConfig("mixed32x512_out", 41, 32, 512, "uniform", 15.0, -15.0,
                                  n_objects=60, r_min=0.5, r_max=80.0, rot_max_deg=5.0, trans_max=1.0,
                                  levels=3, iters=(10, 10, 10), seed_base=4000),
    "mixed32x512_in": PairConfig("mixed32x512_in", 42, 32, 512, "uniform", 15.0, -15.0, scene="indoor",
                                 n_objects=12, r_min=0.3, r_max=40.0, rot_max_deg=5.0, trans_max=1.0,
                                 sigma=0.01, levels=3, iters=(10, 10, 10), huber_delta=0.2, seed_base=4000),
    "mixed64x1024_out": PairConfig("mixed64x1024_out", 43, 64, 1024, "hdl64", n_objects=200, r_min=1.0,
                                   r_max=120.0, rot_max_deg=5.0, trans_max=1.0, levels=4,
                                   iters=(10, 10, 10, 10), seed_base=4000),
    "mixed64x1024_in": PairConfig("mixed64x1024_in", 44, 64, 1024, "hdl64", scene="indoor", n_objects=12,
                                  r_min=0.3, r_max=40.0, rot_max_deg=5.0, trans_max=1.0, sigma=0.01, levels=4,
                                  iters=(10, 10, 10, 10), huber_delta=0.2, seed_base=4000),
    "mixed128x1024_out": PairConfig("mixed128x1024_out", 45, 128, 1024, "uniform", 22.5, -22.5, n_objects=200,
                                    r_min=0.5, r_max=120.0, rot_max_deg=5.0, trans_max=1.0, levels=4,
                                    iters=(10, 10, 10, 10), seed_base=4000),
    "mixed128x1024_in": PairConfig("mixed128x1024_in", 46, 128, 1024, "uniform", 22.5, -22.5, scene="indoor",
                                   n_objects=12, r_min=0.3, r_max=40.0, rot_max_deg=5.0, trans_max=1.0,
                                   sigma=0.01, levels=4, iters=(10, 10, 10, 10), huber_delta=0.2,
                                   seed_base=4000),
    "mixed128x2048_out": PairConfig("mixed128x2048_out", 47, 128, 2048, "uniform", 22.5, -22.5, n_objects=200,
                                    r_min=0.5, r_max=120.0, rot_max_deg=5.0, trans_max=1.0, levels=4,
                                    iters=(10, 10, 10, 10), seed_base=4000),
    "mixed128x2048_in": PairConfig("mixed128x2048_in", 48, 128, 2048, "uniform", 22.5, -22.5, scene="indoor",
                                   n_objects=12, r_min=0.3, r_max=40.0, rot_max_deg=5.0, trans_max=1.0,
                                   sigma=0.01, levels=4, iters=(10, 10, 10, 10), huber_delta=0.2,
                                   seed_base=4000),
    # Learned-proposal workload: the headline sensor and scenes with large
    # motions (rot <= 15 deg, trans <= 3 m); cast on the GPU by synth.gpu.
    "learn64x1024": PairConfig("learn64x1024", 5, 64, 1024, "hdl64",
                               n_objects=200, r_min=1.0, r_max=120.0, rot_max_deg=15.0,
                               trans_max=3.0, levels=4, iters=(10, 10, 10, 10), seed_base=5000),
    # Interlaced sensor with a receiver radius at a realistic size: 64 x 512,
    # theta_lut ~ U(-2, 2) deg, r0 = 1.5 cm (exercises the projection fixed point).
    "lut64x512": PairConfig("lut64x512", 8, 64, 512, "uniform", 10.0, -20.0,
                            theta_max_deg=2.0, r0=0.015, n_objects=100, r_min=0.5, r_max=80.0,
                            rot_max_deg=3.0, trans_max=0.5, levels=3, iters=(10, 10, 10),
                            seed_base=8000),
    # Tiny stress sensor for round trips and LUT handling: interlaced theta,
    # receiver radius; too sparse for stable registration (parity of single
    # steps only).
    "stress16x64": PairConfig("stress16x64", 9, 16, 64, "uniform", 10.0, -20.0,
                              theta_max_deg=2.0, r0=0.015, n_objects=12, r_min=0.5,
                              r_max=60.0, rot_max_deg=3.0, trans_max=0.3, levels=2,
                              iters=(5, 5), seed_base=9000),
}


def make_pair(cfg, index):
    """Return dict(src_range, dst_range float32 [H, W], T_gt float64 4x4, sensor,
    cfg, index).  Deterministic in (cfg.config_id, index)."""
    key = [cfg.config_id, cfg.seed_base + index]
    rng_pose = np.random.default_rng(np.random.SeedSequence(key + [_PURPOSE_POSE]))
    W1 = np.eye(4)
    yaw = rng_pose.uniform(0, 2 * np.pi)
    W1[:3, :3] = np.array([[np.cos(yaw), -np.sin(yaw), 0], [np.sin(yaw), np.cos(yaw), 0], [0, 0, 1]])
    height = 1.7 if cfg.scene == "outdoor" else 1.2
    W1[:3, 3] = [0.0, 0.0, height]
    dT = random_delta_pose(rng_pose, cfg.rot_max_deg, cfg.trans_max)
    if cfg.scene == "indoor":
        # keep both sensors inside the room: place them near its centre
        shift = rng_pose.uniform(-1.0, 1.0, size=2)
        W1[:2, 3] = shift
    W2 = W1 @ dT
    rng_scene = np.random.default_rng(np.random.SeedSequence(key + [_PURPOSE_SCENE]))
    if cfg.scene == "outdoor":
        scene = outdoor_scene(rng_scene, cfg.n_objects, cfg.r_max, keep_clear=(W1[:3, 3], W2[:3, 3]))
    else:
        scene = indoor_scene(rng_scene, cfg.n_objects, keep_clear=(W1[:3, 3], W2[:3, 3]))
        # the room must contain both sensors with a margin
        hx, hy = scene.room[3], scene.room[4]
        lim = min(hx, hy) - 0.5
        for Wk in (W1, W2):
            Wk[:2, 3] = np.clip(Wk[:2, 3], -lim, lim)
        dT = np.linalg.inv(W1) @ W2
    sensor = cfg.sensor()
    rng_d = np.random.default_rng(np.random.SeedSequence(key + [_PURPOSE_NOISE_DST]))
    rng_s = np.random.default_rng(np.random.SeedSequence(key + [_PURPOSE_NOISE_SRC]))
    dst = raycast(scene, sensor, W1, cfg.r_min, cfg.r_max, cfg.sigma, cfg.dropout, rng_d)
    src = raycast(scene, sensor, W2, cfg.r_min, cfg.r_max, cfg.sigma, cfg.dropout, rng_s)
    return dict(src_range=src, dst_range=dst, T_gt=dT, sensor=sensor, cfg=cfg, index=index)


def _make_pair_star(args):
    name, idx = args
    p = make_pair(CONFIGS[name], idx)
    return p["src_range"], p["dst_range"], p["T_gt"]


def make_pairs(cfg, indices, processes=1):
    """Generate several pairs; returns (src [n,H,W] f32, dst [n,H,W] f32, T_gt [n,4,4]).
    With processes > 1 a 'spawn' pool is used (safe after CUDA initialisation)."""
    indices = list(indices)
    if processes > 1 and len(indices) > 1:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        with ctx.Pool(processes) as pool:
            out = pool.map(_make_pair_star, [(cfg.name, i) for i in indices], chunksize=4)
    else:
        out = [_make_pair_star((cfg.name, i)) for i in indices]
    src = np.stack([o[0] for o in out]) if out else np.zeros((0, cfg.H, cfg.W), np.float32)
    dst = np.stack([o[1] for o in out]) if out else np.zeros((0, cfg.H, cfg.W), np.float32)
    T = np.stack([o[2] for o in out]) if out else np.zeros((0, 4, 4))
    return src, dst, T


MIXED_KINDS = ["mixed32x512_out", "mixed32x512_in", "mixed64x1024_out", "mixed64x1024_in",
               "mixed128x1024_out", "mixed128x1024_in", "mixed128x2048_out", "mixed128x2048_in"]


def mixed_batch_plan(n_pairs, seed=4000):
    """The uneven batched workload: each of n_pairs pairs draws its size
    uniformly from {32x512, 64x1024, 128x1024, 128x2048} and its scene from
    outdoor / indoor (50/50).  Returns {kind: [pair indices]} (pair index i
    of a kind is generated with make_pair(CONFIGS[kind], i))."""
    rng = np.random.default_rng(np.random.SeedSequence([50, seed]))
    kinds = rng.integers(0, len(MIXED_KINDS), size=n_pairs)
    plan = {}
    for j, k in enumerate(kinds):
        plan.setdefault(MIXED_KINDS[k], []).append(j)
    return plan
