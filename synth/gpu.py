"""Seeded scan pairs cast on the GPU (for training sets of 10^5 pairs).

Pair i of a configuration is drawn on the host from numpy generators seeded
by (config id, seed_base + i, purpose), like synth.configs.make_pair, but with
the objects drawn as arrays (rejected objects redrawn together), and cast by
the CUDA ray caster of csrc/raycast.cu (float32, one ray per pixel, the same
rays and primitives as synth.scenes.raycast).  Range noise and dropout come
from a counter-based hash on the device instead of numpy draws, so a pair cast
here equals the numpy cast of the same scene up to float32 rounding before
noise, and has the same noise statistics after it.

Relative poses: rotation axis uniform on the sphere, angle U(0, rot_max);
translation magnitude U(0, trans_max) along a direction drawn uniformly on the
sphere whose vertical component is then scaled by 0.1 (and the direction
renormalised), so that a 3 m displacement keeps the 1.7 m high sensor above
the ground.
"""
import ctypes
import os

import numpy as np

from .scenes import Scene

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsynth.so")
MAX_OBJ = 512
_PURPOSE_SCENE, _PURPOSE_POSE = 0, 1
_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsynth.so not built ({LIB_PATH}); run `python -m synth.build`")
        _lib = ctypes.CDLL(LIB_PATH)
        f = _lib.synth_raycast
        f.restype = ctypes.c_int
        vp = ctypes.c_void_p
        f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_float, vp, vp, ctypes.c_int, vp,
                      ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, vp, vp, vp]
    return _lib


def _rotation(axis, angle):
    K = np.array([[0.0, -axis[2], axis[1]], [axis[2], 0.0, -axis[0]], [-axis[1], axis[0], 0.0]])
    return np.eye(3) + np.sin(angle) * K + (1.0 - np.cos(angle)) * K @ K


def _unit(rng):
    while True:
        a = rng.normal(size=3)
        n = np.linalg.norm(a)
        if n > 1e-6:
            return a / n


def level_delta_pose(rng, rot_max_deg, trans_max, vertical=0.1):
    T = np.eye(4)
    T[:3, :3] = _rotation(_unit(rng), np.deg2rad(rng.uniform(0, rot_max_deg)))
    d = _unit(rng) * np.array([1.0, 1.0, vertical])
    T[:3, 3] = d / np.linalg.norm(d) * rng.uniform(0, trans_max)
    return T


def outdoor_objects(rng, n_objects, r_max, keep, margin=1.5):
    """n_objects boxes / cylinders (50/50) with centres 3 .. 0.8 r_max m from
    the origin, none within `margin` of a point in `keep` (xy); records as in
    csrc/raycast.cu."""
    keep = np.asarray(keep, dtype=np.float64).reshape(-1, 2)
    rec = np.zeros((n_objects, 8))
    todo = np.arange(n_objects)
    for _ in range(1000):
        if todo.size == 0:
            break
        m = todo.size
        rad = rng.uniform(3.0, 0.8 * r_max, m)
        ang = rng.uniform(0, 2 * np.pi, m)
        cx, cy = rad * np.cos(ang), rad * np.sin(ang)
        box = rng.random(m) < 0.5
        hx, hy = rng.uniform(0.5, 6.0, m) / 2, rng.uniform(0.5, 6.0, m) / 2
        yaw = rng.uniform(0, 2 * np.pi, m)
        rr = rng.uniform(0.2, 1.5, m)
        h = rng.uniform(1.0, 6.0, m)
        bound = np.where(box, np.hypot(hx, hy), rr)
        dist = np.min(np.hypot(cx[:, None] - keep[None, :, 0], cy[:, None] - keep[None, :, 1]), axis=1)
        ok = dist >= bound + margin
        r = np.zeros((m, 8))
        r[:, 0] = np.where(box, 0.0, 1.0)
        r[:, 1], r[:, 2] = cx, cy
        r[:, 3] = np.where(box, np.cos(yaw), rr)
        r[:, 4] = np.where(box, np.sin(yaw), h)
        r[:, 5] = np.where(box, hx, 0.0)
        r[:, 6] = np.where(box, hy, 0.0)
        r[:, 7] = np.where(box, h, 0.0)
        rec[todo[ok]] = r[ok]
        todo = todo[~ok]
    if todo.size:
        raise RuntimeError("could not place every object")
    return rec


def draw_pair(cfg, index):
    """(W1, W2, T_gt, objects float64 [n_objects][8]) of pair `index`."""
    key = [cfg.config_id, cfg.seed_base + index]
    rng_pose = np.random.default_rng(np.random.SeedSequence(key + [_PURPOSE_POSE]))
    W1 = np.eye(4)
    yaw = rng_pose.uniform(0, 2 * np.pi)
    W1[:3, :3] = np.array([[np.cos(yaw), -np.sin(yaw), 0], [np.sin(yaw), np.cos(yaw), 0], [0, 0, 1]])
    W1[:3, 3] = [0.0, 0.0, 1.7]
    dT = level_delta_pose(rng_pose, cfg.rot_max_deg, cfg.trans_max)
    W2 = W1 @ dT
    rng_scene = np.random.default_rng(np.random.SeedSequence(key + [_PURPOSE_SCENE]))
    obj = outdoor_objects(rng_scene, cfg.n_objects, cfg.r_max, keep=(W1[:2, 3], W2[:2, 3]))
    return W1, W2, dT, obj


def scene_of(objects):
    """The synth.scenes.Scene with the same ground, boxes and cylinders."""
    box = objects[objects[:, 0] == 0]
    cyl = objects[objects[:, 0] == 1]
    boxes = np.stack([box[:, 1], box[:, 2], np.arctan2(box[:, 4], box[:, 3]), box[:, 5], box[:, 6], box[:, 7]], -1)
    cyls = np.stack([cyl[:, 1], cyl[:, 2], cyl[:, 3], cyl[:, 4]], -1)
    return Scene(ground=True, boxes=boxes.reshape(-1, 6), cylinders=cyls.reshape(-1, 4))


def sensor_rows(sensor):
    """float32 [H][4]: cos phi, sin phi, theta, 0 (the ray caster's row table)."""
    rows = np.zeros((sensor.H, 4), np.float32)
    rows[:, 0] = np.cos(sensor.phi_lut)
    rows[:, 1] = np.sin(sensor.phi_lut)
    rows[:, 2] = sensor.theta_lut
    return rows


def pair_seed(cfg, index):
    """64-bit key of pair `index`'s device noise."""
    return int(np.random.SeedSequence([cfg.config_id, cfg.seed_base + index, 7]).generate_state(1, np.uint64)[0])


def _draw_many(args):
    name, indices = args
    from .configs import CONFIGS
    cfg = CONFIGS[name]
    n = len(indices)
    objs = np.zeros((n, cfg.n_objects, 8), np.float32)
    poses = np.zeros((n, 2, 12))
    seeds = np.zeros(n, np.uint64)
    T = np.zeros((n, 4, 4))
    for j, i in enumerate(indices):
        W1, W2, dT, ob = draw_pair(cfg, i)
        objs[j] = ob
        for k, Wk in enumerate((W1, W2)):
            poses[j, k, :9] = Wk[:3, :3].ravel()
            poses[j, k, 9:] = Wk[:3, 3]
        seeds[j] = pair_seed(cfg, i)
        T[j] = dT
    return objs, poses, seeds, T


def draw_pairs(cfg, indices, processes=1):
    """Host side of make_pairs_gpu: object records, world poses, noise keys
    and T_gt of pairs `indices` (a 'spawn' pool when processes > 1)."""
    indices = list(indices)
    if processes > 1 and len(indices) >= 256:
        import multiprocessing as mp
        step = (len(indices) + 4 * processes - 1) // (4 * processes)
        parts = [indices[i:i + step] for i in range(0, len(indices), step)]
        with mp.get_context("spawn").Pool(processes) as pool:
            out = pool.map(_draw_many, [(cfg.name, p) for p in parts])
        return tuple(np.concatenate([o[k] for o in out]) for k in range(4))
    return _draw_many((cfg.name, indices))


def make_pairs_gpu(cfg, indices, noise=True, device="cuda", processes=1, drawn=None):
    """Cast pairs `indices` of `cfg` on the GPU (on torch's current stream).
    Returns (src, dst) float32 torch tensors [n, H, W] on the device and T_gt
    float64 numpy [n, 4, 4].  `drawn`: a draw_pairs() result to reuse."""
    import torch
    lib = _load()
    indices = list(indices)
    n = len(indices)
    sensor = cfg.sensor()
    H, W = cfg.H, cfg.W
    no = cfg.n_objects
    if no > MAX_OBJ:
        raise ValueError("too many objects")
    objs, poses, seeds, T = drawn if drawn is not None else draw_pairs(cfg, indices, processes)
    out = torch.empty((2, n, H, W), dtype=torch.float32, device=device)
    rows = torch.from_numpy(sensor_rows(sensor)).to(device)
    d_objs = torch.from_numpy(objs).to(device)
    d_nobj = torch.full((n,), no, dtype=torch.int32, device=device)
    d_poses = torch.from_numpy(poses).to(device)
    d_seed = torch.from_numpy(seeds.view(np.int64)).to(device)
    st = torch.cuda.current_stream().cuda_stream
    chunk = 32767
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        tmp = out if (c0 == 0 and c1 == n) else torch.empty((2, c1 - c0, H, W), dtype=torch.float32, device=device)
        rc = lib.synth_raycast(c1 - c0, H, W, rows.data_ptr(), float(sensor.r0), d_objs[c0:c1].data_ptr(),
                               d_nobj[c0:c1].data_ptr(), no, d_poses[c0:c1].data_ptr(), float(cfg.r_min),
                               float(cfg.r_max), float(cfg.sigma if noise else 0.0),
                               float(cfg.dropout if noise else 0.0), d_seed[c0:c1].data_ptr(), tmp.data_ptr(), st)
        if rc != 0:
            raise RuntimeError(f"synth_raycast failed ({rc})")
        if tmp is not out:
            out[:, c0:c1] = tmp
    return out[1], out[0], T


def make_sequence_gpu(cfg, n_scans, seed, step=1.0, device="cuda"):
    """n_scans scans of ONE outdoor scene of `cfg` (objects drawn as in
    draw_pair, clear of every sensor position), the sensor 1.7 m above the
    ground moving `step` m along x per scan with a slow yaw drift (0.02 rad
    per scan).  Returns (ranges [n, H, W] float32 on the device, world poses
    [n, 4, 4] float64: sensor -> world)."""
    import torch
    lib = _load()
    sensor = cfg.sensor()
    rng = np.random.default_rng(np.random.SeedSequence([cfg.config_id, seed, 11]))
    poses = np.zeros((n_scans, 4, 4))
    for k in range(n_scans):
        yaw = 0.02 * k
        poses[k] = np.eye(4)
        poses[k, :3, :3] = [[np.cos(yaw), -np.sin(yaw), 0], [np.sin(yaw), np.cos(yaw), 0], [0, 0, 1]]
        poses[k, :3, 3] = [step * (k - 0.5 * (n_scans - 1)), 0.0, 1.7]
    obj = outdoor_objects(rng, cfg.n_objects, cfg.r_max, keep=poses[:, :2, 3]).astype(np.float32)
    n_pairs = (n_scans + 1) // 2
    objs = np.broadcast_to(obj, (n_pairs,) + obj.shape).copy()
    P = np.zeros((n_pairs, 2, 12))
    for k in range(2 * n_pairs):
        W = poses[min(k, n_scans - 1)]
        P[k // 2, k % 2, :9] = W[:3, :3].ravel()
        P[k // 2, k % 2, 9:] = W[:3, 3]
    seeds = np.array([pair_seed(cfg, 10 ** 6 + seed * 4096 + p) for p in range(n_pairs)], np.uint64)
    out = torch.empty((2, n_pairs, cfg.H, cfg.W), dtype=torch.float32, device=device)
    rows = torch.from_numpy(sensor_rows(sensor)).to(device)
    d_objs = torch.from_numpy(objs).to(device)
    d_nobj = torch.full((n_pairs,), obj.shape[0], dtype=torch.int32, device=device)
    d_poses = torch.from_numpy(P).to(device)
    d_seed = torch.from_numpy(seeds.view(np.int64)).to(device)
    rc = lib.synth_raycast(n_pairs, cfg.H, cfg.W, rows.data_ptr(), float(sensor.r0), d_objs.data_ptr(),
                           d_nobj.data_ptr(), obj.shape[0], d_poses.data_ptr(), float(cfg.r_min), float(cfg.r_max),
                           float(cfg.sigma), float(cfg.dropout), d_seed.data_ptr(), out.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    if rc != 0:
        raise RuntimeError(f"synth_raycast failed ({rc})")
    # scan 2p + k is out[k, p]
    scans = out.permute(1, 0, 2, 3).reshape(2 * n_pairs, cfg.H, cfg.W)[:n_scans].contiguous()
    return scans, poses
