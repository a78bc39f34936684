"""Procedural scenes and an analytic ray caster for a simulated spinning LiDAR.

The simulated sensor fires, for every pixel (u, v) of an H x W image, one ray
from a receiver on a cylinder of radius r0 around the sensor centre.  The
receiver sits at azimuth 2*pi*u/W; the ray leaves at azimuth
2*pi*u/W + theta_lut[v] and elevation phi_lut[v].  This is the physical
sensor the paper models (its Section 3), written here only to *simulate*
measurements; the range stored per pixel is the distance from the receiver to
the first surface hit.
"""
from dataclasses import dataclass, field
import numpy as np


@dataclass
class Sensor:
    H: int
    W: int
    phi_lut: np.ndarray      # float64 [H], radians
    theta_lut: np.ndarray    # float64 [H], radians
    r0: float = 0.0

    def rays(self):
        """Receiver origins and unit directions in the sensor frame, both (H*W, 3)."""
        H, W = self.H, self.W
        u = np.arange(W, dtype=np.float64)[None, :]
        col_az = 2.0 * np.pi * u / W                                  # [1, W]
        az = col_az + self.theta_lut[:, None]                          # [H, W]
        el = np.broadcast_to(self.phi_lut[:, None], (H, W))
        d = np.stack([np.cos(az) * np.cos(el), np.sin(az) * np.cos(el), np.sin(el)], -1)
        o = np.zeros((H, W, 3))
        o[..., 0] = self.r0 * np.cos(col_az)
        o[..., 1] = self.r0 * np.sin(col_az)
        return o.reshape(-1, 3), d.reshape(-1, 3)


@dataclass
class Scene:
    """Ground plane z = 0 (optional), vertical boxes and cylinders standing on
    z = 0, and optionally one closed room seen from inside."""
    ground: bool = True
    # boxes: (cx, cy, yaw, half_x, half_y, height)
    boxes: np.ndarray = field(default_factory=lambda: np.zeros((0, 6)))
    # cylinders: (cx, cy, radius, height)
    cylinders: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))
    # room: (cx, cy, yaw, half_x, half_y, height) or None
    room: np.ndarray = None


def _rot_axis_angle(axis, angle):
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * (K @ K)


def _unit_sphere(rng):
    while True:
        a = rng.normal(size=3)
        n = np.linalg.norm(a)
        if n > 1e-6:
            return a / n


def random_delta_pose(rng, rot_max_deg, trans_max):
    """Relative pose: axis uniform on the sphere, angle U(0, rot_max), translation
    direction uniform on the sphere, magnitude U(0, trans_max).  4x4 float64."""
    T = np.eye(4)
    T[:3, :3] = _rot_axis_angle(_unit_sphere(rng), np.deg2rad(rng.uniform(0, rot_max_deg)))
    T[:3, 3] = _unit_sphere(rng) * rng.uniform(0, trans_max)
    return T


def outdoor_scene(rng, n_objects, r_max, keep_clear=(), clear_margin=1.5):
    """Ground plane plus ``n_objects`` boxes/cylinders (50/50) whose centres lie
    3 .. 0.8*r_max m from the origin.  Objects whose footprint would come
    within ``clear_margin`` of any point in ``keep_clear`` (sensor positions)
    are redrawn, so every sensor sees all objects from outside."""
    boxes, cyls = [], []
    keep = [np.asarray(k, dtype=np.float64)[:2] for k in keep_clear] or [np.zeros(2)]
    while len(boxes) + len(cyls) < n_objects:
        rad = rng.uniform(3.0, 0.8 * r_max)
        ang = rng.uniform(0, 2 * np.pi)
        c = np.array([rad * np.cos(ang), rad * np.sin(ang)])
        if rng.random() < 0.5:
            hx, hy = rng.uniform(0.5, 6.0, size=2) / 2
            bound = np.hypot(hx, hy)
            obj = ("box", (c[0], c[1], rng.uniform(0, 2 * np.pi), hx, hy, rng.uniform(1.0, 6.0)))
        else:
            rr = rng.uniform(0.2, 1.5)
            bound = rr
            obj = ("cyl", (c[0], c[1], rr, rng.uniform(1.0, 6.0)))
        if any(np.linalg.norm(c - k) < bound + clear_margin for k in keep):
            continue
        (boxes if obj[0] == "box" else cyls).append(obj[1])
    return Scene(ground=True, boxes=np.array(boxes).reshape(-1, 6),
                 cylinders=np.array(cyls).reshape(-1, 4))


def indoor_scene(rng, n_furniture=12, keep_clear=(), clear_margin=0.8):
    """A closed room (sides 4-20 m, height 2.5-4 m) centred at the origin with
    furniture boxes inside; sensors in ``keep_clear`` stay clear of furniture."""
    hx, hy = rng.uniform(4.0, 20.0, size=2) / 2
    height = rng.uniform(2.5, 4.0)
    room = np.array([0.0, 0.0, rng.uniform(0, 2 * np.pi), hx, hy, height])
    cr, sr = np.cos(room[2]), np.sin(room[2])
    keep = [np.asarray(k, dtype=np.float64)[:2] for k in keep_clear] or [np.zeros(2)]
    boxes = []
    tries = 0
    while len(boxes) < n_furniture and tries < 10000:
        tries += 1
        bx, by = rng.uniform(0.3, 2.0, size=2) / 2
        lx = rng.uniform(-hx + bx, hx - bx) if hx > bx else 0.0
        ly = rng.uniform(-hy + by, hy - by) if hy > by else 0.0
        c = np.array([cr * lx - sr * ly, sr * lx + cr * ly])
        if any(np.linalg.norm(c - k) < np.hypot(bx, by) + clear_margin for k in keep):
            continue
        boxes.append((c[0], c[1], rng.uniform(0, 2 * np.pi), bx, by, rng.uniform(0.5, 2.0)))
    return Scene(ground=False, boxes=np.array(boxes).reshape(-1, 6),
                 cylinders=np.zeros((0, 4)), room=room)


# ----------------------------------------------------------------------------
# Ray/primitive intersections (world frame).  Each returns the hit distance t
# along the unit direction d (inf on a miss) for arrays of rays o, d (n, 3).

def _hit_ground(o, d):
    t = np.full(o.shape[0], np.inf)
    m = d[:, 2] < -1e-12
    t[m] = -o[m, 2] / d[m, 2]
    t[t <= 0] = np.inf
    return t


def _to_local(o, d, cx, cy, yaw):
    c, s = np.cos(yaw), np.sin(yaw)
    ox, oy = o[:, 0] - cx, o[:, 1] - cy
    lo = np.stack([c * ox + s * oy, -s * ox + c * oy, o[:, 2]], -1)
    ld = np.stack([c * d[:, 0] + s * d[:, 1], -s * d[:, 0] + c * d[:, 1], d[:, 2]], -1)
    return lo, ld


def _slab(lo, ld, lo_b, hi_b):
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / ld
        t1 = (lo_b - lo) * inv
        t2 = (hi_b - lo) * inv
    tmin = np.nanmax(np.minimum(t1, t2), axis=1)
    tmax = np.nanmin(np.maximum(t1, t2), axis=1)
    return tmin, tmax


def _hit_box(o, d, box):
    cx, cy, yaw, hx, hy, h = box
    lo, ld = _to_local(o, d, cx, cy, yaw)
    tmin, tmax = _slab(lo, ld, np.array([-hx, -hy, 0.0]), np.array([hx, hy, h]))
    t = np.where((tmax >= tmin) & (tmin > 0), tmin, np.inf)
    return t


def _hit_room_inside(o, d, room):
    cx, cy, yaw, hx, hy, h = room
    lo, ld = _to_local(o, d, cx, cy, yaw)
    _, tmax = _slab(lo, ld, np.array([-hx, -hy, 0.0]), np.array([hx, hy, h]))
    return np.where(tmax > 0, tmax, np.inf)


def _hit_cylinder(o, d, cyl):
    cx, cy, rr, h = cyl
    px, py = o[:, 0] - cx, o[:, 1] - cy
    a = d[:, 0] ** 2 + d[:, 1] ** 2
    b = 2 * (px * d[:, 0] + py * d[:, 1])
    c = px * px + py * py - rr * rr
    disc = b * b - 4 * a * c
    t = np.full(o.shape[0], np.inf)
    m = (disc >= 0) & (a > 1e-14)
    sq = np.sqrt(np.where(m, disc, 0.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        t_side = np.where(m, (-b - sq) / (2 * np.where(m, a, 1.0)), np.inf)
    with np.errstate(invalid="ignore"):
        z_side = o[:, 2] + t_side * d[:, 2]
    ok = m & (t_side > 0) & (z_side >= 0) & (z_side <= h)
    t[ok] = t_side[ok]
    # top cap
    with np.errstate(divide="ignore", invalid="ignore"):
        t_cap = np.where(np.abs(d[:, 2]) > 1e-12, (h - o[:, 2]) / d[:, 2], np.inf)
    with np.errstate(invalid="ignore"):
        xc, yc = px + t_cap * d[:, 0], py + t_cap * d[:, 1]
    okc = (t_cap > 0) & (xc * xc + yc * yc <= rr * rr)
    t = np.where(okc & (t_cap < t), t_cap, t)
    return t


def raycast(scene, sensor, pose, r_min, r_max, noise_sigma=0.0, dropout=0.0, rng=None):
    """Range image (float32 [H, W]) of ``scene`` seen by ``sensor`` placed at world
    pose ``pose`` (4x4).  Misses and ranges outside [r_min, r_max] are 0; then
    Gaussian range noise (sigma, metres) is added to valid pixels and a
    Bernoulli(dropout) fraction of pixels is set to 0 (invalid)."""
    o_s, d_s = sensor.rays()
    R, tw = pose[:3, :3], pose[:3, 3]
    o = o_s @ R.T + tw
    d = d_s @ R.T
    n = o.shape[0]
    t = np.full(n, np.inf)
    if scene.ground:
        t = np.minimum(t, _hit_ground(o, d))
    if scene.room is not None:
        t = np.minimum(t, _hit_room_inside(o, d, scene.room))
    # Cull objects by horizontal azimuth: a vertical prism/cylinder can only be
    # hit by rays whose horizontal heading passes within its bounding circle.
    az = np.arctan2(d[:, 1], d[:, 0])
    horiz = np.hypot(d[:, 0], d[:, 1]) > 1e-9
    order = np.argsort(az)
    az_sorted = az[order]
    slack = sensor.r0 + 1e-3

    def candidates(cx, cy, bound):
        D = np.hypot(cx - tw[0], cy - tw[1])
        if D <= bound + slack + 1e-6:
            return np.arange(n)
        beta = np.arcsin(min(1.0, (bound + slack) / (D - slack))) + 1e-6
        a0 = np.arctan2(cy - tw[1], cx - tw[0])
        lo, hi = a0 - beta, a0 + beta
        parts = []
        for l, h in ((lo, hi), (lo + 2 * np.pi, hi + 2 * np.pi), (lo - 2 * np.pi, hi - 2 * np.pi)):
            i0 = np.searchsorted(az_sorted, max(l, -np.pi), "left")
            i1 = np.searchsorted(az_sorted, min(h, np.pi), "right")
            if i1 > i0:
                parts.append(order[i0:i1])
        idx = np.concatenate(parts) if parts else np.zeros(0, dtype=np.int64)
        return idx[horiz[idx]]

    for box in scene.boxes:
        idx = candidates(box[0], box[1], np.hypot(box[3], box[4]))
        if idx.size:
            t[idx] = np.minimum(t[idx], _hit_box(o[idx], d[idx], box))
    for cyl in scene.cylinders:
        idx = candidates(cyl[0], cyl[1], cyl[2])
        if idx.size:
            t[idx] = np.minimum(t[idx], _hit_cylinder(o[idx], d[idx], cyl))
    rng_img = np.where((t >= r_min) & (t <= r_max), t, 0.0)
    if rng is not None and noise_sigma > 0:
        valid = rng_img > 0
        rng_img = np.where(valid, rng_img + rng.normal(0.0, noise_sigma, size=n), 0.0)
        rng_img = np.where(rng_img > 0, rng_img, 0.0)
    if rng is not None and dropout > 0:
        rng_img = np.where(rng.random(n) < dropout, 0.0, rng_img)
    return rng_img.reshape(sensor.H, sensor.W).astype(np.float32)
