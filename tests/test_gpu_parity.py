"""GPU parity: every step of the CUDA path, through the C ABI, against the FP64
oracle on the same seeded inputs.

Bars (derived in the design notes):
  * integer work (pyramid copies, association indices, validity masks) is
    bit-exact, except association/validity decisions the oracle flags as
    near-ties (a continuous quantity within 1e-3 px, 1e-3 row spacings or a
    relative 1e-3 of a normal-degeneracy threshold of a decision boundary);
  * points: |xyz_gpu - xyz_oracle| <= 16 u (r + r0) + 1e-7 (u = 2^-24);
  * normals: per pixel 32 u |P| (1/|a| + 1/|b|) + 1e-6 (a, b the central
    differences), planes' offsets d to the same relative bound times |P|;
  * reduced sums: |S_gpu - S_oracle| <= rel * sum|terms| (rel 1e-3) plus two
    times the largest term per association that differs on a near-tie;
  * poses: 1e-4 rad and 1e-4 m against the oracle's registration.
"""
import numpy as np
import pytest

from oracle import rimg_oracle as O
from synth import CONFIGS, Sensor, make_pair, make_pairs, uniform_phi
from tests.gpu_common import (U32, f32, oracle_params, gpu_sensor, planes_for, src_pyramid, gpu_register,
                              oracle_register, shadowed_check, groups_runner)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_02779_b300.rimg as R   # fails loudly when librimg.so is missing
    return R


CFG_LEVELS = [("pair32x512", 3), ("pair64x1024", 4), ("lut64x512", 3), ("stress16x64", 2)]


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,levels", CFG_LEVELS)
def test_unproject_parity(R, name, levels):
    cfg = CONFIGS[name]
    p = make_pair(cfg, 0)
    s = p["sensor"]
    sens = gpu_sensor(R, s, levels)
    img = p["dst_range"].copy()
    img[0, :5] = np.nan
    img[1, :5] = np.inf
    img[2, :5] = -1.0
    for l in range(levels):
        st = 1 << l
        rl = np.ascontiguousarray(img[::st, ::st])
        H, W = rl.shape
        rt = torch.from_numpy(rl)[None].cuda()
        xyz = torch.zeros((1, 3, H, W), dtype=torch.float32, device="cuda")
        mask = torch.zeros((1, H, W), dtype=torch.uint8, device="cuda")
        R.rimg_unproject(sens, l, rt, xyz, mask)
        ph, th = O.level_tables(s.phi_lut, s.theta_lut, l)
        P, ok = O.unproject(rl, ph, th, s.r0)
        m = mask[0].cpu().numpy().astype(bool)
        assert np.array_equal(m, ok)
        g = xyz[0].cpu().numpy().transpose(1, 2, 0)
        r = np.where(ok, rl, 0.0).astype(np.float64)
        tol = 16 * U32 * (r + s.r0) + 1e-7
        assert np.all(np.abs(g - P).max(-1) <= tol)


@pytest.mark.parametrize("channels", [1, 4])
def test_pyramid_bit_exact(R, channels):
    rng = np.random.default_rng(21)
    for (n, H, W, L) in [(3, 24, 40, 3), (2, 64, 1024, 4), (1, 8, 8, 4)]:
        shape = (n, H, W) if channels == 1 else (n, H, W, 4)
        a = rng.standard_normal(shape).astype(np.float32)
        t = torch.from_numpy(a).cuda()
        outs = [None] + [torch.full((n, H >> l, W >> l) + (() if channels == 1 else (4,)), np.nan,
                                    dtype=torch.float32, device="cuda") for l in range(1, L)]
        R.rimg_pyramid(n, H, W, L, channels, t, outs)
        for l in range(1, L):
            st = 1 << l
            assert np.array_equal(outs[l].cpu().numpy(), a[:, ::st, ::st])


def _normal_tolerance(P, ok):
    a = np.roll(P, -1, axis=1) - np.roll(P, 1, axis=1)
    b = np.zeros_like(P)
    b[1:-1] = P[2:] - P[:-2]
    an = np.linalg.norm(a, axis=-1)
    bn = np.linalg.norm(b, axis=-1)
    pn = np.linalg.norm(P, axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = 32 * U32 * pn * (1 / an + 1 / bn)
    return np.where(ok, rel + 1e-6, np.inf), pn


def _check_normals(R, s, sens, imgs, levels):
    params = R.rimg_default_params()
    planes, mask = planes_for(R, torch, sens, torch.from_numpy(imgs).cuda(), params)
    for i in range(imgs.shape[0]):
        n_o, ok_o, margin = O.normals(imgs[i], s.phi_lut, s.theta_lut, s.r0, f32(0.1), return_margin=True)
        P, _ = O.unproject(imgs[i], s.phi_lut, s.theta_lut, s.r0)
        m = mask[i].cpu().numpy().astype(bool)
        near = margin < 1e-3
        assert np.array_equal(m[~near], ok_o[~near])
        pl = planes[0][i].cpu().numpy()
        assert np.array_equal(np.any(pl[..., :3] != 0, axis=-1), m)
        both = m & ok_o
        tol, pn = _normal_tolerance(P, ok_o)
        ng = pl[..., :3]
        # orientation is a sign decision on n . P; where that is a near-tie
        # either sign is accepted (point-to-plane terms do not depend on it)
        grazing = np.abs(np.sum(n_o * P, -1)) < 1e-3 * pn
        err = np.abs(ng - n_o).max(-1)
        err = np.where(grazing, np.minimum(err, np.abs(ng + n_o).max(-1)), err)
        assert np.all(err[both] <= tol[both])
        d_o = np.sum(n_o * P, -1)
        derr = np.abs(pl[..., 3] - d_o)
        derr = np.where(grazing, np.minimum(derr, np.abs(pl[..., 3] + d_o)), derr)
        with np.errstate(invalid="ignore"):
            dtol = np.where(both, tol * pn + 16 * U32 * pn, 0.0)
        assert np.all(derr[both] <= dtol[both])
        for l in range(1, levels):
            st = 1 << l
            assert np.array_equal(planes[l][i].cpu().numpy(), pl[::st, ::st])
    return mask


@pytest.mark.parametrize("name,levels", CFG_LEVELS)
def test_normals_parity(R, name, levels):
    cfg = CONFIGS[name]
    s = cfg.sensor()
    sens = gpu_sensor(R, s, levels)
    imgs = np.stack([make_pair(cfg, i)["dst_range"] for i in range(2)])
    _check_normals(R, s, sens, imgs, levels)


@pytest.mark.parametrize("H,W,levels", [(8, 136, 1), (12, 64, 2), (24, 1152, 3), (16, 4, 1), (20, 136, 2)])
def test_normals_parity_strip_edges(R, H, W, levels):
    """Widths that end inside a 128-column strip (136, 64, 4: the wrap lands in
    a lane of the same warp), a width of nine strips, and heights that end
    inside an 8-row strip (12, 20) or on a strip boundary (8, 16, 24)."""
    from synth import Sensor, outdoor_scene, raycast, uniform_phi
    rng = np.random.default_rng(H * 1000 + W)
    s = Sensor(H, W, uniform_phi(H, 8.0, -20.0), rng.uniform(-0.01, 0.01, H), 0.04)
    scene = outdoor_scene(rng, 60, 40.0)
    Wd = np.eye(4)
    Wd[2, 3] = 1.7
    imgs = np.stack([raycast(scene, s, Wd, 1.0, 60.0, 0.01, 0.05, rng) for _ in range(2)]).astype(np.float32)
    sens = gpu_sensor(R, s, levels)
    mask = _check_normals(R, s, sens, imgs, levels)
    if W >= 64:
        assert mask.sum().item() > 0.1 * imgs.size


# ---------------------------------------------------------------------------
def _icp_case(R, name, levels, level, pose_kind, params_kw=None, idx=0):
    cfg = CONFIGS[name] if isinstance(name, str) else name
    pair = make_pair(cfg, idx)
    s = pair["sensor"]
    sens = gpu_sensor(R, s, levels)
    kw = dict(huber_delta=cfg.huber_delta)
    kw.update(params_kw or {})
    params = R.rimg_default_params(**kw)
    src = torch.from_numpy(pair["src_range"])[None].cuda()
    dst = torch.from_numpy(pair["dst_range"])[None].cuda()
    planes, _ = planes_for(R, torch, sens, dst, params)
    spyr = src_pyramid(R, torch, sens, src)
    dpyr = src_pyramid(R, torch, sens, dst)
    if pose_kind == "identity":
        T = np.eye(4)
    else:
        T = O.se3_exp(np.array([2e-3, -1e-3, 3e-3, 0.02, -0.01, 0.015])) @ pair["T_gt"]
    pose = torch.from_numpy(T.reshape(1, 16).copy()).cuda()
    H, W = s.H >> level, s.W >> level
    assoc = torch.full((1, H, W), -7, dtype=torch.int32, device="cuda")
    out29 = torch.zeros((1, 29), dtype=torch.float64, device="cuda")
    ws = torch.empty(R.rimg_icp_workspace_bytes(sens, 1), dtype=torch.uint8, device="cuda")
    R.rimg_icp_step(sens, sens, level, 1, spyr[level], planes[level],
                    dpyr[level] if params.max_corr_dist > 0 else None, pose, params, 0, out29, assoc, None, ws)
    torch.cuda.synchronize()
    tgt = O.Target(pair["dst_range"], s.phi_lut, s.theta_lut, s.r0, levels, f32(0.1))
    P, sv = O.source_points(pair["src_range"], s.phi_lut, s.theta_lut, s.r0, level)
    rng_l, n_l, nv_l, ph, th = tgt.level(level)
    terms = O.icp_terms(P, sv, T, rng_l, n_l, nv_l, ph, th, s.r0, f32(params.huber_delta),
                        f32(params.max_corr_dist), dst_n_margin=tgt.nmargin[level])
    return assoc[0].cpu().numpy().reshape(-1), out29[0].cpu().numpy(), terms, T, pose.cpu().numpy()


def _sum_bounds(terms, n_mismatch, rel=1e-3):
    """Per-quantity tolerance: rel * sum|term_i| plus, per association that
    differs on a near-tie, twice the largest single term."""
    J, e, w = terms["J"], terms["e"], terms["w"]
    wJ = J * w[:, None]
    cols = [wJ[:, i] * J[:, j] for i in range(6) for j in range(i, 6)]
    cols += [wJ[:, i] * e for i in range(6)] + [w * e * e]
    A = np.abs(np.stack(cols, 1)) if len(e) else np.zeros((0, 28))
    s = A.sum(0) if len(e) else np.zeros(28)
    m = A.max(0) if len(e) else np.zeros(28)
    return np.concatenate([rel * s + 2 * n_mismatch * m, [n_mismatch]])


def _check_icp_levels(R, cfg, levels, pose_kind):
    for level in range(levels):
        assoc, out29, terms, T, pose_after = _icp_case(R, cfg, levels, level, pose_kind)
        assert np.array_equal(pose_after.reshape(4, 4), T)          # update = 0 leaves the pose alone
        near = terms["near_tie"]
        a_o = terms["assoc"]
        diff = (assoc != a_o)
        assert not np.any(diff & ~near), f"level {level}: {np.sum(diff & ~near)} non-near-tie mismatches"
        n_mis = int(np.sum(diff))
        assert n_mis <= max(3, 1e-3 * np.sum(a_o >= 0))
        ref = O.pack29(terms)
        bound = _sum_bounds(terms, n_mis)
        err = np.abs(out29 - ref)
        assert np.all(err <= bound + 1e-9), (level, err / np.maximum(bound, 1e-30))


@pytest.mark.parametrize("name,levels", CFG_LEVELS)
@pytest.mark.parametrize("pose_kind", ["identity", "near"])
def test_icp_step_parity(R, name, levels, pose_kind):
    _check_icp_levels(R, name, levels, pose_kind)


def _fast_projection(sens, level):
    """Whether the association kernels project into this level without the
    boundary walk and the azimuth offsets, wrapping columns by a mask (exact
    inverse table, theta_lut = 0, power-of-two width)."""
    L = sens.struct.level[level]
    return bool(L.bins_exact) and not L.has_theta and L.W > 0 and (L.W & (L.W - 1)) == 0


def test_configs_cover_both_projection_forms(R):
    """The parity configurations reach the branch-free projection (exact
    tables, no azimuth offsets, power-of-two widths) and the general one
    (azimuth offsets, or a table uneven enough to need the boundary walk;
    the ragged 24 x 48 case has a width that is not a power of two)."""
    forms = set()
    for name, levels in CFG_LEVELS:
        sens = gpu_sensor(R, CONFIGS[name].sensor(), levels)
        forms |= {_fast_projection(sens, l) for l in range(levels)}
    assert forms == {True, False}
    s = CONFIGS["pair64x1024"].sensor()
    assert all(_fast_projection(gpu_sensor(R, s, 4), l) for l in range(4))   # the headline sensor


@pytest.mark.parametrize("name,r0", [("pair64x1024", 0.0), ("pair32x512", 0.015)])
def test_fast_form_equals_general_form(R, name, r0):
    """The branch-free projection (exact table, one comparison, column wrapped
    by a mask) takes the same decisions as the general form with the boundary
    walk and the conditional wraps: a step's 29 sums are bit-identical between
    the two (the association output selects the general form; both walk chunks
    in the same order), at every level, at poses that move points across the
    field-of-view edges."""
    import dataclasses
    cfg = dataclasses.replace(CONFIGS[name], config_id=91 if r0 else CONFIGS[name].config_id, r0=r0)
    levels = cfg.levels
    pair = make_pair(cfg, 1)
    s = pair["sensor"]
    sens = gpu_sensor(R, s, levels)
    assert all(_fast_projection(sens, l) for l in range(levels))
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    src = torch.from_numpy(pair["src_range"])[None].cuda()
    dst = torch.from_numpy(pair["dst_range"])[None].cuda()
    planes, _ = planes_for(R, torch, sens, dst, params)
    spyr = src_pyramid(R, torch, sens, src)
    ws = torch.empty(R.rimg_icp_workspace_bytes(sens, 1), dtype=torch.uint8, device="cuda")
    for pose in (np.eye(4), O.se3_exp(np.array([0.05, -0.08, 0.02, 0.3, -0.2, 0.9])) @ pair["T_gt"],
                 O.se3_exp(np.array([0.0, 0.2, 0.0, 0.0, 0.0, -1.5]))):
        for level in range(levels):
            out = []
            for with_assoc in (True, False):
                T = torch.from_numpy(pose.reshape(1, 16).copy()).cuda()
                o29 = torch.zeros((1, 29), dtype=torch.float64, device="cuda")
                assoc = (torch.empty((1, s.H >> level, s.W >> level), dtype=torch.int32, device="cuda")
                         if with_assoc else None)
                R.rimg_icp_step(sens, sens, level, 1, spyr[level], planes[level], None, T, params, 0, o29, assoc,
                                None, ws)
                torch.cuda.synchronize()
                out.append(o29.cpu().numpy())
            assert np.array_equal(out[0], out[1]), (level, out[0] - out[1])


@pytest.mark.parametrize("pose_kind", ["identity", "near"])
def test_icp_step_parity_fast_projection_with_receiver_offset(R, pose_kind):
    """Exact tables and no azimuth offsets, with a receiver offset r0 = 1.5 cm:
    the branch-free projection inside the receiver-offset fixed point (every
    level of one step, then registrations) against the oracle."""
    import dataclasses
    cfg = dataclasses.replace(CONFIGS["pair32x512"], name="pair32x512_r0", config_id=91, r0=0.015)
    sens = gpu_sensor(R, cfg.sensor(), 3)
    assert all(_fast_projection(sens, l) for l in range(3))
    _check_icp_levels(R, cfg, 3, pose_kind)
    if pose_kind == "identity":
        s = cfg.sensor()
        params = R.rimg_default_params(huber_delta=cfg.huber_delta)
        pairs = [make_pair(cfg, i) for i in range(3)]   # a derived config: not in the pool's table
        src = np.stack([q["src_range"] for q in pairs])
        dst = np.stack([q["dst_range"] for q in pairs])
        Tg, _ = gpu_register(R, torch, sens, src, dst, np.tile(np.eye(4), (3, 1, 1)), 3, cfg.iters, params)
        for i in range(3):
            To, _ = oracle_register(src[i], dst[i], s, np.eye(4), 3, cfg.iters, oracle_params(cfg))
            eR, et = O.pose_error(Tg[i], To)
            assert eR <= 1e-4 and et <= 1e-4, (i, eR, et)


def test_icp_step_gate_parity(R):
    for level in range(3):
        assoc, out29, terms, T, _ = _icp_case(R, "pair32x512", 3, level, "identity",
                                              params_kw=dict(max_corr_dist=0.5))
        diff = assoc != terms["assoc"]
        assert not np.any(diff & ~terms["near_tie"])
        assert abs(out29[28] - terms["count"]) <= np.sum(diff)


def test_icp_step_update_matches_oracle_step(R):
    """update = 1 applies the FP64 Cholesky + SE(3) step; from the same pose
    the result matches the oracle's single step."""
    cfg = CONFIGS["pair32x512"]
    pair = make_pair(cfg, 1)
    s = pair["sensor"]
    sens = gpu_sensor(R, s, 3)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    src = torch.from_numpy(pair["src_range"])[None].cuda()
    dst = torch.from_numpy(pair["dst_range"])[None].cuda()
    planes, _ = planes_for(R, torch, sens, dst, params)
    pose = torch.eye(4, dtype=torch.float64, device="cuda").reshape(1, 16).contiguous()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(R.rimg_icp_workspace_bytes(sens, 1), dtype=torch.uint8, device="cuda")
    R.rimg_icp_step(sens, sens, 0, 1, src, planes[0], None, pose, params, 1, None, None, status, ws)
    tgt = O.Target(pair["dst_range"], s.phi_lut, s.theta_lut, s.r0, 3, f32(0.1))
    P, sv = O.source_points(pair["src_range"], s.phi_lut, s.theta_lut, s.r0, 0)
    T1, ok, _ = O.icp_step(P, sv, tgt, 0, np.eye(4), oracle_params(cfg))
    Tg = pose.cpu().numpy().reshape(4, 4)
    eR, et = O.pose_error(Tg, T1)
    assert ok and status.item() == 0
    assert eR < 1e-5 and et < 1e-5


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,levels,n", [("pair32x512", 3, 8), ("pair64x1024", 4, 2), ("lut64x512", 3, 4)])
def test_register_pose_parity(R, name, levels, n):
    cfg = CONFIGS[name]
    s = cfg.sensor()
    sens = gpu_sensor(R, s, levels)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    src, dst, Tgt = make_pairs(cfg, range(n))
    T0 = np.tile(np.eye(4), (n, 1, 1))
    Tg, status = gpu_register(R, torch, sens, src, dst, T0, levels, cfg.iters, params)
    for i in range(n):
        To, deg = oracle_register(src[i], dst[i], s, np.eye(4), levels, cfg.iters, oracle_params(cfg))
        eR, et = O.pose_error(Tg[i], To)
        assert eR <= 1e-4 and et <= 1e-4, (i, eR, et)
        assert bool(status[i] & 1) == deg


def test_register_with_gate_parity(R):
    cfg = CONFIGS["pair32x512"]
    s = cfg.sensor()
    sens = gpu_sensor(R, s, 3)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta, max_corr_dist=1.0)
    src, dst, _ = make_pairs(cfg, range(3))
    Tg, _ = gpu_register(R, torch, sens, src, dst, np.tile(np.eye(4), (3, 1, 1)), 3, cfg.iters, params)
    for i in range(3):
        To, _ = oracle_register(src[i], dst[i], s, np.eye(4), 3, cfg.iters, oracle_params(cfg, gate=1.0))
        eR, et = O.pose_error(Tg[i], To)
        assert eR <= 1e-4 and et <= 1e-4


def test_register_kahan_and_plain_both_match(R):
    cfg = CONFIGS["indoor128x2048"]
    s = cfg.sensor()
    sens = gpu_sensor(R, s, 4)
    src, dst, _ = make_pairs(cfg, range(1))
    To, _ = oracle_register(src[0], dst[0], s, np.eye(4), 4, cfg.iters, oracle_params(cfg))
    for kahan in (1, 0):
        params = R.rimg_default_params(huber_delta=cfg.huber_delta, kahan=kahan)
        Tg, _ = gpu_register(R, torch, sens, src, dst, np.eye(4)[None], 4, cfg.iters, params)
        eR, et = O.pose_error(Tg[0], To)
        assert eR <= 1e-4 and et <= 1e-4, (kahan, eR, et)


def test_register_host_matches_device(R):
    cfg = CONFIGS["pair32x512"]
    s = cfg.sensor()
    sens = gpu_sensor(R, s, 3)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    n = 7
    src, dst, _ = make_pairs(cfg, range(n))
    T0 = np.tile(np.eye(4), (n, 1, 1))
    Tg, st_dev = gpu_register(R, torch, sens, src, dst, T0, 3, cfg.iters, params)
    for chunk in (0, 3):
        hs = torch.from_numpy(src).pin_memory()
        hd = torch.from_numpy(dst).pin_memory()
        hT0 = torch.from_numpy(T0.reshape(n, 16).copy()).pin_memory()
        hT1 = torch.zeros((n, 16), dtype=torch.float64).pin_memory()
        hst = torch.full((n,), -7, dtype=torch.int32).pin_memory()
        ws = torch.empty(R.rimg_register_host_workspace_bytes(sens, sens, n, 3, chunk), dtype=torch.uint8,
                         device="cuda")
        R.rimg_register_host(sens, sens, n, hs, hd, hT0, hT1, 3, cfg.iters, params, hst, chunk, ws)
        Th = hT1.numpy().reshape(n, 4, 4)
        if chunk == 0:
            # same batch, same block decomposition: bit-identical
            assert np.array_equal(Th, Tg)
        else:
            # a smaller batch may split pairs into a different number of blocks
            # (a different FP32 summation order)
            for i in range(n):
                eR, et = O.pose_error(Th[i], Tg[i])
                assert eR <= 1e-7 and et <= 1e-7
        assert np.array_equal(hst.numpy(), st_dev)


# ---------------------------------------------------------------------------
def test_empty_batches_are_noops(R):
    cfg = CONFIGS["stress16x64"]
    s = cfg.sensor()
    sens = gpu_sensor(R, s, 2)
    params = R.rimg_default_params()
    e = torch.zeros((0, s.H, s.W), dtype=torch.float32, device="cuda")
    R.rimg_normals(sens, e, params, [torch.zeros(0, device="cuda")] * 2)
    R.rimg_register(sens, sens, 0, e, e, torch.zeros(0, dtype=torch.float64, device="cuda"),
                    torch.zeros(0, dtype=torch.float64, device="cuda"), 2, (1, 1), params,
                    workspace=torch.empty(256, dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()


def test_invalid_and_nonfinite_inputs(R):
    """All-invalid sources give a degenerate system: the pose is unchanged and
    the flag set.  NaN / inf / negative ranges behave exactly like 0."""
    cfg = CONFIGS["pair32x512"]
    s = cfg.sensor()
    sens = gpu_sensor(R, s, 3)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    pair = make_pair(cfg, 2)
    zero = np.zeros_like(pair["src_range"])
    T0 = O.se3_exp(np.array([0.01, 0, 0, 0.1, 0, 0]))
    Tg, st = gpu_register(R, torch, sens, zero[None], pair["dst_range"][None], T0[None], 3, cfg.iters, params)
    assert np.array_equal(Tg[0], T0) and st[0] & 1
    src = pair["src_range"].copy()
    rng = np.random.default_rng(3)
    bad = rng.random(src.shape) < 0.05
    vals = np.array([np.nan, np.inf, -np.inf, -2.0], np.float32)
    src_bad = src.copy()
    src_bad[bad] = vals[rng.integers(0, 4, size=bad.sum())]
    src_zero = src.copy()
    src_zero[bad] = 0.0
    Ta, _ = gpu_register(R, torch, sens, src_bad[None], pair["dst_range"][None], np.eye(4)[None], 3, cfg.iters,
                         params)
    Tb, _ = gpu_register(R, torch, sens, src_zero[None], pair["dst_range"][None], np.eye(4)[None], 3, cfg.iters,
                         params)
    assert np.array_equal(Ta, Tb)
    assert np.all(np.isfinite(Ta))


def test_ragged_small_image_parity(R):
    """A 24 x 48 image (rows and chunks not multiples of the block shape),
    batch of 3 different pairs."""
    H, W = 24, 48
    sensor = Sensor(H, W, uniform_phi(H, 8.0, -22.0), np.zeros(H), 0.0)
    from synth.scenes import outdoor_scene, raycast, random_delta_pose
    rng = np.random.default_rng(5)
    srcs, dsts = [], []
    for i in range(3):
        W1 = np.eye(4); W1[2, 3] = 1.7
        dT = random_delta_pose(rng, 2.0, 0.2)
        scene = outdoor_scene(rng, 30, 40.0, keep_clear=(W1[:3, 3], (W1 @ dT)[:3, 3]))
        dsts.append(raycast(scene, sensor, W1, 0.5, 40.0, 0.01, 0.05, rng))
        srcs.append(raycast(scene, sensor, W1 @ dT, 0.5, 40.0, 0.01, 0.05, rng))
    src, dst = np.stack(srcs), np.stack(dsts)
    sens = gpu_sensor(R, sensor, 2)
    params = R.rimg_default_params(huber_delta=0.5)
    Tg, _ = gpu_register(R, torch, sens, src, dst, np.tile(np.eye(4), (3, 1, 1)), 2, (5, 5), params)
    for i in range(3):
        To, _ = oracle_register(src[i], dst[i], sensor, np.eye(4), 2, (5, 5),
                                dict(huber_delta=f32(0.5), normal_rel_jump=f32(0.1)))
        eR, et = O.pose_error(Tg[i], To)
        assert eR <= 1e-4 and et <= 1e-4


def test_workspace_too_small_is_rejected(R):
    cfg = CONFIGS["stress16x64"]
    s = cfg.sensor()
    sens = gpu_sensor(R, s, 2)
    params = R.rimg_default_params()
    x = torch.zeros((1, s.H, s.W), dtype=torch.float32, device="cuda")
    T = torch.eye(4, dtype=torch.float64, device="cuda").reshape(1, 16).contiguous()
    with pytest.raises(R.RimgError) as ei:
        R.rimg_register(sens, sens, 1, x, x, T, T, 2, (1, 1), params,
                        workspace=torch.empty(256, dtype=torch.uint8, device="cuda"))
    assert ei.value.code == -4


# ---------------------------------------------------------------------------
def test_full_size_batch_sampled_against_oracle(R):
    """The benchmark's launch configuration: 512 pairs of 64 x 1024 in one
    call.  Eight distinct seeded pairs are tiled into the batch (distinct
    buffers); every copy of a pair must give the bit-identical pose (position
    in the batch does not matter) and the distinct pairs match the oracle."""
    cfg = CONFIGS["pair64x1024"]
    s = cfg.sensor()
    sens = gpu_sensor(R, s, 4)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    k, n = 8, 512
    src, dst, _ = make_pairs(cfg, range(k), processes=4)
    reps = n // k
    Tg, status = gpu_register(R, torch, sens, np.tile(src, (reps, 1, 1)), np.tile(dst, (reps, 1, 1)),
                              np.tile(np.eye(4), (n, 1, 1)), 4, cfg.iters, params)
    Tg = Tg.reshape(reps, k, 4, 4)
    assert np.all(Tg == Tg[0:1])
    for i in range(0, k, 2):
        To, _ = oracle_register(src[i], dst[i], s, np.eye(4), 4, cfg.iters, oracle_params(cfg))
        eR, et = O.pose_error(Tg[0, i], To)
        assert eR <= 1e-4 and et <= 1e-4


def test_register_sub_batch_streams_agree(R):
    """Splitting a batch over internal streams changes only the FP32 summation
    order of each pair's reduction (the block decomposition depends on the
    sub-batch size): poses agree within the parity bar."""
    cfg = CONFIGS["pair32x512"]
    s = cfg.sensor()
    sens = gpu_sensor(R, s, 3)
    n = 128
    src, dst, _ = make_pairs(cfg, range(8))
    src, dst = np.tile(src, (16, 1, 1)), np.tile(dst, (16, 1, 1))
    T0 = np.tile(np.eye(4), (n, 1, 1))
    out = {}
    for streams in (1, 2, 3, 4):
        params = R.rimg_default_params(huber_delta=cfg.huber_delta, streams=streams)
        out[streams], _ = gpu_register(R, torch, sens, src, dst, T0, 3, cfg.iters, params)
    for streams in (2, 3, 4):
        for i in range(n):
            eR, et = O.pose_error(out[streams][i], out[1][i])
            assert eR <= 1e-4 and et <= 1e-4


def test_register_host_async_two_streams(R):
    """Two asynchronous host-buffer registrations queued back to back on two
    streams with separate workspaces give the same poses as the synchronous
    call (the second batch is the first one reversed)."""
    cfg = CONFIGS["pair32x512"]
    s = cfg.sensor()
    sens = gpu_sensor(R, s, 3)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    n = 40
    src, dst, _ = make_pairs(cfg, range(8))
    src, dst = np.tile(src, (5, 1, 1)), np.tile(dst, (5, 1, 1))
    batches = [(src, dst), (np.ascontiguousarray(src[::-1]), np.ascontiguousarray(dst[::-1]))]
    T0 = torch.from_numpy(np.tile(np.eye(4), (n, 1, 1)).reshape(n, 16).copy()).pin_memory()
    nbytes = R.rimg_register_host_workspace_bytes(sens, sens, n, 3, 16)
    ref, outs, keep = [], [], []
    for bs, bd in batches:
        hs, hd = torch.from_numpy(bs).pin_memory(), torch.from_numpy(bd).pin_memory()
        out = torch.zeros((n, 16), dtype=torch.float64).pin_memory()
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        R.rimg_register_host(sens, sens, n, hs, hd, T0, out, 3, cfg.iters, params, None, 16, ws)
        ref.append(out.numpy().copy())
        keep.append((hs, hd, ws))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    # each queued call needs its own workspace, alive until its stream is drained
    wss = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
    for j, (hs, hd, _) in enumerate(keep):
        out = torch.full((n, 16), np.nan, dtype=torch.float64).pin_memory()
        R.rimg_register_host_async(sens, sens, n, hs, hd, T0, out, 3, cfg.iters, params, None, 16, wss[j],
                                   streams[j])
        outs.append(out)
    for st in streams:
        st.synchronize()
    for j in range(2):
        assert np.array_equal(outs[j].numpy(), ref[j])
    assert np.allclose(ref[0], ref[1][::-1], atol=1e-9)


def _group_inputs(R, kinds, counts):
    groups, keep = [], []
    for kind, n in zip(kinds, counts):
        cfg = CONFIGS[kind]
        s = cfg.sensor()
        sens = gpu_sensor(R, s, cfg.levels)
        src, dst, _ = make_pairs(cfg, range(n))
        params = R.rimg_default_params(huber_delta=cfg.huber_delta)
        T0 = torch.eye(4, dtype=torch.float64, device="cuda").reshape(1, 16).repeat(n, 1).contiguous()
        g = dict(src=sens, dst=sens, n_pairs=n, levels=cfg.levels, iters=cfg.iters, params=params,
                 src_range=torch.from_numpy(src).cuda(), dst_range=torch.from_numpy(dst).cuda(), T_init=T0,
                 T_out=torch.empty_like(T0), status=torch.zeros(n, dtype=torch.int32, device="cuda"))
        groups.append(g)
        keep.append((cfg, s, src, dst))
    return groups, keep


def _agree_or_explained(R, g, cfg, s, src, dst, T_test, T_other):
    """Two GPU registrations of group g whose launches sum in different
    orders (block decompositions, queue blocks): each pair's poses agree
    within 1e-4 rad / 1e-4 m, or, where a near-tie re-association parted
    them, the run under test (T_test, rimg_register_groups with the current
    tuning state) passes the per-level oracle check on that pair.  Those
    pairs stay a minority.  Returns their indices."""
    far = [i for i in range(len(T_test)) if max(O.pose_error(T_test[i], T_other[i])) > 1e-4]
    if far:
        rep = shadowed_check(R, torch, g["src"], s, src[far], dst[far], cfg.levels, cfg.iters, g["params"],
                             oracle_params(cfg), runner=_subset_runner(R, g, far))
        print(cfg.name, "pairs beyond 1e-4 between the two GPU runs:", far, rep["max_err"], rep["explained"])
        assert rep["levels_checked"] == len(far) * cfg.levels
    assert len(far) <= max(1, int(0.1 * len(T_test))), (cfg.name, far)
    return far


def _subset_runner(R, g, idx):
    """groups_runner of group g, poses of the pairs idx only."""
    run = groups_runner(R, torch, g)
    return lambda sched: run(sched)[idx]


def test_register_groups_matches_per_group_register_and_oracle(R):
    """Uneven sizes in one call: each group's poses agree with those of a plain
    rimg_register of that group within the pose tolerance (the group call runs
    the coarse levels in the persistent queue's 256-thread blocks, which sum in
    another order than rimg_register's blocks), and sampled pairs match the
    oracle level by level."""
    groups, keep = _group_inputs(R, ["pair32x512", "lut64x512", "mixed128x1024_in"], [5, 3, 2])
    G = R.Groups(groups)
    ws = torch.empty(R.rimg_register_groups_workspace_bytes(G), dtype=torch.uint8, device="cuda")
    R.rimg_register_groups(G, ws)
    torch.cuda.synchronize()
    for g, (cfg, s, src, dst) in zip(groups, keep):
        Tref, _ = gpu_register(R, torch, g["src"], src, dst, np.tile(np.eye(4), (g["n_pairs"], 1, 1)), cfg.levels,
                               cfg.iters, g["params"])
        Tg = g["T_out"].cpu().numpy().reshape(-1, 4, 4)
        _agree_or_explained(R, g, cfg, s, src, dst, Tg, Tref)
        To, _ = oracle_register(src[0], dst[0], s, np.eye(4), cfg.levels, cfg.iters, oracle_params(cfg))
        eR, et = O.pose_error(Tg[0], To)
        assert eR <= 1e-4 and et <= 1e-4


def test_register_groups_queue_mixed_forms_and_degenerate_pairs(R):
    """The persistent small-level queue across kernel forms and edge cases in
    one call: a receiver-offset group (its own queue launch), a group with the
    distance gate (not queued), a group of zero pairs, a pair without any valid
    source pixel (degenerate: status flag, pose unchanged), repeated calls on
    the same workspace giving identical poses, against per-group rimg_register
    (pose tolerance) and statuses."""
    import dataclasses
    r0cfg = dataclasses.replace(CONFIGS["pair32x512"], name="pair32x512_r0", config_id=91, r0=0.015)
    kinds = [("pair32x512", 6, {}), (r0cfg, 3, {}), ("pair32x512", 2, dict(max_corr_dist=0.5)),
             ("mixed64x1024_out", 3, {}), ("pair32x512", 0, {})]
    groups, keep = [], []
    for kind, n, kw in kinds:
        cfg = CONFIGS[kind] if isinstance(kind, str) else kind
        s = cfg.sensor()
        sens = gpu_sensor(R, s, cfg.levels)
        if n:
            pairs = [make_pair(cfg, i) for i in range(n)]
            src = np.stack([q["src_range"] for q in pairs])
            dst = np.stack([q["dst_range"] for q in pairs])
        else:
            src = np.zeros((0, cfg.H, cfg.W), np.float32)
            dst = np.zeros((0, cfg.H, cfg.W), np.float32)
        if kind == "pair32x512" and not kw and n == 6:
            src[2] = 0.0                                  # no valid source pixel
        params = R.rimg_default_params(huber_delta=cfg.huber_delta, **kw)
        T0 = torch.eye(4, dtype=torch.float64, device="cuda").reshape(1, 16).repeat(max(n, 1), 1)[:n].contiguous()
        groups.append(dict(src=sens, dst=sens, n_pairs=n, levels=cfg.levels, iters=cfg.iters, params=params,
                           src_range=torch.from_numpy(src).cuda(), dst_range=torch.from_numpy(dst).cuda(),
                           T_init=T0, T_out=torch.empty_like(T0),
                           status=torch.full((n,), -5, dtype=torch.int32, device="cuda")))
        keep.append((cfg, src, dst))
    G = R.Groups(groups)
    ws = torch.empty(R.rimg_register_groups_workspace_bytes(G), dtype=torch.uint8, device="cuda")
    R.rimg_register_groups(G, ws)
    torch.cuda.synchronize()
    first = [g["T_out"].clone() for g in groups]
    R.rimg_register_groups(G, ws)
    torch.cuda.synchronize()
    for g, f in zip(groups, first):
        assert torch.equal(g["T_out"], f)
    for g, (cfg, src, dst) in zip(groups, keep):
        n = g["n_pairs"]
        if n == 0:
            continue
        Tg = g["T_out"].cpu().numpy().reshape(n, 4, 4)
        st = g["status"].cpu().numpy()
        ws1 = torch.empty(R.rimg_register_workspace_bytes(g["src"], g["src"], n, cfg.levels), dtype=torch.uint8,
                          device="cuda")
        T1 = torch.empty_like(g["T_init"])
        st1 = torch.full((n,), -5, dtype=torch.int32, device="cuda")
        R.rimg_register(g["src"], g["src"], n, g["src_range"], g["dst_range"], g["T_init"], T1, cfg.levels, cfg.iters,
                        g["params"], st1, ws1)
        torch.cuda.synchronize()
        Tref = T1.cpu().numpy().reshape(n, 4, 4)
        assert np.array_equal(st, st1.cpu().numpy()), (cfg.name, st, st1)
        for i in range(n):
            eR, et = O.pose_error(Tg[i], Tref[i])
            assert eR <= 1e-4 and et <= 1e-4, (cfg.name, i, eR, et)
        if cfg.name == "pair32x512" and g["params"].max_corr_dist == 0 and n == 6:
            assert st[2] & R.RIMG_FLAG_DEGENERATE and np.array_equal(Tg[2], np.eye(4))
            assert not np.any(st[[0, 1, 3, 4, 5]])


def test_autotune_keeps_results(R):
    """The autotuner only changes launch shapes and schedules: poses after
    tuning agree with the untuned ones within 1e-4, except where the other
    FP32 summation order of another block decomposition decided a near-tie
    association the other way; those pairs pass the per-level oracle check
    with the tuned launches."""
    groups, keep = _group_inputs(R, ["pair32x512", "lut64x512"], [40, 33])
    G = R.Groups(groups)
    ws = torch.empty(R.rimg_register_groups_workspace_bytes(G), dtype=torch.uint8, device="cuda")
    R.rimg_autotune_clear()
    R.rimg_register_groups(G, ws)
    torch.cuda.synchronize()
    before = [g["T_out"].cpu().numpy().reshape(-1, 4, 4) for g in groups]
    n_set = R.rimg_autotune(G, ws)
    assert n_set >= 0
    R.rimg_register_groups(G, ws)
    torch.cuda.synchronize()
    try:
        for g, b, (cfg, s, src, dst) in zip(groups, before, keep):
            a = g["T_out"].cpu().numpy().reshape(-1, 4, 4)
            if n_set == 0:        # the tuning was not faster: the table is as before
                assert np.array_equal(a, b)
            _agree_or_explained(R, g, cfg, s, src, dst, a, b)
    finally:
        R.rimg_autotune_clear()


def test_autotune_register_keeps_results(R):
    """rimg_autotune_register tunes a batch in rimg_register's own context;
    poses after tuning agree with the untuned ones or pass the per-level
    oracle check, and an empty result leaves the table (and the poses) as they
    were."""
    groups, keep = _group_inputs(R, ["pair32x512"], [40])
    g = groups[0]
    cfg, s, src, dst = keep[0]
    n = g["n_pairs"]
    ws = torch.empty(R.rimg_register_workspace_bytes(g["src"], g["src"], n, cfg.levels), dtype=torch.uint8,
                     device="cuda")
    T1 = torch.empty_like(g["T_init"])

    def reg():
        R.rimg_register(g["src"], g["src"], n, g["src_range"], g["dst_range"], g["T_init"], T1, cfg.levels,
                        cfg.iters, g["params"], None, ws)
        torch.cuda.synchronize()
        return T1.cpu().numpy().reshape(-1, 4, 4)

    R.rimg_autotune_clear()
    before = reg()
    try:
        n_set = R.rimg_autotune_register(g["src"], g["src"], n, g["src_range"], g["dst_range"], g["T_init"], T1,
                                         cfg.levels, cfg.iters, g["params"], ws)
        assert n_set >= 0
        assert np.array_equal(T1.cpu().numpy(), g["T_init"].cpu().numpy())    # T_out ends as T_init
        after = reg()
        if n_set == 0:
            assert np.array_equal(after, before)
        far = [i for i in range(n) if max(O.pose_error(after[i], before[i])) > 1e-4]
        if far:
            from tests.gpu_common import register_runner
            # the whole tuned batch (the table is keyed by the batch size), poses of the pairs `far`
            run = register_runner(R, torch, g["src"], g["src_range"], g["dst_range"], g["T_init"], cfg.levels,
                                  g["params"])
            rep = shadowed_check(R, torch, g["src"], s, src[far], dst[far], cfg.levels, cfg.iters, g["params"],
                                 oracle_params(cfg), runner=lambda sched: run(sched)[far])
            assert rep["levels_checked"] == len(far) * cfg.levels
        assert len(far) <= 4
        with pytest.raises(R.RimgError):
            R.rimg_autotune_register(g["src"], g["src"], n, g["src_range"], g["dst_range"], g["T_init"], T1,
                                     cfg.levels, cfg.iters, g["params"], ws[:1024])
    finally:
        R.rimg_autotune_clear()


def test_register_last_sums_record_the_final_step(R):
    """rimg_register_last_sums: the final step's sums (at the pose it started
    from) and the size of the update it applied, against the oracle's
    Gauss-Newton step from the same pose."""
    cfg = CONFIGS["pair32x512"]
    pair = make_pair(cfg, 3)
    s = pair["sensor"]
    sens = gpu_sensor(R, s, 1)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    T = O.se3_exp(np.array([2e-3, -1e-3, 3e-3, 0.02, -0.01, 0.015])) @ pair["T_gt"]
    src = torch.from_numpy(pair["src_range"])[None].cuda()
    dst = torch.from_numpy(pair["dst_range"])[None].cuda()
    T0 = torch.from_numpy(T.reshape(1, 16).copy()).cuda()
    T1 = torch.empty_like(T0)
    ws = torch.empty(R.rimg_register_workspace_bytes(sens, sens, 1, 1), dtype=torch.uint8, device="cuda")
    R.rimg_register(sens, sens, 1, src, dst, T0, T1, 1, [1], params, None, ws)
    rec = torch.zeros((1, 32), dtype=torch.float64, device="cuda")
    R.rimg_register_last_sums(sens, sens, 1, 1, ws, rec)
    torch.cuda.synchronize()
    rec = rec[0].cpu().numpy()
    tgt = O.Target(pair["dst_range"], s.phi_lut, s.theta_lut, s.r0, 1, f32(0.1))
    P, sv = O.source_points(pair["src_range"], s.phi_lut, s.theta_lut, s.r0, 0)
    rng_l, n_l, nv_l, ph, th = tgt.level(0)
    terms = O.icp_terms(P, sv, T, rng_l, n_l, nv_l, ph, th, s.r0, f32(params.huber_delta), 0.0,
                        dst_n_margin=tgt.nmargin[0])
    n_mis = int(np.sum(terms["near_tie"]))
    assert np.all(np.abs(rec[:29] - O.pack29(terms)) <= _sum_bounds(terms, n_mis) + 1e-9)
    xi, ok = O.cholesky_solve(terms["H"], terms["g"])
    assert ok and rec[31] == 1.0
    np.testing.assert_allclose(rec[29:31], [np.linalg.norm(xi[:3]), np.linalg.norm(xi[3:])], rtol=1e-3, atol=1e-9)
