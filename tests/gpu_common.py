"""Helpers shared by the GPU parity tests: build sensors and buffers, run the
library's entry points, and run the oracle on the same inputs."""
import numpy as np

from oracle import rimg_oracle as O

U32 = 2.0 ** -24     # unit roundoff of float32


def f32(x):
    return float(np.float32(x))


def oracle_params(cfg=None, huber=None, gate=0.0, jump=0.1):
    d = cfg.huber_delta if huber is None else huber
    return dict(huber_delta=f32(d), max_corr_dist=f32(gate), normal_rel_jump=f32(jump))


def gpu_sensor(R, sensor, levels):
    return R.rimg_sensor_build(sensor.H, sensor.W, levels, sensor.phi_lut, sensor.theta_lut, sensor.r0)


def planes_for(R, torch, sens, dst, params):
    """GPU plane pyramid (list per level) and finest mask for a batch [n, H, W]."""
    n = dst.shape[0]
    L = sens.levels
    planes = [torch.zeros((n, sens.H >> l, sens.W >> l, 4), dtype=torch.float32, device="cuda") for l in range(L)]
    mask = torch.zeros((n, sens.H, sens.W), dtype=torch.uint8, device="cuda")
    R.rimg_normals(sens, dst, params, planes, mask)
    return planes, mask


def src_pyramid(R, torch, sens, src):
    n = src.shape[0]
    out = [src] + [torch.zeros((n, sens.H >> l, sens.W >> l), dtype=torch.float32, device="cuda")
                   for l in range(1, sens.levels)]
    R.rimg_pyramid(n, sens.H, sens.W, sens.levels, 1, src, out)
    return out


def gpu_register(R, torch, sens, src_np, dst_np, T_init_np, levels, iters, params):
    n = src_np.shape[0]
    src = torch.from_numpy(np.ascontiguousarray(src_np)).cuda()
    dst = torch.from_numpy(np.ascontiguousarray(dst_np)).cuda()
    T0 = torch.from_numpy(np.ascontiguousarray(T_init_np.reshape(n, 16))).cuda()
    T1 = torch.empty_like(T0)
    status = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    ws = torch.empty(R.rimg_register_workspace_bytes(sens, sens, n, levels), dtype=torch.uint8, device="cuda")
    R.rimg_register(sens, sens, n, src, dst, T0, T1, levels, iters, params, status, ws)
    torch.cuda.synchronize()
    return T1.cpu().numpy().reshape(n, 4, 4), status.cpu().numpy()


def oracle_register(pair_src, pair_dst, sensor, T_init, levels, iters, params):
    sens = (sensor.phi_lut, sensor.theta_lut, sensor.r0)
    return O.register(pair_src, pair_dst, sens, sens, T_init, levels, iters, params)


# ---------------------------------------------------------------------------
# Shadowed per-level pose parity (the oracle side is oracle/shadow.py)

POSE_TOL = 1e-4        # rad and m: per-level final poses against the oracle
STEP_TOL = 1e-6        # rad and m: one Gauss-Newton step from the same pose and associations
# Relative error allowed in the reduced FP32 sums of one step: the terms'
# own FP32 rounding (one product and one sum each, u each) and the
# compensated reduction (about u): 4 u of FP32.  A step whose 6x6 system has
# condition number c and size |x| may then differ from the FP64 step by
# c * FP32_SUM_REL * |x| (first-order perturbation bound of a linear system);
# the step tolerance is the larger of that and STEP_TOL.
FP32_SUM_REL = 4 * 2.0 ** -24


def step_tolerance(cond, step_size, step_tol=STEP_TOL):
    """Per-step tolerance of the step-arithmetic comparison (rad and m).  A
    step of size zero (a degenerate system, skipped) has a zero perturbation
    bound whatever its condition number (a singular system has cond = inf;
    inf * 0 is taken as 0, not NaN)."""
    cond = np.asarray(cond, np.float64)
    size = np.asarray(step_size, np.float64)
    with np.errstate(invalid="ignore"):
        bound = np.where(size > 0, cond * FP32_SUM_REL * size, 0.0)
    return np.maximum(step_tol, bound)


def truncated_schedule(iters, k, j):
    """The schedule cut after the first k levels and j steps of level k."""
    return [iters[q] for q in range(k)] + [j] + [0] * (len(iters) - k - 1)


def register_runner(R, torch, sens, src_t, dst_t, T0_t, levels, params):
    """A function schedule -> poses [n, 4, 4] of the batch registered by
    rimg_register with that schedule (the same launches as the full
    registration, cut short: every earlier step is computed identically)."""
    ws = torch.empty(R.rimg_register_workspace_bytes(sens, sens, src_t.shape[0], levels), dtype=torch.uint8,
                     device="cuda")

    def run(sched):
        T1 = torch.empty_like(T0_t)
        R.rimg_register(sens, sens, src_t.shape[0], src_t, dst_t, T0_t, T1, levels, list(sched), params, None, ws)
        torch.cuda.synchronize()
        return T1.cpu().numpy().reshape(-1, 4, 4)
    return run


def groups_runner(R, torch, group):
    """A function schedule -> poses [n, 4, 4] of one rimg_register_groups
    group registered alone with that schedule (a group's sub-batches and its
    queue items do not depend on the other groups of a call)."""
    def run(sched):
        g = dict(group, iters=list(sched), T_out=torch.empty_like(group["T_init"]), status=None)
        G = R.Groups([g])
        ws = torch.empty(R.rimg_register_groups_workspace_bytes(G), dtype=torch.uint8, device="cuda")
        R.rimg_register_groups(G, ws)
        torch.cuda.synchronize()
        return g["T_out"].cpu().numpy().reshape(-1, 4, 4)
    return run


def gpu_assoc(R, torch, sens, src, dst, level, T, params):
    """Association indices [H_l * W_l] of one pair at pose T (rimg_icp_step
    with the association output, no update)."""
    s = 1 << level
    H, W = sens.H >> level, sens.W >> level
    sl = torch.from_numpy(np.ascontiguousarray(src[::s, ::s]))[None].cuda()
    dt = torch.from_numpy(np.ascontiguousarray(dst))[None].cuda()
    planes = [torch.zeros((1, sens.H >> q, sens.W >> q, 4), dtype=torch.float32, device="cuda")
              for q in range(sens.levels)]
    R.rimg_normals(sens, dt, params, planes)
    dl = torch.from_numpy(np.ascontiguousarray(dst[::s, ::s]))[None].cuda() if params.max_corr_dist > 0 else None
    pose = torch.from_numpy(np.ascontiguousarray(T.reshape(1, 16))).cuda()
    assoc = torch.full((1, H, W), -7, dtype=torch.int32, device="cuda")
    ws = torch.empty(R.rimg_icp_workspace_bytes(sens, 1), dtype=torch.uint8, device="cuda")
    R.rimg_icp_step(sens, sens, level, 1, sl, planes[level], dl, pose, params, 0, None, assoc, None, ws)
    torch.cuda.synchronize()
    return assoc[0].cpu().numpy().reshape(-1)


def _shadow_one(args):
    from oracle import shadow as SH
    src, dst, sens, levels, iters, o_params, T_init, ends = args
    err, _ = SH.level_errors(src, dst, sens, levels, iters, o_params, T_init, ends)
    return err


def _explain_one(args):
    from oracle import shadow as SH
    src, dst, sens, levels, k, iters, o_params, traj, assoc = args
    return SH.explain_level(src, dst, sens, levels, k, iters, o_params, traj, assoc)


def oracle_pool_map(fn, tasks, procs=None):
    import multiprocessing as mp
    import os
    procs = procs or max(1, min(32, (os.cpu_count() or 2) - 1, len(tasks)))
    env = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env}
    os.environ.update({k: "1" for k in env})
    try:
        if procs <= 1:
            return [fn(t) for t in tasks]
        with mp.get_context("spawn").Pool(procs) as pool:
            return pool.map(fn, tasks, chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def shadowed_check(R, torch, sens, sensor, src, dst, levels, iters, params, o_params, pairs=None, final=None,
                   T_init=None, pose_tol=POSE_TOL, step_tol=STEP_TOL, strict=True, runner=None):
    """Per-level parity of the batch registration of (src, dst) [n, H, W]
    against the oracle, on the pairs `pairs` (default all).

    Each level of the schedule is compared on its own: the oracle runs level
    k from the pose the GPU started it from and must end within pose_tol (rad
    and m) of the GPU's level-end pose.  A level that does not is accepted only
    with the step-by-step reading of oracle.shadow.explain_level: the GPU's
    association indices at each of its poses equal to the oracle's off
    near-ties, each GPU step within step_tol of the oracle's step from the
    same pose with the GPU's associations imposed, and the first pixel
    associated differently -- by the GPU and the oracle at one pose, or by
    the oracle at the GPU's pose and at its own trajectory's pose -- a
    near-tie, like every other pixel that differs at that step (where the
    trajectories split).  A level without such a split is accepted only when
    its steps are ill-conditioned enough that FP32 sums can move them beyond
    step_tol (some step's step_tolerance above it): the GPU's steps then
    match the oracle's within that bound and the level-end difference is the
    FP32 arithmetic the level amplifies ("conditioning" in the report; the
    others are "near-tie").  `final` (optional,
    [m, 4, 4] for the checked pairs) is the registration under test, which the
    truncated runs must reproduce bit for bit.  runner (optional): the
    function schedule -> GPU poses of the registration under test (default:
    rimg_register of the whole batch, see register_runner).  Returns a report
    dict; with
    strict (the tests) a level that is beyond pose_tol and not explained
    fails an assertion, otherwise it is only counted (the benchmark)."""
    n = src.shape[0]
    pairs = list(range(n)) if pairs is None else list(pairs)
    T_init = np.tile(np.eye(4), (n, 1, 1)) if T_init is None else np.asarray(T_init)
    if runner is None:
        src_t = torch.from_numpy(np.ascontiguousarray(src)).cuda()
        dst_t = torch.from_numpy(np.ascontiguousarray(dst)).cuda()
        T0_t = torch.from_numpy(np.ascontiguousarray(T_init.reshape(n, 16))).cuda()
        runner = register_runner(R, torch, sens, src_t, dst_t, T0_t, levels, params)
    ends = [runner(truncated_schedule(iters, k, iters[k])) for k in range(levels)]
    if final is not None:
        assert np.array_equal(ends[-1][pairs], np.asarray(final).reshape(-1, 4, 4)), "truncated runs differ"
    so = (sensor.phi_lut, sensor.theta_lut, sensor.r0)
    errs = oracle_pool_map(_shadow_one, [(src[i], dst[i], so, levels, iters, o_params, T_init[i],
                                          [ends[k][i] for k in range(levels)]) for i in pairs])
    report = dict(pairs=len(pairs), levels_checked=len(pairs) * levels, max_err=np.max(errs, axis=(0, 1)).tolist(),
                  beyond=[], explained=0, unexplained=0, by_kind={})
    bad = [(i, k) for i, e in zip(pairs, errs) for k in range(levels) if np.any(e[k] > pose_tol)]
    if not bad:
        return report
    trajs = {}
    for k in sorted({k for _, k in bad}):
        trajs[k] = [runner(truncated_schedule(iters, k, j)) for j in range(iters[k] + 1)]
    tasks = []
    for i, k in bad:
        l = levels - 1 - k
        traj = [trajs[k][j][i] for j in range(iters[k] + 1)]
        assoc = [gpu_assoc(R, torch, sens, src[i], dst[i], l, traj[j], params) for j in range(iters[k])]
        tasks.append((src[i], dst[i], so, levels, k, iters, o_params, traj, assoc))
    expl = oracle_pool_map(_explain_one, tasks)
    for (i, k), e, err in zip(bad, expl, [errs[pairs.index(i)][k] for i, k in bad]):
        rec = dict(pair=i, level_index=k, err=err.tolist(), split=e["split"], split_ties=int(e["split_ties"]),
                   split_off_tie=int(e["split_off_tie"]),
                   split_drift=(e["drift"][e["split"]].tolist() if e["split"] is not None else None),
                   step_err_given_max=np.max(e["step_err_given"], 0).tolist(),
                   step_err_max=np.max(e["step_err"], 0).tolist(), mismatch=int(e["mismatch"].sum()),
                   off_tie_mismatch=int(e["off_tie_mismatch"].sum()), cond_max=float(np.max(e["cond"])))
        report["beyond"].append(rec)
        tol = step_tolerance(e["cond"], e["step_size"], step_tol)
        steps_ok = rec["off_tie_mismatch"] == 0 and np.all(e["step_err_given"] <= tol[:, None])
        if e["split"] is not None:
            kind = "near-tie" if rec["split_off_tie"] == 0 else None
        else:
            kind = "conditioning" if np.any(tol > step_tol) else None
        ok = bool(steps_ok and kind is not None)
        rec["kind"] = kind if ok else None
        if ok:
            report["by_kind"][kind] = report["by_kind"].get(kind, 0) + 1
        rec["explained"] = bool(ok)
        if strict:
            assert ok, rec
        report["explained" if ok else "unexplained"] += 1
    return report
