"""Learned pose proposal: training set, training loop and evaluation driver.

Host logic only: the scans are cast by synth's GPU ray caster, the labels,
coarse images, proposals, gradients and optimizer steps all come from
librimg's kernels (rimg_register, rimg_pyramid, rimg_propose,
rimg_cnn_train_step); torch holds device memory and draws minibatch indices.

Workload (64 x 1024 scans, HDL-64-like elevation table, 200 objects,
rot <= 15 deg, trans <= 3 m; the "learn64x1024" configuration):
  * label of a pair: the pose the plain multi-scale method converges to when
    started at the ground truth (4 levels x 10 iterations, Section 6.1);
  * network input: the coarsest pyramid level (8 x 128) of both scans;
  * evaluation on held-out pairs: the plain method from the identity with
    the full schedule against the proposal T0 followed by shorter schedules,
    pose error against the label, and pairs/s of each pipeline.  The
    registration judges each proposal-started result by its own convergence:
    the Gauss-Newton step xi = -(J^T W J)^-1 J^T W e of its last iteration
    (from rimg_register_last_sums).  A pair whose last step is larger than
    the threshold taken from the labelled training runs is registered again
    by the plain method from the identity (the fallback).

    python -m paper_2112_02779_b300.learned --train 100000 --test 10000 --out report.json
"""
import argparse
import json
import math
import os
import time

import numpy as np

CFG = "learn64x1024"
SUCCESS_ROT = 1e-3        # rad: a result counts as converged to the label within these
SUCCESS_TRANS = 1e-2      # m


def _torch():
    import torch
    return torch


def pose_errors(T, T_ref):
    """Rotation angle (rad) and translation distance (m), arrays [n] (host)."""
    T = np.asarray(T).reshape(-1, 4, 4)
    T_ref = np.asarray(T_ref).reshape(-1, 4, 4)
    M = np.einsum("nij,nkj->nik", T[:, :3, :3], T_ref[:, :3, :3])
    c = np.clip((np.trace(M, axis1=1, axis2=2) - 1.0) / 2.0, -1.0, 1.0)
    return np.arccos(c), np.linalg.norm(T[:, :3, 3] - T_ref[:, :3, 3], axis=1)


class Registrar:
    """rimg_register over batches of device images, with cached workspaces."""

    def __init__(self, cfg, R):
        self.cfg, self.R = cfg, R
        s = cfg.sensor()
        self.sens = R.rimg_sensor_build(cfg.H, cfg.W, cfg.levels, s.phi_lut, s.theta_lut, s.r0)
        self.params = R.rimg_default_params(huber_delta=cfg.huber_delta)
        self._ws = {}

    def workspace(self, n):
        torch = _torch()
        ws = self._ws.get(n)
        if ws is None:
            nb = self.R.rimg_register_workspace_bytes(self.sens, self.sens, n, self.cfg.levels)
            ws = self._ws[n] = torch.empty(nb, dtype=torch.uint8, device="cuda")
        return ws

    def __call__(self, src, dst, T_init, iters, fitness=False):
        """T_out [n, 16] (and the last step's record [n, 32] when fitness)."""
        torch = _torch()
        n = src.shape[0]
        T_out = torch.empty((n, 16), dtype=torch.float64, device="cuda")
        ws = self.workspace(n)
        self.R.rimg_register(self.sens, self.sens, n, src, dst, T_init, T_out, self.cfg.levels, list(iters),
                             self.params, None, ws)
        if not fitness:
            return T_out
        s32 = torch.empty((n, 32), dtype=torch.float64, device="cuda")
        self.R.rimg_register_last_sums(self.sens, self.sens, n, self.cfg.levels, ws, s32)
        return T_out, s32

    def coarse(self, img):
        """The coarsest pyramid level of [n, H, W] images (rimg_pyramid)."""
        torch = _torch()
        n, H, W = img.shape
        L = self.cfg.levels
        out = [img] + [torch.empty((n, H >> l, W >> l), dtype=torch.float32, device="cuda") for l in range(1, L)]
        self.R.rimg_pyramid(n, H, W, L, 1, img, out)
        return out[-1]


def last_step(s32):
    """Rotation (rad) and translation (m) size of each pair's last
    Gauss-Newton update, as recorded by the solve kernel (host copy);
    inf where the last update was skipped (degenerate system)."""
    s = s32.cpu().numpy() if hasattr(s32, "cpu") else np.asarray(s32)
    out = s[:, 29:31].copy()
    out[s[:, 31] == 0] = np.inf
    return out


def make_dataset(reg, indices, keep_full=False, chunk=8192, processes=1, label_iters=None, log=print):
    """Cast pairs on the GPU and label them.  Returns dict of device tensors:
    src_c, dst_c [n, 8, 128]; T_gt, T_label [n, 16]; label_step [n, 2]
    (host: the last Gauss-Newton step of each label run); src, dst [n, H, W]
    when keep_full."""
    torch = _torch()
    from synth import gpu as G
    cfg = reg.cfg
    indices = list(indices)
    parts = {k: [] for k in ("src_c", "dst_c", "T_gt", "T_label", "src", "dst")}
    steps = []
    t0 = time.time()
    for c0 in range(0, len(indices), chunk):
        idx = indices[c0:c0 + chunk]
        drawn = G.draw_pairs(cfg, idx, processes)
        src, dst, T = G.make_pairs_gpu(cfg, idx, drawn=drawn)
        T_gt = torch.from_numpy(T.reshape(len(idx), 16)).cuda()
        T_label, s32 = reg(src, dst, T_gt, label_iters or cfg.iters, fitness=True)
        steps.append(last_step(s32))
        parts["src_c"].append(reg.coarse(src))
        parts["dst_c"].append(reg.coarse(dst))
        parts["T_gt"].append(T_gt)
        parts["T_label"].append(T_label)
        if keep_full:
            parts["src"].append(src)
            parts["dst"].append(dst)
        log(f"  pairs {c0 + len(idx)}/{len(indices)}  {time.time() - t0:.1f} s")
    out = {k: torch.cat(v) for k, v in parts.items() if v}
    out["label_step"] = np.concatenate(steps)
    return out


def lr_at(step, steps, lr, lr_min, warmup):
    if step <= warmup:
        return lr * step / warmup
    q = (step - warmup) / max(1, steps - warmup)
    return lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * q))


def train(R, net, data, steps, batch=256, lr=1e-3, lr_min=1e-5, warmup=200, seed=0, log=print, log_every=500):
    torch = _torch()
    N = data["src_c"].shape[0]
    g = torch.Generator(device="cuda").manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    hist = []
    t0 = time.time()
    for step in range(1, steps + 1):
        idx = torch.randint(0, N, (batch,), generator=g, device="cuda", dtype=torch.int32)
        R.rimg_cnn_train_step(net, data["src_c"], data["dst_c"], data["T_label"], step,
                              lr=lr_at(step, steps, lr, lr_min, warmup), index=idx, loss=loss)
        if step % log_every == 0 or step == steps:
            hist.append((step, loss.item()))
            log(f"  step {step}  loss {hist[-1][1]:.5f}  {time.time() - t0:.1f} s")
    torch.cuda.synchronize()
    if net.err.item() != 0:
        raise RuntimeError("a tensor-core wait timed out during training")
    return hist, time.time() - t0


def propose(R, net, src, dst, chunk=8192):
    torch = _torch()
    n = src.shape[0]
    T0 = torch.empty((n, 16), dtype=torch.float64, device="cuda")
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        R.rimg_propose(net, src[c0:c1], dst[c0:c1], T_out=T0[c0:c1])
    return T0


def _timed(fn, reps=3):
    torch = _torch()
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return best


def summarize(err_r, err_t):
    ok = (err_r <= SUCCESS_ROT) & (err_t <= SUCCESS_TRANS)
    return {"success": float(ok.mean()), "median_rot_rad": float(np.median(err_r)),
            "median_trans_m": float(np.median(err_t)), "p95_rot_rad": float(np.quantile(err_r, 0.95)),
            "p95_trans_m": float(np.quantile(err_t, 0.95))}


# plain schedules of the ablation beside the proposal's own schedules: fewer
# iterations on every level, or on the coarse levels only
PLAIN_ABLATION = [(10, 8, 8, 8), (10, 6, 6, 6), (10, 5, 5, 5), (10, 10, 10, 5), (8, 8, 8, 8), (6, 6, 6, 6),
                  (5, 5, 5, 5), (5, 10, 10, 10)]
MATCH_SUCCESS = 0.005     # two pipelines count as equally accurate when their success rates differ by less


def evaluate(R, net, reg, test, schedules, tau, timing_pairs=4096, log=print, plain_schedules=None):
    """Plain (identity start, full schedule) against proposal + each schedule
    with the convergence judge (last step above tau = (rad, m): rejected) and
    the plain fallback.

    Ablation: the plain method from the identity is also run at every
    schedule of `schedules` and of `plain_schedules`, so that a gain is
    claimed only against the fastest plain schedule that is as accurate:
    each proposal entry gets `matched_plain`, the fastest plain run whose
    success rate is at least the entry's minus MATCH_SUCCESS, and
    `gain_vs_matched` = its pairs/s over that run's."""
    torch = _torch()
    cfg = reg.cfg
    src, dst = test["src"], test["dst"]
    n = src.shape[0]
    label = test["T_label"].cpu().numpy()
    eye = torch.eye(4, dtype=torch.float64, device="cuda").reshape(1, 16).repeat(n, 1)
    full = tuple(cfg.iters)
    T_plain = reg(src, dst, eye, full).cpu().numpy()
    gt = test["T_gt"].cpu().numpy()
    res = {"pairs": n, "plain": {"iters": list(full), **summarize(*pose_errors(T_plain, label)),
                                 "vs_gt": summarize(*pose_errors(T_plain, gt))}}
    T0 = propose(R, net, src, dst)
    res["proposal_only"] = summarize(*pose_errors(T0.cpu().numpy(), label))
    res["identity_start"] = summarize(*pose_errors(np.tile(np.eye(4), (n, 1, 1)), label))
    # timing on the first timing_pairs pairs
    m = min(n, timing_pairs)
    s_m, d_m, e_m = src[:m], dst[:m], eye[:m]
    t_plain = _timed(lambda: reg(s_m, d_m, e_m, full))
    res["plain"]["pairs_per_s"] = m / t_plain
    # the ablation: plain from the identity at every schedule
    res["plain_schedules"] = [dict(res["plain"], iters=list(full))]
    seen = {tuple(full)}
    for sched in list(schedules) + list(plain_schedules or []):
        if tuple(sched) in seen:
            continue
        seen.add(tuple(sched))
        T_p = reg(src, dst, eye, sched).cpu().numpy()
        entry = {"iters": list(sched), **summarize(*pose_errors(T_p, label))}
        entry["pairs_per_s"] = m / _timed(lambda: reg(s_m, d_m, e_m, sched))
        res["plain_schedules"].append(entry)
        log(f"  plain {sched}: success {entry['success']:.4f}, {entry['pairs_per_s']:.0f} pairs/s")
    res["learned"] = []
    for sched in schedules:
        T_l, s32 = reg(src, dst, T0, sched, fitness=True)
        stp = last_step(s32)
        T_l = T_l.cpu().numpy()
        rej = (stp[:, 0] > tau[0]) | (stp[:, 1] > tau[1])
        T_j = T_l.copy()
        T_j[rej] = T_plain[rej]                  # fallback: the plain method's result
        er, et = pose_errors(T_l, label)
        jr, jt = pose_errors(T_j, label)
        entry = {"iters": list(sched), "no_judge": summarize(er, et), "judged": summarize(jr, jt),
                 "judged_vs_gt": summarize(*pose_errors(T_j, gt)), "rejected": float(rej.mean())}

        rej_m = torch.from_numpy(np.nonzero(rej[:m])[0]).cuda()

        def pipeline():
            T0m = torch.empty((m, 16), dtype=torch.float64, device="cuda")
            R.rimg_propose(net, s_m, d_m, T_out=T0m)
            Tm, s = reg(s_m, d_m, T0m, sched, fitness=True)
            last_step(s)                         # the judge, on the host
            if rej_m.numel():
                k = rej_m.numel()
                reg(s_m.index_select(0, rej_m), d_m.index_select(0, rej_m), e_m[:k], full)
            return Tm

        t_l = _timed(pipeline)
        entry["pairs_per_s"] = m / t_l
        same = [p for p in res["plain_schedules"] if p["success"] >= entry["judged"]["success"] - MATCH_SUCCESS]
        if same:
            best = max(same, key=lambda p: p["pairs_per_s"])
            entry["matched_plain"] = {"iters": best["iters"], "success": best["success"],
                                      "pairs_per_s": best["pairs_per_s"]}
            entry["gain_vs_matched"] = entry["pairs_per_s"] / best["pairs_per_s"]
        else:
            entry["matched_plain"] = None            # more accurate than every plain schedule
            entry["gain_vs_matched"] = None
        res["learned"].append(entry)
        mp = entry["matched_plain"]
        log(f"  sched {sched}: success {entry['judged']['success']:.4f} (no judge {entry['no_judge']['success']:.4f}),"
            f" rejected {entry['rejected']:.4f}, {entry['pairs_per_s']:.0f} pairs/s"
            f" (plain {res['plain']['success']:.4f}, {res['plain']['pairs_per_s']:.0f} pairs/s; fastest plain as"
            f" accurate: {mp['iters'] if mp else None}, gain {entry['gain_vs_matched']})")
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=100000)
    ap.add_argument("--test", type=int, default=10000)
    ap.add_argument("--steps", type=int, default=0, help="0: 30 epochs of the training set")
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--processes", type=int, default=max(1, min(16, (os.cpu_count() or 2) - 1)))
    ap.add_argument("--label-iters", default="10,10,10,10", help="schedule of the label runs (from T_gt)")
    ap.add_argument("--out", default=None)
    ap.add_argument("--save", default=None, help="write the trained FP32 parameters (.npy)")
    a = ap.parse_args(argv)
    torch = _torch()
    from . import rimg as R
    from synth import CONFIGS
    cfg = CONFIGS[CFG]
    reg = Registrar(cfg, R)
    report = {"workload": f"{CFG}: {cfg.H}x{cfg.W}, {cfg.n_objects} objects, rot <= {cfg.rot_max_deg} deg, "
                          f"trans <= {cfg.trans_max} m, labels from the plain method started at T_gt "
                          f"({cfg.levels} levels x {list(cfg.iters)})",
              "train_pairs": a.train, "test_pairs": a.test}
    t0 = time.time()
    label_iters = tuple(int(x) for x in a.label_iters.split(","))
    report["label_iters"] = list(label_iters)
    print("training set")
    train_set = make_dataset(reg, range(a.train), processes=a.processes, label_iters=label_iters)
    print("test set")
    test_set = make_dataset(reg, range(a.train, a.train + a.test), keep_full=True, processes=a.processes,
                            label_iters=label_iters)
    report["data_seconds"] = time.time() - t0
    st = train_set["label_step"]
    report["label_last_step_quantiles"] = {q: [float(np.quantile(st[:, 0], q)), float(np.quantile(st[:, 1], q))]
                                           for q in (0.5, 0.9, 0.99)}
    tau = (float(np.quantile(st[:, 0], 0.99)), float(np.quantile(st[:, 1], 0.99)))
    report["judge_threshold"] = {"last_step_rot_rad": tau[0], "last_step_trans_m": tau[1],
                                 "rule": "99th percentile of the label runs' last Gauss-Newton step"}
    lab_err = pose_errors(train_set["T_label"].cpu().numpy(), train_set["T_gt"].cpu().numpy())
    report["label_vs_gt_median"] = [float(np.median(lab_err[0])), float(np.median(lab_err[1]))]
    net = R.ProposalNet(seed=a.seed)
    steps = a.steps or 30 * max(1, a.train // a.batch)
    print(f"training {steps} steps")
    hist, t_train = train(R, net, train_set, steps, batch=a.batch, lr=a.lr, seed=a.seed)
    report.update(train_steps=steps, batch=a.batch, train_seconds=t_train, loss_history=hist)
    print("evaluation")
    L = cfg.levels
    schedules = [(k,) + tuple(cfg.iters[1:]) for k in (0, 2, 5, 10)] + [
        (2, 8, 8, 8), (2, 7, 7, 7), (2, 6, 6, 6), (2, 5, 5, 5), (2, 3, 3, 3), (2, 10, 10, 5), (2, 5, 5, 8),
        (2, 3, 3, 8)]
    schedules = [s[:L] for s in schedules]
    plain_extra = [s[:L] for s in PLAIN_ABLATION]
    report["eval"] = evaluate(R, net, reg, test_set, schedules, tau, plain_schedules=plain_extra)
    if a.save:
        np.save(a.save, net.params.cpu().numpy())
    if a.out:
        with open(a.out, "w") as f:
            json.dump(report, f, indent=1)
    print(json.dumps({k: v for k, v in report.items() if k != "loss_history"}, indent=1))


if __name__ == "__main__":
    main()
