"""Shadowed per-level comparison of a registration against the FP64 oracle.

TEST INFRASTRUCTURE ONLY (imported by the test-suite and the benchmark's
CPU-baseline leg; never by the library).  It runs the oracle from poses that
the caller supplies as plain arrays and shares no code with the CUDA path.

Multi-scale registration (Section 4.1) runs a fixed number of Gauss-Newton
steps per pyramid level, coarse to fine (schedule of Section 6.1).  Comparing
only the final poses of two implementations compounds every level's
difference.  Here each level is compared on its own: the oracle starts the
level from the pose the registration under test started it from, runs the
same number of steps, and the two level-end poses are compared.

Projective re-association is discrete, so a pose difference far below any
tolerance can still put a source point on the other side of a pixel boundary
a few steps later; on a pair whose iteration has not settled within the
schedule, such a flip can move the level-end pose further than the tolerance
even though every single step was computed correctly.  `explain_level`
checks that reading step by step for a level whose end poses disagree, from
the registration's own poses at every step of the level and its association
indices at those poses:

* its associations may differ from the oracle's at the same pose only on
  pixels the oracle flags as near-ties (`off_tie_mismatch` must be 0);
* with its associations imposed, the oracle's step from the same pose must
  land where the registration's step did (`step_err_given`: the step's
  arithmetic, apart from the discrete decisions);
* the trajectories split at the first step where a pixel is associated
  differently -- by the registration and the oracle at the same pose, or by
  the oracle at the registration's pose and at the pose of its own trajectory
  from the level's start (rounding-level pose differences moving a point
  across a boundary) -- and every pixel that differs there must be a
  near-tie (`split_off_tie` must be 0).
"""
import numpy as np

from . import rimg_oracle as O


def step_with_assoc(src_pts, src_valid, target, level, T, params, assoc, return_terms=False):
    """The oracle's Gauss-Newton step from T with the association indices
    `assoc` imposed (icp_terms' assoc argument): the step's arithmetic alone.
    return_terms adds the step's association terms."""
    rng_l, n_l, nv_l, ph, th = target.level(level)
    terms = O.icp_terms(src_pts, src_valid, T, rng_l, n_l, nv_l, ph, th, target.r0,
                        params.get("huber_delta", 0.5), params.get("max_corr_dist", 0.0), assoc=assoc)
    T_new, _ = O.gn_update(T, terms)
    return (T_new, terms) if return_terms else T_new


def system_condition(terms):
    """2-norm condition number of the step's 6x6 Gauss-Newton matrix
    J^T W J (the ratio of its extreme eigenvalues; inf when it is singular).
    A relative perturbation eps of the matrix and of the right-hand side
    moves the solution by up to about cond * eps * |x| (first-order
    perturbation bound of a linear system), which is how far reduced sums
    carried in a lower precision can move one step."""
    ev = np.linalg.eigvalsh(np.asarray(terms["H"], np.float64))
    return float(ev[-1] / ev[0]) if ev[0] > 0 else float("inf")


def run_level(src_pts, src_valid, target, level, T0, steps, params, keep_terms=False):
    """The oracle's Gauss-Newton steps at one level from T0: the poses after
    each step (T0 first) and, with keep_terms, each step's association terms."""
    poses, terms = [np.array(T0, np.float64)], []
    T = poses[0]
    for _ in range(steps):
        T, _, t = O.icp_step(src_pts, src_valid, target, level, T, params)
        poses.append(T)
        if keep_terms:
            terms.append(t)
    return poses, terms


def level_errors(src_range, dst_range, sensor, levels, iters, params, T_init, level_end):
    """Per-level shadowed errors.  level_end[k] is the pose the registration
    under test reached at the end of the k-th level of the schedule (coarse
    -> fine, `iters[k]` steps at pyramid level levels-1-k); the oracle runs the
    k-th level from level_end[k-1] (T_init for k = 0).  Returns an array
    [levels, 2] of (rad, m) errors and the oracle's level-end poses."""
    sp, st, r0 = sensor
    target = O.Target(dst_range, sp, st, r0, levels, params.get("normal_rel_jump", np.float32(0.1)),
                      params.get("normal_method", "cross"))
    err = np.zeros((levels, 2))
    ends = []
    for k in range(levels):
        l = levels - 1 - k
        P, sv = O.source_points(src_range, sp, st, r0, l)
        start = T_init if k == 0 else level_end[k - 1]
        poses, _ = run_level(P, sv, target, l, start, iters[k], params)
        ends.append(poses[-1])
        err[k] = O.pose_error(level_end[k], poses[-1])
    return err, ends


def explain_level(src_range, dst_range, sensor, levels, k, iters, params, traj, assoc):
    """Step-by-step reading of level k (schedule order) for a registration
    whose poses at that level are traj[0..iters[k]] (traj[0] the level start)
    and whose association indices at those poses are assoc[0..iters[k]-1]
    (flat, v * W_l + u or -1).  Returns a dict:

      step_err[j]         (rad, m) between traj[j+1] and the oracle's step from traj[j]
      step_err_given[j]   the same with the registration's associations at traj[j]
                          imposed on the oracle
      mismatch[j]         association indices that differ from the oracle's at traj[j]
      off_tie_mismatch[j] of those, the ones the oracle does not flag as near-ties
      split               first step j at which a pixel is associated differently by the
                          registration and the oracle at traj[j], or by the oracle at traj[j]
                          and at its own trajectory's pose (None: never)
      split_ties          pixels associated differently there
      split_off_tie       of those, the ones the oracle flags as near-ties at neither pose
      drift[j]            (rad, m) between traj[j] and the oracle's own trajectory
                          from traj[0]
      cond[j]             condition number of the step's 6x6 system with the
                          registration's associations imposed (system_condition)
      step_size[j]        size of that oracle step: its rotation angle (rad) and translation
                          change (m) combined as sqrt(angle^2 + change^2), mixed as in the solve
    """
    sp, st, r0 = sensor
    l = levels - 1 - k
    target = O.Target(dst_range, sp, st, r0, levels, params.get("normal_rel_jump", np.float32(0.1)),
                      params.get("normal_method", "cross"))
    P, sv = O.source_points(src_range, sp, st, r0, l)
    n = iters[k]
    out = dict(step_err=np.zeros((n, 2)), step_err_given=np.zeros((n, 2)), mismatch=np.zeros(n, int),
               off_tie_mismatch=np.zeros(n, int), split=None, split_ties=0, split_off_tie=0,
               drift=np.zeros((n + 1, 2)), cond=np.zeros(n), step_size=np.zeros(n))
    T_own = np.array(traj[0], np.float64)
    for j in range(n):
        out["drift"][j] = O.pose_error(traj[j], T_own)
        T_next, _, t = O.icp_step(P, sv, target, l, traj[j], params)
        T_own_next, _, ot = O.icp_step(P, sv, target, l, T_own, params)
        out["step_err"][j] = O.pose_error(traj[j + 1], T_next)
        a = np.asarray(assoc[j]).reshape(-1)
        diff_a = a != t["assoc"]
        out["mismatch"][j] = int(diff_a.sum())
        out["off_tie_mismatch"][j] = int((diff_a & ~t["near_tie"]).sum())
        T_given, t_given = step_with_assoc(P, sv, target, l, traj[j], params, a, return_terms=True)
        out["step_err_given"][j] = O.pose_error(traj[j + 1], T_given)
        out["cond"][j] = system_condition(t_given)
        out["step_size"][j] = float(np.hypot(*O.pose_error(T_given, traj[j])))
        diff_b = t["assoc"] != ot["assoc"]
        if out["split"] is None and (diff_a.any() or diff_b.any()):
            out["split"] = j
            out["split_ties"] = int((diff_a | diff_b).sum())
            out["split_off_tie"] = int((diff_a & ~t["near_tie"]).sum()
                                       + (diff_b & ~(t["near_tie"] | ot["near_tie"])).sum())
        T_own = T_own_next
    out["drift"][n] = O.pose_error(traj[n], T_own)
    return out
