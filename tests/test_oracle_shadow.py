"""Pins of the step-by-step reading (oracle/shadow.py) that the per-level
parity tests use to accept a level beyond the pose tolerance: it must report
the oracle's own trajectory as matching to rounding, find a step that was
planted wrong in a trajectory, count an association that was planted off a
near-tie, and give the condition number of a system with known eigenvalues."""
import numpy as np
import pytest

from oracle import rimg_oracle as O
from oracle import shadow
from synth import CONFIGS, make_pair
from tests.gpu_common import STEP_TOL, FP32_SUM_REL, oracle_params, step_tolerance

CFG = CONFIGS["pair32x512"]
K = 0                      # schedule index 0: the coarsest level (8 x 128)


@pytest.fixture(scope="module")
def case():
    p = make_pair(CFG, 1)
    s = CFG.sensor()
    so = (s.phi_lut, s.theta_lut, s.r0)
    params = oracle_params(CFG)
    l = CFG.levels - 1 - K
    target = O.Target(p["dst_range"], *so, CFG.levels, params["normal_rel_jump"], "cross")
    P, sv = O.source_points(p["src_range"], *so, l)
    traj, assoc = [np.eye(4)], []
    for _ in range(CFG.iters[K]):
        T, _, t = O.icp_step(P, sv, target, l, traj[-1], params)
        assoc.append(t["assoc"].copy())
        traj.append(T)
    return dict(src=p["src_range"], dst=p["dst_range"], so=so, params=params, traj=traj, assoc=assoc,
                target=target, P=P, sv=sv, l=l, near=[])


def _explain(case, traj, assoc):
    return shadow.explain_level(case["src"], case["dst"], case["so"], CFG.levels, K, CFG.iters, case["params"],
                                traj, assoc)


def test_own_trajectory_matches_exactly(case):
    e = _explain(case, case["traj"], case["assoc"])
    assert np.all(e["step_err"] == 0) and np.all(e["step_err_given"] == 0)
    assert np.all(e["mismatch"] == 0) and e["split"] is None and np.all(e["drift"] == 0)
    assert np.all(np.isfinite(e["cond"])) and np.all(e["cond"] >= 1)
    # the step sizes are those of the trajectory itself
    for j in range(len(case["assoc"])):
        assert e["step_size"][j] == pytest.approx(np.hypot(*O.pose_error(case["traj"][j + 1], case["traj"][j])))


def test_planted_step_error_is_found_at_its_step(case):
    j = 3
    traj = [T.copy() for T in case["traj"]]
    c, s = np.cos(1e-3), np.sin(1e-3)
    Rz = np.eye(4)
    Rz[:2, :2] = [[c, -s], [s, c]]
    traj[j + 1] = Rz @ traj[j + 1]            # one step 1 mrad off; the later ones start from there
    assoc = list(case["assoc"])
    P, sv, tg, l, prm = case["P"], case["sv"], case["target"], case["l"], case["params"]
    for i in range(j + 1, len(assoc)):
        T, _, t = O.icp_step(P, sv, tg, l, traj[i], prm)
        assoc[i] = t["assoc"].copy()
        traj[i + 1] = T
    e = _explain(case, traj, assoc)
    assert e["step_err_given"][j, 0] == pytest.approx(1e-3, rel=1e-6)
    assert e["step_err"][j, 0] == pytest.approx(1e-3, rel=1e-6)
    others = [i for i in range(len(assoc)) if i != j]
    assert np.all(e["step_err_given"][others] < 1e-12)
    assert np.all(e["mismatch"] == 0)
    assert e["drift"][j + 1, 0] == pytest.approx(1e-3, rel=1e-6)


def test_planted_association_off_a_near_tie_is_counted(case):
    j = 2
    t = O.icp_step(case["P"], case["sv"], case["target"], case["l"], case["traj"][j], case["params"])[2]
    a = case["assoc"][j].copy()
    cand = np.flatnonzero((a >= 0) & ~t["near_tie"])
    assert cand.size > 0
    px = cand[cand.size // 2]
    a[px] = (a[px] + 5) % (case["target"].level(case["l"])[0].size)     # a pixel five columns away
    assoc = list(case["assoc"])
    assoc[j] = a
    e = _explain(case, case["traj"], assoc)
    assert e["mismatch"][j] == 1 and e["off_tie_mismatch"][j] == 1
    assert e["split"] == j and e["split_off_tie"] == 1
    assert e["mismatch"].sum() == 1


def test_system_condition_of_known_spectrum():
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    lam = np.array([0.5, 1.0, 2.0, 4.0, 8.0, 50.0])
    H = Q @ np.diag(lam) @ Q.T
    assert shadow.system_condition({"H": H}) == pytest.approx(100.0, rel=1e-9)
    H0 = Q @ np.diag([0.0, 1, 2, 3, 4, 5]) @ Q.T
    assert shadow.system_condition({"H": H0}) == float("inf") or shadow.system_condition({"H": H0}) > 1e14


def test_step_tolerance_floor_and_scaling():
    assert step_tolerance(1.0, 1e-3) == STEP_TOL
    big = step_tolerance(1e4, 10.0)
    assert big == pytest.approx(1e4 * FP32_SUM_REL * 10.0)
    np.testing.assert_allclose(step_tolerance([1.0, 1e4], [1e-3, 10.0]), [STEP_TOL, big])
    # a skipped step (singular system: cond inf, size 0) keeps the floor, not NaN;
    # a step taken on a singular system is unbounded
    np.testing.assert_array_equal(step_tolerance([np.inf, np.inf], [0.0, 1.0]), [STEP_TOL, np.inf])
