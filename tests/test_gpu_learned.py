"""What the trained proposal network gains over the method without it, on
held-out pairs of the large-motion workload (64 x 1024, rot <= 15 deg,
trans <= 3 m), at a reduced scale (20 000 training pairs, 3 000 steps, 4 000
test pairs; the full 100 000 / 10 000 run is the module's command line).

The gain is measured against the plain method run from the identity at every
schedule of the evaluation (the proposal's shortened schedules and further
ones with fewer coarse or fine iterations): a proposal pipeline must beat, in
pairs/s, the fastest plain schedule that is as accurate (success rate within
0.005), not just the plain method's full schedule.

Deterministic: seeded pairs, seeded minibatches, and kernels without atomics
or data-dependent summation order."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_02779_b300.rimg as R
    from paper_2112_02779_b300 import learned as Lr
    from synth import CONFIGS
    cfg = CONFIGS[Lr.CFG]
    reg = Lr.Registrar(cfg, R)
    quiet = lambda *a, **k: None  # noqa: E731
    train = Lr.make_dataset(reg, range(20000), processes=4, log=quiet)
    test = Lr.make_dataset(reg, range(20000, 24000), keep_full=True, processes=4, log=quiet)
    net = R.ProposalNet(seed=1)
    hist, _ = Lr.train(R, net, train, 3000, log=quiet)
    st = train["label_step"]
    tau = (float(np.quantile(st[:, 0], 0.99)), float(np.quantile(st[:, 1], 0.99)))
    res = Lr.evaluate(R, net, reg, test, [(2, 10, 10, 10), (2, 6, 6, 6), (2, 5, 5, 5)], tau, timing_pairs=4000,
                      log=print, plain_schedules=Lr.PLAIN_ABLATION)
    print("plain", res["plain"])
    for e in res["learned"]:
        print("learned", e["iters"], e["judged"]["success"], e["pairs_per_s"], e["matched_plain"], e["gain_vs_matched"])
    return hist, res


def test_training_converges(run):
    hist, _ = run
    assert hist[-1][1] < 0.5 * hist[0][1]


def test_proposal_is_closer_than_the_identity(run):
    _, res = run
    p, i = res["proposal_only"], res["identity_start"]
    assert p["median_rot_rad"] < 0.6 * i["median_rot_rad"]
    assert p["median_trans_m"] < 0.6 * i["median_trans_m"]


def test_fewer_coarse_iterations_at_equal_accuracy(run):
    """2 instead of 10 iterations on the coarsest level after the proposal:
    as accurate as the plain method's full schedule (within 0.005)."""
    _, res = run
    plain = res["plain"]
    l2 = res["learned"][0]
    assert l2["iters"] == [2, 10, 10, 10]
    assert l2["judged"]["success"] >= plain["success"] - 0.005
    assert l2["judged"]["median_rot_rad"] <= 1.2 * plain["median_rot_rad"]


def test_ablation_covers_the_proposal_schedules(run):
    """The plain method was run from the identity at every schedule the
    proposal was evaluated at."""
    _, res = run
    plain_iters = {tuple(p["iters"]) for p in res["plain_schedules"]}
    assert all(tuple(e["iters"]) in plain_iters for e in res["learned"])


def test_proposal_beats_the_fastest_equally_accurate_plain_schedule(run):
    """Some proposal pipeline (proposal + shortened schedule + judge +
    fallback) is faster than every plain schedule that is as accurate, and
    its success rate is within 0.005 of that plain schedule's."""
    _, res = run
    wins = [e for e in res["learned"] if e["matched_plain"] is not None and e["gain_vs_matched"] > 1.0
            and e["judged"]["success"] >= e["matched_plain"]["success"] - 0.005]
    assert wins, [(e["iters"], e["judged"]["success"], e["pairs_per_s"], e["matched_plain"]) for e in res["learned"]]
