"""What the trained proposal network gains over the method without it, on
held-out pairs of the large-motion workload (64 x 1024, rot <= 15 deg,
trans <= 3 m), at a reduced scale (20 000 training pairs, 3 000 steps, 4 000
test pairs; the full 100 000 / 10 000 run is the module's command line).

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
    res = Lr.evaluate(R, net, reg, test, [(2, 10, 10, 10), (2, 5, 5, 5)], tau, timing_pairs=4000, log=print)
    print("plain", res["plain"])
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
    _, res = run
    plain = res["plain"]
    l2 = res["learned"][0]            # 2 instead of 10 iterations on the coarsest level
    assert l2["judged"]["success"] >= plain["success"]
    assert l2["judged"]["median_rot_rad"] <= 1.2 * plain["median_rot_rad"]


def test_shorter_schedule_is_faster_at_about_equal_accuracy(run):
    _, res = run
    plain = res["plain"]
    l0 = res["learned"][1]            # proposal, then 2 / 5 / 5 / 5 iterations
    assert l0["judged"]["success"] >= plain["success"] - 0.03
    assert l0["pairs_per_s"] >= 1.2 * plain["pairs_per_s"]
