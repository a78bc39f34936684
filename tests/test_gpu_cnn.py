"""The proposal network's CUDA path (tcgen05 GEMMs, im2col / col2im,
transposes, loss, Adam) against the FP64 oracle of the same network.

Tolerances.  The oracle with BF16 rounding emulated at the network's rounding
points differs from the GPU only by FP32 accumulation order and by the rare
BF16 rounding that lands on the other side of a rounding boundary; outputs
agree to ~1e-3 of their scale (the bar: 5e-3).  Against the plain FP64
network the BF16 path differs by a few per cent of the gradient's norm (the
bar: 10%, as for the oracle's own BF16-vs-FP64 check)."""
import numpy as np
import pytest

from oracle import cnn_oracle as C
from synth import CONFIGS, make_pairs, random_delta_pose

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_02779_b300.rimg as R
    return R


def _params(rng):
    out = []
    for cin, cout in C.LAYERS:
        out.append((rng.normal(size=(cout, 9 * cin)) * np.sqrt(2.0 / (9 * cin)), rng.normal(size=cout) * 0.05))
    out.append((rng.normal(size=(6, 512)) * np.sqrt(1.0 / 512), rng.normal(size=6) * 0.05))
    return C.pack(out).astype(np.float32)


@pytest.fixture(scope="module")
def scans():
    """Six 64 x 1024 scan pairs (full images; the network reads stride 8)."""
    src, dst, T = make_pairs(CONFIGS["pair64x1024"], range(6))
    return src, dst, T


def _labels(rng, n):
    return np.stack([random_delta_pose(rng, 15.0, 3.0) for _ in range(n)])


def _batch(rng, scans, n):
    """n pairs: the six scans, then seeded random images with invalid pixels."""
    src, dst, _ = scans
    k = min(n, src.shape[0])
    s = np.concatenate([src[:k, ::8, ::8], rng.uniform(0.5, 80.0, (n - k, 8, 128))]).astype(np.float32)
    d = np.concatenate([dst[:k, ::8, ::8], rng.uniform(0.5, 80.0, (n - k, 8, 128))]).astype(np.float32)
    s[k:][rng.random(s[k:].shape) < 0.15] = 0.0
    d[k:][rng.random(d[k:].shape) < 0.15] = np.nan
    return s, d


def _net(R, theta):
    net = R.ProposalNet(params=torch.from_numpy(theta).cuda())
    return net


@pytest.mark.parametrize("n", [1, 6, 37, 300])
def test_forward_matches_oracle(R, scans, n):
    rng = np.random.default_rng(100 + n)
    theta = _params(rng)
    s, d = _batch(rng, scans, n)
    net = _net(R, theta)
    pred = torch.zeros((n, 6), device="cuda")
    T = torch.zeros((n, 16), dtype=torch.float64, device="cuda")
    R.rimg_propose(net, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), pred=pred, T_out=T)
    torch.cuda.synchronize()
    assert net.err.item() == 0
    x = C.net_input(s, d)
    pq, _ = C.forward(theta.astype(np.float64), x, q=C.bf16_round)
    p64, _ = C.forward(theta.astype(np.float64), x)
    g = pred.cpu().numpy()
    scale = max(1.0, np.abs(pq).max())
    assert np.abs(g - pq).max() <= 5e-3 * scale, np.abs(g - pq).max()
    assert np.linalg.norm(g - p64) <= 0.05 * np.linalg.norm(p64)
    To = np.stack([C.pred_to_pose(p) for p in pq])
    # |dT| <= 0.25 |dp_omega| (rotation) and 3 |dp_t| (translation)
    np.testing.assert_allclose(T.cpu().numpy().reshape(n, 4, 4), To, atol=3 * 5e-3 * scale)


def test_stride_and_index_views_agree_bitwise(R, scans):
    rng = np.random.default_rng(7)
    theta = _params(rng)
    net = _net(R, theta)
    src, dst, _ = scans
    full_s, full_d = torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()
    coarse_s = full_s[:, ::8, ::8].contiguous()
    coarse_d = full_d[:, ::8, ::8].contiguous()
    p_full = torch.zeros((6, 6), device="cuda")
    p_coarse = torch.zeros_like(p_full)
    R.rimg_propose(net, full_s, full_d, pred=p_full)
    R.rimg_propose(net, coarse_s, coarse_d, pred=p_coarse)
    idx = torch.tensor([5, 0, 3, 3], dtype=torch.int32, device="cuda")
    p_idx = torch.zeros((4, 6), device="cuda")
    R.rimg_propose(net, coarse_s, coarse_d, index=idx, pred=p_idx)
    torch.cuda.synchronize()
    assert torch.equal(p_full, p_coarse)
    assert torch.equal(p_idx, p_coarse[idx.long()])


@pytest.mark.parametrize("n", [6, 64, 200])
def test_gradient_matches_oracle(R, scans, n):
    rng = np.random.default_rng(200 + n)
    theta = _params(rng)
    s, d = _batch(rng, scans, n)
    Tl = _labels(rng, n)
    net = _net(R, theta)
    grad = torch.zeros(net.n_params, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    R.rimg_cnn_grad(net, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(),
                    torch.from_numpy(Tl.reshape(n, 16)).cuda(), grad, loss=loss)
    torch.cuda.synchronize()
    assert net.err.item() == 0
    x = C.net_input(s, d)
    y = np.stack([C.pose_to_target(T) for T in Tl])
    Lq, gq, _ = C.loss_and_grad(theta.astype(np.float64), x, y, q=C.bf16_round)
    L64, g64, _ = C.loss_and_grad(theta.astype(np.float64), x, y)
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - Lq) <= 5e-3 * Lq
    # block by block (each layer's weights and biases)
    o = 0
    for shp in C.param_shapes():
        k = int(np.prod(shp))
        a, b = g[o:o + k], gq[o:o + k]
        assert np.linalg.norm(a - b) <= 5e-3 * np.linalg.norm(b) + 1e-7, (shp, np.linalg.norm(a - b) / np.linalg.norm(b))
        o += k
    assert np.linalg.norm(g - g64) <= 0.10 * np.linalg.norm(g64)


def test_adam_step_and_weight_copies(R, scans):
    rng = np.random.default_rng(9)
    n = 32
    theta = _params(rng)
    s, d = _batch(rng, scans, n)
    Tl = _labels(rng, n)
    net = _net(R, theta)
    S, D = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
    TL = torch.from_numpy(Tl.reshape(n, 16)).cuda()
    lr = 1e-3
    R.rimg_cnn_train_step(net, S, D, TL, step=1, lr=lr)
    after = net.params.clone()
    torch.cuda.synchronize()
    # first Adam step: -lr * g / (|g| + eps) = -lr sign(g) wherever |g| >> eps
    x = C.net_input(s, d)
    y = np.stack([C.pose_to_target(T) for T in Tl])
    _, gq, _ = C.loss_and_grad(theta.astype(np.float64), x, y, q=C.bf16_round)
    delta = after.cpu().numpy().astype(np.float64) - theta
    big = np.abs(gq) > 1e-2 * np.abs(gq).max()
    np.testing.assert_allclose(delta[big], -lr * np.sign(gq[big]), rtol=1e-3, atol=1e-6)
    # the optimizer's BF16 copies equal a fresh load of the updated parameters
    p1 = torch.zeros((n, 6), device="cuda")
    R.rimg_propose(net, S, D, pred=p1)
    net2 = R.ProposalNet(params=after)
    p2 = torch.zeros_like(p1)
    R.rimg_propose(net2, S, D, pred=p2)
    torch.cuda.synchronize()
    assert torch.equal(p1, p2)


def test_training_reduces_the_loss(R, scans):
    rng = np.random.default_rng(10)
    n = 64
    s, d = _batch(rng, scans, n)
    Tl = _labels(rng, n)
    net = R.ProposalNet(seed=1234)
    S, D = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
    TL = torch.from_numpy(Tl.reshape(n, 16)).cuda()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    hist = []
    for step in range(1, 201):
        R.rimg_cnn_train_step(net, S, D, TL, step=step, lr=1e-3, loss=loss)
        if step in (1, 200):
            torch.cuda.synchronize()
            hist.append(loss.item())
    assert net.err.item() == 0
    assert np.isfinite(hist).all() and hist[1] < 0.2 * hist[0], hist


def test_init_is_seeded_and_bounded(R):
    a = R.ProposalNet(seed=5)
    b = R.ProposalNet(seed=5)
    c = R.ProposalNet(seed=6)
    torch.cuda.synchronize()
    assert torch.equal(a.params, b.params) and not torch.equal(a.params, c.params)
    th = a.params.cpu().numpy().astype(np.float64)
    for (W, bias), cin in zip(C.unpack(th)[:-1], [l[0] for l in C.LAYERS]):
        lim = np.sqrt(6.0 / (9 * cin))
        assert np.abs(W).max() <= lim and np.abs(W).max() > 0.9 * lim and np.all(bias == 0)
    Wf, bf = C.unpack(th)[-1]
    assert np.abs(Wf).max() <= 0.1 * np.sqrt(3.0 / 512) and np.all(bf == 0)
