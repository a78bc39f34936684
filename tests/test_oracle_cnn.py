"""Pins of the FP64 proposal-network oracle against independent definitions:
the convolution against scipy's 2D correlation on explicitly padded images,
im2col / col2im against each other (adjointness), the backward pass against
central finite differences, BF16 rounding against torch's conversion and
hand-worked ties, the rotation maps against scipy's rotation-vector routines."""
import numpy as np
import pytest
from scipy.signal import correlate2d
from scipy.spatial.transform import Rotation

from oracle import cnn_oracle as C


def _conv_reference(x, W, b):
    """One layer: wrap the columns, zero-pad the rows, correlate each output
    channel with its 3 x 3 x C_in kernel, keep every second row and column."""
    n, H, Wd, cin = x.shape
    cout = W.shape[0]
    K = W.reshape(cout, 3, 3, cin)
    xp = np.concatenate([x[:, :, -1:], x, x[:, :, :1]], axis=2)
    xp = np.pad(xp, ((0, 0), (1, 1), (0, 0), (0, 0)))
    ho, wo = (H - 1) // 2 + 1, Wd // 2
    out = np.zeros((n, ho, wo, cout))
    for i in range(n):
        for o in range(cout):
            acc = sum(correlate2d(xp[i, :, :, c], K[o, :, :, c], mode="valid") for c in range(cin))
            out[i, :, :, o] = acc[::2, ::2][:ho, :wo] + b[o]
    return np.maximum(out, 0.0)


@pytest.mark.parametrize("li", [0, 1, 3])
def test_conv_layer_matches_scipy_correlation(li):
    rng = np.random.default_rng(li)
    H, Wd, cin, ho, wo, cout = C.geometry()[li]
    cout = min(cout, 8)
    x = rng.normal(size=(2, H, Wd, cin))
    W = rng.normal(size=(cout, 9 * cin))
    b = rng.normal(size=cout)
    got = np.maximum(C.im2col(x, ho, wo) @ W.T + b, 0.0).reshape(2, ho, wo, cout)
    np.testing.assert_allclose(got, _conv_reference(x, W, b), rtol=1e-12, atol=1e-12)


def test_col2im_is_the_adjoint_of_im2col():
    rng = np.random.default_rng(3)
    for H, Wd, cin, ho, wo, _ in C.geometry():
        x = rng.normal(size=(2, H, Wd, cin))
        D = rng.normal(size=(2 * ho * wo, 9 * cin))
        lhs = np.sum(C.im2col(x, ho, wo) * D)
        rhs = np.sum(x * C.col2im(D, x.shape, ho, wo))
        assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + 1.0)


def _params(rng, scale=1.0):
    out = []
    for (cin, cout) in C.LAYERS:
        out.append((rng.normal(size=(cout, 9 * cin)) * scale * np.sqrt(2.0 / (9 * cin)), rng.normal(size=cout) * 0.1))
    out.append((rng.normal(size=(6, 512)) * np.sqrt(1.0 / 512), rng.normal(size=6) * 0.1))
    return C.pack(out)


def _inputs(rng, n):
    src = rng.uniform(1.0, 60.0, size=(n, 8, 128))
    dst = rng.uniform(1.0, 60.0, size=(n, 8, 128))
    src[rng.random(src.shape) < 0.1] = 0.0
    dst[rng.random(dst.shape) < 0.1] = np.nan
    return C.net_input(src, dst)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(11)
    theta = _params(rng)
    x = _inputs(rng, 3)
    y = rng.normal(size=(3, 6))
    L, g, _ = C.loss_and_grad(theta, x, y)
    # probe parameters in every block: each layer's weights and biases
    offs, o = [], 0
    for s in C.param_shapes():
        k = int(np.prod(s))
        offs.append((o, k))
        o += k
    idx = [off + int(j) for off, k in offs for j in rng.choice(k, size=min(k, 6), replace=False)]
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (C.loss_and_grad(tp, x, y)[0] - C.loss_and_grad(tm, x, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])


def test_forward_prediction_is_linear_in_the_last_layer():
    rng = np.random.default_rng(5)
    theta = _params(rng)
    x = _inputs(rng, 2)
    p, (layers, cache) = C.forward(theta, x)
    flat = cache[-1][0]
    Wf, bf = layers[-1]
    np.testing.assert_allclose(p, flat @ Wf.T + bf)
    # the flattened activation is (w, c) ordered: [n, 1, 4, 128] -> [n, 512]
    a5 = cache[-2][2].reshape(2, 1, 4, 128)
    np.testing.assert_allclose(flat, a5.reshape(2, 512))


def test_bf16_rounding():
    # ties go to the even mantissa; spacing at 1 is 2^-7
    vals = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 3.0e38, 0.0, -0.0, 1e-40])
    got = C.bf16_round(vals)
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == 1 + 2.0 ** -6 and got[3] == -1.0
    assert got[5] == 0.0 and np.signbit(got[6])
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-8, 8, 5000), vals])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(C.bf16_round(x), ref)


def test_rotation_maps_against_scipy():
    rng = np.random.default_rng(2)
    for a in [0.0, 1e-9, 1e-4, 0.3, 1.0, 2.5, np.pi - 1e-3, np.pi - 1e-7]:
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        w = a * axis
        R = C.so3_exp(w)
        np.testing.assert_allclose(R, Rotation.from_rotvec(w).as_matrix(), atol=1e-12)
        np.testing.assert_allclose(C.so3_log(R), Rotation.from_matrix(R).as_rotvec(), atol=2e-7 if a > 3 else 1e-11)
    T = np.eye(4)
    T[:3, :3] = Rotation.from_rotvec([0.1, -0.2, 0.05]).as_matrix()
    T[:3, 3] = [1.5, -0.3, 0.6]
    y = C.pose_to_target(T)
    np.testing.assert_allclose(y, [0.4, -0.8, 0.2, 0.5, -0.1, 0.2], atol=1e-12)
    np.testing.assert_allclose(C.pred_to_pose(y), T, atol=1e-12)


def test_bf16_network_stays_close_to_fp64():
    rng = np.random.default_rng(8)
    theta = _params(rng)
    x = _inputs(rng, 4)
    y = rng.normal(size=(4, 6))
    L64, g64, p64 = C.loss_and_grad(theta, x, y)
    Lb, gb, pb = C.loss_and_grad(theta, x, y, q=C.bf16_round)
    # BF16 keeps 8 significant bits; six layers of it forward and back (and the
    # ReLU masks that flip where a pre-activation rounds across zero) leave a
    # few per cent of the FP64 gradient
    assert np.linalg.norm(pb - p64) <= 0.05 * np.linalg.norm(p64)
    assert np.linalg.norm(gb - g64) <= 0.10 * np.linalg.norm(g64)
    assert not np.array_equal(gb, g64)
