"""FP64 CPU reference of the learned pose-proposal network.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
benchmark's CPU-baseline leg may import this module; the library never does,
and it shares no code, tables or helpers with the CUDA path.

The paper registers scans by Gauss-Newton only and names learned features on
the cylindrical image as future work (Section 7).  The proposal network is an
extension that supplies the initial pose T0 of the multi-scale registration
(Section 4.1, the coarse-to-fine schedule of Section 6.1).  Its definition:

* Input: the coarsest pyramid level (every 8th row and column, Section 4.1)
  of the source and target range images, H x W = 8 x 128, as two channels
  (channel 0 source, channel 1 target), channels-last.  A valid range r
  (finite, > 0, the validity rule of the registration) becomes r / 32; an
  invalid one becomes 0.
* Five 3 x 3 convolutions with stride 2, each followed by ReLU, channels
  2 -> 32 -> 64 -> 64 -> 128 -> 128.  Rows are zero-padded by one; columns
  wrap around (the image covers 360 degrees of azimuth, so column -1 is
  column W-1).  Output size: H_out = floor((H_in - 1) / 2) + 1,
  W_out = W_in / 2; spatial sizes 8x128 -> 4x64 -> 2x32 -> 1x16 -> 1x8 -> 1x4.
* A linear layer 512 -> 6 on the flattened (w, c) activations gives
  p = (omega / 0.25 rad, t / 3 m): T0 = [Exp(omega), t].
* Weight layout (the flat parameter vector): per convolution W [C_out][9 C_in]
  with column index (kh * 3 + kw) * C_in + c, then b [C_out]; then the linear
  layer's W [6][512] (input index w * 128 + c) and b [6].
* Training target: y = (Log(R) / 0.25, t / 3) of a label pose [R, t];
  loss L = 1 / (2 n) * sum_i |p_i - y_i|^2.

Mixed precision.  The CUDA path rounds to BF16 (round to nearest even) at
fixed points: the network input, the weights, every activation passed to the
next layer, and the two gradient operands of the backward contractions
(dL/dp and dL/dZ after the ReLU mask); it accumulates in FP32.  With
``q=bf16_round`` this module rounds at the same points and computes everything
else in FP64; with ``q=None`` it is the plain FP64 network.
"""
import numpy as np

H0, W0, C0 = 8, 128, 2
LAYERS = ((2, 32), (32, 64), (64, 64), (64, 128), (128, 128))
FC_IN, FC_OUT = 512, 6
RANGE_SCALE = 1.0 / 32.0
OMEGA_SCALE = 0.25
T_SCALE = 3.0


def bf16_round(x):
    """Round float64 values to the nearest BF16 value (ties to even), computed
    from the IEEE float32 bit pattern: float32 rounding first, then the low 16
    bits rounded away.  Returns float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    out = b.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def _ident(x):
    return np.asarray(x, dtype=np.float64)


def geometry():
    """Per convolution: (H_in, W_in, C_in, H_out, W_out, C_out)."""
    g = []
    h, w = H0, W0
    for cin, cout in LAYERS:
        ho, wo = (h - 1) // 2 + 1, w // 2
        g.append((h, w, cin, ho, wo, cout))
        h, w = ho, wo
    assert h * w * LAYERS[-1][1] == FC_IN
    return g


def param_shapes():
    shapes = []
    for cin, cout in LAYERS:
        shapes += [(cout, 9 * cin), (cout,)]
    shapes += [(FC_OUT, FC_IN), (FC_OUT,)]
    return shapes


def param_count():
    return int(sum(np.prod(s) for s in param_shapes()))


def unpack(theta):
    """Flat parameter vector -> list of (W, b), conv layers then the linear layer."""
    theta = np.asarray(theta, dtype=np.float64)
    out, o = [], 0
    shapes = param_shapes()
    for i in range(0, len(shapes), 2):
        ws, bs = shapes[i], shapes[i + 1]
        nw, nb = int(np.prod(ws)), int(np.prod(bs))
        out.append((theta[o:o + nw].reshape(ws), theta[o + nw:o + nw + nb]))
        o += nw + nb
    assert o == theta.size
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def net_input(src_coarse, dst_coarse):
    """[n, 8, 128] source and target coarsest-level ranges -> [n, 8, 128, 2]."""
    x = np.stack([np.asarray(src_coarse, np.float64), np.asarray(dst_coarse, np.float64)], axis=-1)
    ok = np.isfinite(x) & (x > 0)
    return np.where(ok, np.where(ok, x, 0.0) * RANGE_SCALE, 0.0)


def im2col(x, ho, wo):
    """x [n, H, W, C] -> columns [n * ho * wo, 9 C]: row (n, i, j) holds the
    3 x 3 window centred at input (2 i, 2 j), rows zero-padded, columns
    wrapped, in (kh, kw, c) order."""
    n, H, W, C = x.shape
    cols = np.zeros((n, ho, wo, 3, 3, C))
    for kh in range(3):
        for kw in range(3):
            for i in range(ho):
                hi = 2 * i - 1 + kh
                if hi < 0 or hi >= H:
                    continue
                wi = (2 * np.arange(wo) - 1 + kw) % W
                cols[:, i, :, kh, kw, :] = x[:, hi, wi, :]
    return cols.reshape(n * ho * wo, 9 * C)


def col2im(dcols, shape, ho, wo):
    """Adjoint of im2col: scatter-add column gradients back onto [n, H, W, C]."""
    n, H, W, C = shape
    d = dcols.reshape(n, ho, wo, 3, 3, C)
    dx = np.zeros(shape)
    for kh in range(3):
        for kw in range(3):
            for i in range(ho):
                hi = 2 * i - 1 + kh
                if hi < 0 or hi >= H:
                    continue
                wi = (2 * np.arange(wo) - 1 + kw) % W
                np.add.at(dx, (slice(None), hi, wi, slice(None)), d[:, i, :, kh, kw, :])
    return dx


def forward(theta, x, q=None):
    """Returns (p [n, 6], cache).  x: net_input() output."""
    q = q or _ident
    layers = [(q(W), b) for W, b in unpack(theta)]
    a = q(x)
    n = a.shape[0]
    cache = []
    for (W, b), (H, Wd, cin, ho, wo, cout) in zip(layers[:-1], geometry()):
        cols = im2col(a, ho, wo)
        y = np.maximum(cols @ W.T + b, 0.0)
        cache.append((a.shape, cols, y))
        a = q(y).reshape(n, ho, wo, cout)
    Wf, bf = layers[-1]
    flat = a.reshape(n, FC_IN)
    p = flat @ Wf.T + bf
    cache.append((flat,))
    return p, (layers, cache)


def loss_and_grad(theta, x, y, q=None):
    """Loss 1/(2n) sum |p - y|^2 and its gradient w.r.t. the flat parameters
    (backpropagation through the definitions above; the BF16 rounding points,
    if any, are treated as identities in the chain rule)."""
    qq = q or _ident
    p, (layers, cache) = forward(theta, x, q)
    n = p.shape[0]
    r = p - y
    loss = 0.5 * np.sum(r * r) / n
    dp = qq(r / n)
    (flat,) = cache[-1]
    Wf, _ = layers[-1]
    grads = [(dp.T @ flat, dp.sum(0))]
    da = dp @ Wf                                       # d loss / d flattened input of the linear layer
    geo = geometry()
    for li in range(len(LAYERS) - 1, -1, -1):
        shape, cols, yv = cache[li]
        H, Wd, cin, ho, wo, cout = geo[li]
        dz = qq(da.reshape(-1, cout) * (yv > 0))
        W, _ = layers[li]
        grads.append((dz.T @ cols, dz.sum(0)))
        if li > 0:
            da = col2im(dz @ W, shape, ho, wo)
    grads = grads[::-1]                                # conv layers first, then the linear layer
    return loss, pack(grads), p


# ----------------------------------------------------------------------------
# Rotation parametrisation of the output and the targets

def hat(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def so3_exp(w):
    """Rodrigues' formula, R = I + sin(a)/a K + (1 - cos(a))/a^2 K^2, K = hat(w)."""
    w = np.asarray(w, dtype=np.float64)
    a = np.linalg.norm(w)
    K = hat(w)
    if a < 1e-8:
        return np.eye(3) + K + 0.5 * K @ K
    return np.eye(3) + np.sin(a) / a * K + (1.0 - np.cos(a)) / (a * a) * K @ K


def so3_log(R):
    """Rotation vector of R (angle in [0, pi]): the inverse of so3_exp."""
    R = np.asarray(R, dtype=np.float64)
    v = 0.5 * np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    c = 0.5 * (np.trace(R) - 1.0)
    s = np.linalg.norm(v)
    a = np.arctan2(s, c)
    if c > -0.9:
        return v * (a / s if s > 1e-12 else 1.0 + a * a / 6.0)
    # near pi: axis from the symmetric part, R + R^T = 2 (cos a I + (1 - cos a) k k^T)
    S = 0.5 * (R + R.T) - c * np.eye(3)
    j = int(np.argmax(np.diag(S)))
    k = S[:, j] / np.sqrt(S[j, j])
    if np.dot(k, v) < 0:
        k = -k
    return a * k / np.linalg.norm(k)


def pose_to_target(T):
    """Label pose (4 x 4) -> the regression target y (6,)."""
    T = np.asarray(T, dtype=np.float64)
    return np.concatenate([so3_log(T[:3, :3]) / OMEGA_SCALE, T[:3, 3] / T_SCALE])


def pred_to_pose(p):
    """Network output (6,) -> T0 = [Exp(0.25 p[0:3]), 3 p[3:6]]."""
    T = np.eye(4)
    T[:3, :3] = so3_exp(OMEGA_SCALE * np.asarray(p[:3], dtype=np.float64))
    T[:3, 3] = T_SCALE * np.asarray(p[3:], dtype=np.float64)
    return T
