"""rimg_gn_update (the FP64 Gauss-Newton update of Section 4.1 on its own)
against the oracle's gn_update on crafted normal equations: well and badly
conditioned systems, the count and pivot tests, both branches of the Exp
coefficients (Taylor series below 0.5 rad, sincos above), and batches whose
size leaves the last four-warp block partly empty.

Bar.  Both sides solve in FP64; the library's scaled LDL^T elimination and
the oracle's textbook Cholesky differ only in rounding order, so the steps
agree to a small multiple of cond(H) u |xi| (u = 2^-53) and the poses to that
plus a few ulps of the composition.  The step record carries FP32 roots
(relative 1e-6)."""
import numpy as np
import pytest

from oracle import rimg_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_02779_b300.rimg as R
    return R


def _pack(H, g, count, e2=0.0):
    """The record layout of out29: 21 upper-triangle entries of H row-major,
    g, sum w e^2, count; slots 29..31 are outputs."""
    t = np.zeros(32)
    q = 0
    for i in range(6):
        for j in range(i, 6):
            t[q] = H[i, j]
            q += 1
    t[21:27] = g
    t[27] = e2
    t[28] = count
    return t


def _pose(rng):
    T = np.eye(4)
    T[:3, :3] = O.se3_exp(np.r_[rng.normal(size=3), 0, 0, 0])[:3, :3]
    T[:3, 3] = rng.normal(size=3) * 5
    return T


def _cases(rng):
    """(H, g, count, label) systems; g = -H xi for a chosen step xi where the
    system is regular."""
    out = []
    D = np.diag([3e2, 3e2, 3e2, 3e1, 3e1, 3e1])          # rotation rows ~ range x translation rows
    for k in range(12):                                   # regular, realistic scaling
        M = rng.normal(size=(6, 6))
        H = D @ (M @ M.T + 0.5 * np.eye(6)) @ D
        xi = rng.normal(size=6) * np.r_[[0.01] * 3, [0.05] * 3]
        out.append((H, -H @ xi, 1000, "regular"))
    for cond_scale in (1e-2, 1e-3):                      # badly conditioned
        M = rng.normal(size=(6, 6))
        Dk = np.diag([1.0, 1.0, cond_scale, 1.0, 1.0, cond_scale])
        H = Dk @ (M @ M.T + 1e-3 * np.eye(6)) @ Dk
        xi = rng.normal(size=6) * 0.01
        out.append((H, -H @ xi, 1000, "ill"))
    for th in (0.2, 0.499, 0.501, 0.9, 1.7, 3.0):         # both Exp branches
        w = rng.normal(size=3)
        w *= th / np.linalg.norm(w)
        xi = np.r_[w, rng.normal(size=3)]
        H = 40.0 * np.eye(6) + 0.5 * np.ones((6, 6))
        out.append((H, -H @ xi, 50, f"rot{th}"))
    M = rng.normal(size=(6, 6))
    H = M @ M.T + np.eye(6)
    out.append((H, rng.normal(size=6), 5, "count5"))      # fewer than 6 correspondences
    Hz = H.copy()
    Hz[0, :] = 0.0
    Hz[:, 0] = 0.0
    out.append((Hz, rng.normal(size=6), 100, "zero_row"))
    M5 = rng.normal(size=(6, 5))
    out.append((M5 @ M5.T, rng.normal(size=6), 100, "rank5"))
    out.append((np.zeros((6, 6)), np.zeros(6), 100, "zero"))
    return out


@pytest.mark.parametrize("n", [1, 23, 37])
def test_gn_update_matches_oracle(R, n):
    rng = np.random.default_rng(11)
    base = _cases(rng)                                   # 24 systems
    cases = (base * 2)[:n] if n > 1 else base[-8:-7]     # 23, 37: the last four-pair block partly empty
    n = len(cases)
    T0 = np.stack([_pose(rng) for _ in range(n)])
    sums = torch.from_numpy(np.stack([_pack(H, g, c) for H, g, c, _ in cases])).cuda()
    pose = torch.from_numpy(T0.reshape(n, 16).copy()).cuda()
    status = torch.zeros(n, dtype=torch.int32, device="cuda")
    R.rimg_gn_update(n, sums, pose, status)
    torch.cuda.synchronize()
    Tg = pose.cpu().numpy().reshape(n, 4, 4)
    rec = sums.cpu().numpy()
    st = status.cpu().numpy()
    for i, (H, g, count, label) in enumerate(cases):
        To, ok = O.gn_update(T0[i], {"H": H, "g": g, "count": count})
        assert bool(rec[i, 31]) == ok, (i, label)
        assert bool(st[i] & 1) == (not ok), (i, label)
        if not ok:
            assert np.array_equal(Tg[i], T0[i]), (i, label)
            assert np.all(rec[i, 29:32] == 0.0), (i, label)
            continue
        xi, _ = O.cholesky_solve(H, g)
        cond = np.linalg.cond(H)
        tol = 64 * cond * U64 * np.linalg.norm(xi) * (1 + np.abs(T0[i]).max()) + 1e-12 * (1 + np.abs(T0[i]).max())
        assert np.abs(Tg[i] - To).max() <= tol, (i, label, np.abs(Tg[i] - To).max(), tol)
        np.testing.assert_allclose(rec[i, 29:31], [np.linalg.norm(xi[:3]), np.linalg.norm(xi[3:])], rtol=1e-6,
                                   atol=1e-30)
        # the updated rotation stays orthonormal to FP64 rounding
        Rm = Tg[i, :3, :3]
        assert np.abs(Rm @ Rm.T - np.eye(3)).max() < 1e-13, (i, label)


def test_gn_update_matches_the_update_inside_icp_step(R):
    """rimg_icp_step with update = 1 and rimg_icp_step (update = 0, out29) then
    rimg_gn_update give bit-identical poses: one solver."""
    from synth import CONFIGS, make_pair
    from tests.gpu_common import gpu_sensor
    cfg = CONFIGS["pair32x512"]
    pair = make_pair(cfg, 4)
    s = pair["sensor"]
    sens = gpu_sensor(R, s, 1)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    src = torch.from_numpy(pair["src_range"])[None].cuda()
    dst = torch.from_numpy(pair["dst_range"])[None].cuda()
    planes = [torch.zeros((1, s.H, s.W, 4), device="cuda")]
    R.rimg_normals(sens, dst, params, planes)
    T0 = torch.from_numpy(O.se3_exp(np.array([3e-3, -2e-3, 1e-3, 0.05, 0.02, -0.03])).reshape(1, 16)).cuda()
    ws = torch.empty(R.rimg_icp_workspace_bytes(sens, 1), dtype=torch.uint8, device="cuda")
    pa = T0.clone()
    R.rimg_icp_step(sens, sens, 0, 1, src, planes[0], None, pa, params, 1, workspace=ws)
    pb = T0.clone()
    out29 = torch.zeros((1, 29), dtype=torch.float64, device="cuda")
    R.rimg_icp_step(sens, sens, 0, 1, src, planes[0], None, pb, params, 0, out29=out29, workspace=ws)
    sums = torch.zeros((1, 32), dtype=torch.float64, device="cuda")
    sums[:, :29] = out29
    R.rimg_gn_update(1, sums, pb)
    torch.cuda.synchronize()
    assert torch.equal(pa, pb)
    assert not torch.equal(pa, T0)
