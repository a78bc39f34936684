"""PCA normals on the GPU (rimg_normals with normal_method = 1) against the
oracle's normals_pca, and registration with them against the oracle's.

Bar.  Each window point carries the unprojection error 16u(r + r0) (u =
2^-24), so the offsets to the centre carry twice that and the scatter matrix
C an error of at most 2 sqrt(9 tr C) * 32u(r + r0); the closed-form FP32
eigen-solver adds ~16u tr C.  An eigenvector moves by the matrix error over
the gap lambda_1 - lambda_0: |dn| <= (192u (r + r0) sqrt(tr C) + 16u tr C) /
(lambda_1 - lambda_0) + 1e-6, and the plane offset by |dn| |P| + 16u |P|.
Validity is bit-exact except where the collinearity test lies within 1 % of
its threshold (near-ties of the eigenvalue ratio)."""
import numpy as np
import pytest

from oracle import rimg_oracle as O
from synth import CONFIGS, make_pair, make_pairs
from tests.gpu_common import gpu_sensor, f32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_02779_b300.rimg as R
    return R


@pytest.mark.parametrize("name,levels", [("pair32x512", 3), ("pair64x1024", 4), ("lut64x512", 3)])
def test_pca_normals_match_oracle(R, name, levels):
    cfg = CONFIGS[name]
    pair = make_pair(cfg, 2)
    s = pair["sensor"]
    sens = gpu_sensor(R, s, levels)
    params = R.rimg_default_params(normal_method=1)
    dst = torch.from_numpy(pair["dst_range"])[None].cuda()
    planes = [torch.zeros((1, s.H >> l, s.W >> l, 4), device="cuda") for l in range(levels)]
    mask = torch.zeros((1, s.H, s.W), dtype=torch.uint8, device="cuda")
    R.rimg_normals(sens, dst, params, planes, mask)
    torch.cuda.synchronize()
    n_o, ok_o, det = O.normals_pca(pair["dst_range"], s.phi_lut, s.theta_lut, s.r0, f32(0.1), return_detail=True)
    pl = planes[0][0].cpu().numpy().astype(np.float64)
    ok_g = mask[0].cpu().numpy().astype(bool)
    near = det["margin"] < 1e-2
    assert np.array_equal(ok_g[~near], ok_o[~near])
    both = ok_g & ok_o
    P, _ = O.unproject(pair["dst_range"].astype(np.float64), s.phi_lut, s.theta_lut, s.r0)
    lam = det["lam"]
    tr = lam.sum(-1)
    r = np.linalg.norm(P, axis=-1)
    bar = (192 * U32 * (r + s.r0) * np.sqrt(np.maximum(tr, 0)) + 16 * U32 * tr) / np.maximum(
        lam[..., 1] - lam[..., 0], 1e-30) + 1e-6
    dn = np.linalg.norm(pl[..., :3] - n_o, axis=-1)
    assert np.all(dn[both] <= bar[both]), np.max(dn[both] / bar[both])
    d_o = np.sum(n_o * P, axis=-1)
    assert np.all(np.abs(pl[..., 3] - d_o)[both] <= (bar * r + 16 * U32 * r)[both])
    assert both.sum() > 0.2 * s.H * s.W
    # the coarse levels are strided copies of the finest plane image
    for l in range(1, levels):
        assert torch.equal(planes[l][0], planes[0][0][::1 << l, ::1 << l])


def test_register_with_pca_normals_matches_oracle(R):
    cfg = CONFIGS["pair32x512"]
    n = 4
    src, dst, _ = make_pairs(cfg, range(n))
    s = cfg.sensor()
    sens = gpu_sensor(R, s, cfg.levels)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta, normal_method=1)
    T0 = torch.eye(4, dtype=torch.float64, device="cuda").reshape(1, 16).repeat(n, 1).contiguous()
    T1 = torch.empty_like(T0)
    ws = torch.empty(R.rimg_register_workspace_bytes(sens, sens, n, cfg.levels), dtype=torch.uint8, device="cuda")
    R.rimg_register(sens, sens, n, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), T0, T1, cfg.levels,
                    cfg.iters, params, None, ws)
    torch.cuda.synchronize()
    Tg = T1.cpu().numpy().reshape(n, 4, 4)
    sens_o = (s.phi_lut, s.theta_lut, s.r0)
    for i in range(n):
        To, _ = O.register(src[i], dst[i], sens_o, sens_o, np.eye(4), cfg.levels, cfg.iters,
                           dict(huber_delta=f32(cfg.huber_delta), normal_rel_jump=f32(0.1), normal_method="pca"))
        eR, et = O.pose_error(Tg[i], To)
        assert eR <= 1e-4 and et <= 1e-4, (i, eR, et)
