"""rimg_icp_step_static: the workspace-free step for callers that cannot
allocate device memory (allocation-free real-time loops, plug-ins limited to
the buffers they are given).  It must give the same results as rimg_icp_step
with a caller workspace, call after call, although its scratch array is
shared and keeps the previous call's contents.

This file is named to be collected last, so a run that stops at the first
failure has run every other test before it."""
import ctypes

import numpy as np
import pytest

from synth import CONFIGS, make_pairs
from tests.gpu_common import gpu_sensor, planes_for, src_pyramid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_02779_b300.rimg as R
    return R


def _raw_static(R, src, dst, level, n, s_l, planes_l, pose, params, update, out29, assoc, status):
    """Call the entry point through the C ABI directly (ctypes, raw pointers)."""
    lib = R.lib()
    return lib.rimg_icp_step_static(src.ref(), dst.ref(), level, n, s_l.data_ptr(), planes_l.data_ptr(), None,
                                    pose.data_ptr(), ctypes.byref(params), update, out29.data_ptr(),
                                    assoc.data_ptr(), status.data_ptr(), torch.cuda.current_stream().cuda_stream)


def test_static_scratch_step_matches_workspace_step_twice(R):
    cfg = CONFIGS["pair64x1024"]
    s = cfg.sensor()
    sens = gpu_sensor(R, s, cfg.levels)
    params = R.rimg_default_params(huber_delta=cfg.huber_delta)
    n = 3
    src_np, dst_np, _ = make_pairs(cfg, range(n))
    src = torch.from_numpy(src_np).cuda()
    dst = torch.from_numpy(dst_np).cuda()
    planes, _ = planes_for(R, torch, sens, dst, params)
    spyr = src_pyramid(R, torch, sens, src)
    T0 = torch.eye(4, dtype=torch.float64, device="cuda").reshape(1, 16).repeat(n, 1).contiguous()
    ws = torch.empty(R.rimg_icp_workspace_bytes(sens, n), dtype=torch.uint8, device="cuda")

    pose_ref, pose_st = T0.clone(), T0.clone()
    for call in range(2):               # two calls in a row, each updating the pose
        level = 1 if call == 0 else 0
        H, W = s.H >> level, s.W >> level
        out_ref = torch.zeros((n, 29), dtype=torch.float64, device="cuda")
        out_st = torch.full((n, 29), np.nan, dtype=torch.float64, device="cuda")
        a_ref = torch.zeros((n, H, W), dtype=torch.int32, device="cuda")
        a_st = torch.full((n, H, W), -9, dtype=torch.int32, device="cuda")
        st_ref = torch.zeros(n, dtype=torch.int32, device="cuda")
        st_st = torch.zeros(n, dtype=torch.int32, device="cuda")
        R.rimg_icp_step(sens, sens, level, n, spyr[level], planes[level], None, pose_ref, params, 1, out_ref,
                        a_ref, st_ref, ws)
        rc = _raw_static(R, sens, sens, level, n, spyr[level], planes[level], pose_st, params, 1, out_st, a_st,
                         st_st)
        assert rc == 0
        torch.cuda.synchronize()
        assert torch.equal(a_st, a_ref)
        assert torch.equal(st_st, st_ref)
        # the same kernel and block decomposition: results agree to the
        # reduced-sum tolerance of the parity tests (in practice bit for bit)
        o_ref, o_st = out_ref.cpu().numpy(), out_st.cpu().numpy()
        assert np.all(np.abs(o_st - o_ref) <= 1e-6 * np.abs(o_ref) + 1e-9)
        assert np.allclose(pose_st.cpu().numpy(), pose_ref.cpu().numpy(), rtol=0, atol=1e-9)


def test_static_scratch_rejects_oversized_batch(R):
    cfg = CONFIGS["pair64x1024"]
    s = cfg.sensor()
    sens = gpu_sensor(R, s, cfg.levels)
    params = R.rimg_default_params()
    n = 4096                                 # far beyond the fixed scratch
    need = R.rimg_icp_workspace_bytes(sens, n)
    assert need > R.RIMG_STATIC_SCRATCH_BYTES
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    T = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RimgError) as ei:
        R.rimg_icp_step_static(sens, sens, 0, n, x, x, None, T, params, 0)
    assert ei.value.code == -4
