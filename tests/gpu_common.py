"""Helpers shared by the GPU parity tests: build sensors and buffers, run the
library's entry points, and run the oracle on the same inputs."""
import numpy as np

from oracle import rimg_oracle as O

U32 = 2.0 ** -24     # unit roundoff of float32


def f32(x):
    return float(np.float32(x))


def oracle_params(cfg=None, huber=None, gate=0.0, jump=0.1):
    d = cfg.huber_delta if huber is None else huber
    return dict(huber_delta=f32(d), max_corr_dist=f32(gate), normal_rel_jump=f32(jump))


def gpu_sensor(R, sensor, levels):
    return R.rimg_sensor_build(sensor.H, sensor.W, levels, sensor.phi_lut, sensor.theta_lut, sensor.r0)


def planes_for(R, torch, sens, dst, params):
    """GPU plane pyramid (list per level) and finest mask for a batch [n, H, W]."""
    n = dst.shape[0]
    L = sens.levels
    planes = [torch.zeros((n, sens.H >> l, sens.W >> l, 4), dtype=torch.float32, device="cuda") for l in range(L)]
    mask = torch.zeros((n, sens.H, sens.W), dtype=torch.uint8, device="cuda")
    R.rimg_normals(sens, dst, params, planes, mask)
    return planes, mask


def src_pyramid(R, torch, sens, src):
    n = src.shape[0]
    out = [src] + [torch.zeros((n, sens.H >> l, sens.W >> l), dtype=torch.float32, device="cuda")
                   for l in range(1, sens.levels)]
    R.rimg_pyramid(n, sens.H, sens.W, sens.levels, 1, src, out)
    return out


def gpu_register(R, torch, sens, src_np, dst_np, T_init_np, levels, iters, params):
    n = src_np.shape[0]
    src = torch.from_numpy(np.ascontiguousarray(src_np)).cuda()
    dst = torch.from_numpy(np.ascontiguousarray(dst_np)).cuda()
    T0 = torch.from_numpy(np.ascontiguousarray(T_init_np.reshape(n, 16))).cuda()
    T1 = torch.empty_like(T0)
    status = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    ws = torch.empty(R.rimg_register_workspace_bytes(sens, sens, n, levels), dtype=torch.uint8, device="cuda")
    R.rimg_register(sens, sens, n, src, dst, T0, T1, levels, iters, params, status, ws)
    torch.cuda.synchronize()
    return T1.cpu().numpy().reshape(n, 4, 4), status.cpu().numpy()


def oracle_register(pair_src, pair_dst, sensor, T_init, levels, iters, params):
    sens = (sensor.phi_lut, sensor.theta_lut, sensor.r0)
    return O.register(pair_src, pair_dst, sens, sens, T_init, levels, iters, params)
