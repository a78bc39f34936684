"""Python binding of librimg (include/rimg.h): argument marshalling only.

Every function here has the name of the C entry point it calls and forwards
device pointers taken from torch tensors; all computation happens in the CUDA
library.  The library must be built (``python -m paper_2112_02779_b300.build``
or ``__graft_entry__.build()``); importing this package fails loudly if it is
missing.  torch is used only for device memory and streams.
"""
import ctypes
import os

import numpy as np

from ._abi import (RIMG_MAX_LEVELS, RIMG_FLAG_DEGENERATE, RIMG_STATIC_SCRATCH_BYTES, rimg_level, rimg_sensor, rimg_params,
                   rimg_group, rimg_adam, rimg_grid, RIMG_CNN_IN_H, RIMG_CNN_IN_W, RIMG_CNN_MAX_BATCH,
                   STATUS_NAMES, HEADER_FUNCTIONS)

_HERE = os.path.dirname(os.path.abspath(__file__))
# RIMG_LIBRARY: path of an alternative build of librimg.so (same ABI)
LIB_PATH = os.environ.get("RIMG_LIBRARY") or os.path.join(_HERE, "_lib", "librimg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"librimg.so not built ({LIB_PATH}); run `python -m paper_2112_02779_b300.build`")

_lib = ctypes.CDLL(LIB_PATH)

_c_int, _c_size, _vp = ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p
_P = ctypes.POINTER


def _sig(name, restype, *argtypes):
    f = getattr(_lib, name)
    f.restype = restype
    f.argtypes = list(argtypes)
    return f


_sig("rimg_default_params", _c_int, _P(rimg_params))
_sig("rimg_status_string", ctypes.c_char_p, _c_int)
_sig("rimg_last_error", ctypes.c_char_p)
_sig("rimg_sensor_table_bytes", _c_int, _c_int, _c_int, _c_int, _P(_c_size))
_sig("rimg_sensor_build", _c_int, _c_int, _c_int, _c_int, _P(ctypes.c_double), _P(ctypes.c_double),
     ctypes.c_double, _vp, _c_size, _P(rimg_sensor))
_sig("rimg_unproject", _c_int, _P(rimg_sensor), _c_int, _c_int, _vp, _vp, _vp, _vp)
_sig("rimg_pyramid", _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, _vp, _P(_vp), _vp)
_sig("rimg_normals", _c_int, _P(rimg_sensor), _c_int, _vp, _P(rimg_params), _P(_vp), _vp, _vp)
_sig("rimg_icp_workspace_bytes", _c_int, _P(rimg_sensor), _c_int, _P(_c_size))
_sig("rimg_icp_step", _c_int, _P(rimg_sensor), _P(rimg_sensor), _c_int, _c_int, _vp, _vp, _vp, _vp,
     _P(rimg_params), _c_int, _vp, _vp, _vp, _vp, _c_size, _vp)
_sig("rimg_icp_step_static", _c_int, _P(rimg_sensor), _P(rimg_sensor), _c_int, _c_int, _vp, _vp, _vp, _vp,
     _P(rimg_params), _c_int, _vp, _vp, _vp, _vp)
_sig("rimg_gn_update", _c_int, _c_int, _vp, _vp, _vp, _vp)
_sig("rimg_register_workspace_bytes", _c_int, _P(rimg_sensor), _P(rimg_sensor), _c_int, _c_int, _P(_c_size))
_sig("rimg_register", _c_int, _P(rimg_sensor), _P(rimg_sensor), _c_int, _vp, _vp, _vp, _vp, _c_int,
     _P(_c_int), _P(rimg_params), _vp, _vp, _c_size, _vp)
_sig("rimg_register_last_sums", _c_int, _P(rimg_sensor), _P(rimg_sensor), _c_int, _c_int, _vp, _c_size, _vp, _vp)
_sig("rimg_register_host_workspace_bytes", _c_int, _P(rimg_sensor), _P(rimg_sensor), _c_int, _c_int,
     _c_int, _P(_c_size))
_sig("rimg_register_host", _c_int, _P(rimg_sensor), _P(rimg_sensor), _c_int, _vp, _vp, _vp, _vp, _c_int,
     _P(_c_int), _P(rimg_params), _vp, _c_int, _vp, _c_size, _vp)
_sig("rimg_register_host_async", _c_int, _P(rimg_sensor), _P(rimg_sensor), _c_int, _vp, _vp, _vp, _vp, _c_int,
     _P(_c_int), _P(rimg_params), _vp, _c_int, _vp, _c_size, _vp)
_sig("rimg_register_groups_workspace_bytes", _c_int, _c_int, _P(rimg_group), _P(_c_size))
_sig("rimg_register_groups", _c_int, _c_int, _P(rimg_group), _vp, _c_size, _vp)
_sig("rimg_autotune", _c_int, _c_int, _P(rimg_group), _vp, _c_size, _vp)
_sig("rimg_autotune_clear", _c_int)
_sig("rimg_autotune_register", _c_int, _P(rimg_sensor), _P(rimg_sensor), _c_int, _vp, _vp, _vp, _vp, _c_int,
     _P(_c_int), _P(rimg_params), _vp, _c_size, _vp)
_sig("rimg_autotune_set", _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int)
_sig("rimg_gemm_bf16", _c_int, _c_int, _c_int, _c_int, _vp, _c_int, _vp, _c_int, _vp, _c_int, _vp, _vp, _c_int,
     _c_int, _vp, _vp)
_sig("rimg_cnn_param_count", _c_int, _P(_c_size))
_sig("rimg_cnn_state_bytes", _c_int, _P(_c_size))
_sig("rimg_cnn_workspace_bytes", _c_int, _c_int, _P(_c_size))
_sig("rimg_cnn_init", _c_int, _vp, _c_size, ctypes.c_uint64, _vp)
_sig("rimg_cnn_load", _c_int, _vp, _c_size, _vp, _vp)
_sig("rimg_propose", _c_int, _vp, _c_int, _c_int, _c_int, _c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _c_size, _vp)
_sig("rimg_cnn_grad", _c_int, _vp, _c_int, _c_int, _c_int, _c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
     _c_size, _vp)
_sig("rimg_cnn_train_step", _c_int, _vp, _c_size, _c_int, _c_int, _c_int, _c_int, _vp, _vp, _vp, _vp,
     _P(rimg_adam), _c_int, _vp, _vp, _vp, _c_size, _vp)
_sig("rimg_sdf_integrate", _c_int, _P(rimg_sensor), _c_int, _c_int, _vp, _vp, _P(rimg_grid), ctypes.c_float, _vp, _vp,
     _P(rimg_params), _vp)
_sig("rimg_center_init", _c_int, _P(rimg_sensor), _P(rimg_sensor), _c_int, _c_int, _vp, _vp, _vp, _vp, _vp)
_sig("rimg_points_to_range", _c_int, _P(rimg_sensor), _c_int, _c_int, _c_int, _vp, _vp, _vp, _vp, _P(rimg_params), _vp)
_sig("rimg_profile_begin", _c_int, _c_int)
_sig("rimg_profile_end", _c_int, _c_int, _P(_c_int), _P(_c_int), _P(_c_int), _P(ctypes.c_float), _P(ctypes.c_float))


class RimgError(RuntimeError):
    def __init__(self, fn, code):
        msg = _lib.rimg_status_string(code).decode()
        extra = _lib.rimg_last_error().decode() if code == -5 else ""
        super().__init__(f"{fn} failed: {code} ({msg}){': ' + extra if extra else ''}")
        self.code = code


def _check(fn, code):
    if code != 0:
        raise RimgError(fn, code)


def lib():
    """The loaded ctypes library (for tests that call entry points raw)."""
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr_array(tensors, n):
    arr = (_vp * n)()
    for i, t in enumerate(tensors):
        arr[i] = _ptr(t) if t is not None else None
    return arr


# ---------------------------------------------------------------------------

def rimg_default_params(**overrides):
    p = rimg_params()
    _check("rimg_default_params", _lib.rimg_default_params(ctypes.byref(p)))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def rimg_status_string(code):
    return _lib.rimg_status_string(code).decode()


def rimg_sensor_table_bytes(H, W, levels):
    b = _c_size(0)
    _check("rimg_sensor_table_bytes", _lib.rimg_sensor_table_bytes(H, W, levels, ctypes.byref(b)))
    return b.value


class Sensor:
    """A built sensor: the rimg_sensor struct plus the torch tensor holding its
    device tables (kept alive with the struct)."""

    def __init__(self, struct, tables):
        self.struct = struct
        self.tables = tables

    @property
    def H(self):
        return self.struct.H

    @property
    def W(self):
        return self.struct.W

    @property
    def levels(self):
        return self.struct.levels

    def ref(self):
        return ctypes.byref(self.struct)


def rimg_sensor_build(H, W, levels, phi_lut, theta_lut, r0, device="cuda"):
    import torch
    nbytes = rimg_sensor_table_bytes(H, W, levels)
    tables = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
    phi = np.ascontiguousarray(phi_lut, dtype=np.float64)
    th = np.ascontiguousarray(theta_lut, dtype=np.float64)
    s = rimg_sensor()
    _check("rimg_sensor_build", _lib.rimg_sensor_build(
        H, W, levels, phi.ctypes.data_as(_P(ctypes.c_double)), th.ctypes.data_as(_P(ctypes.c_double)),
        float(r0), tables.data_ptr(), tables.numel(), ctypes.byref(s)))
    return Sensor(s, tables)


def rimg_unproject(sensor, level, range_l, xyz, mask=None, stream=None):
    n = range_l.shape[0] if range_l.dim() == 3 else 1
    _check("rimg_unproject", _lib.rimg_unproject(sensor.ref(), level, n, _ptr(range_l), _ptr(xyz), _ptr(mask),
                                                 _stream(stream)))


def rimg_pyramid(n_images, H, W, levels, channels, inp, out_levels, stream=None):
    arr = _ptr_array(out_levels, RIMG_MAX_LEVELS)
    _check("rimg_pyramid", _lib.rimg_pyramid(n_images, H, W, levels, channels, _ptr(inp), arr, _stream(stream)))


def rimg_normals(sensor, range_img, params, planes_levels, mask0=None, stream=None):
    n = range_img.shape[0] if range_img.dim() == 3 else 1
    arr = _ptr_array(planes_levels, RIMG_MAX_LEVELS)
    _check("rimg_normals", _lib.rimg_normals(sensor.ref(), n, _ptr(range_img), ctypes.byref(params), arr,
                                             _ptr(mask0), _stream(stream)))


def rimg_icp_workspace_bytes(src, n_pairs):
    b = _c_size(0)
    _check("rimg_icp_workspace_bytes", _lib.rimg_icp_workspace_bytes(src.ref(), n_pairs, ctypes.byref(b)))
    return b.value


def rimg_icp_step(src, dst, level, n_pairs, src_range_l, dst_planes_l, dst_range_l, pose, params, update,
                  out29=None, assoc=None, status=None, workspace=None, stream=None):
    _check("rimg_icp_step", _lib.rimg_icp_step(
        src.ref(), dst.ref(), level, n_pairs, _ptr(src_range_l), _ptr(dst_planes_l), _ptr(dst_range_l),
        _ptr(pose), ctypes.byref(params), int(update), _ptr(out29), _ptr(assoc), _ptr(status),
        _ptr(workspace), workspace.numel() if workspace is not None else 0, _stream(stream)))


def rimg_gn_update(n_pairs, sums, pose, status=None, stream=None):
    """The Gauss-Newton update alone: sums float64 [n][32] (0..28 read, 29..31
    written), pose float64 [n][16], both device tensors, updated in place."""
    _check("rimg_gn_update", _lib.rimg_gn_update(n_pairs, _ptr(sums), _ptr(pose), _ptr(status), _stream(stream)))


def rimg_icp_step_static(src, dst, level, n_pairs, src_range_l, dst_planes_l, dst_range_l, pose, params, update,
                         out29=None, assoc=None, status=None, stream=None):
    """rimg_icp_step with its scratch in the library's fixed device array (no
    workspace argument; for callers that cannot allocate)."""
    _check("rimg_icp_step_static", _lib.rimg_icp_step_static(
        src.ref(), dst.ref(), level, n_pairs, _ptr(src_range_l), _ptr(dst_planes_l), _ptr(dst_range_l),
        _ptr(pose), ctypes.byref(params), int(update), _ptr(out29), _ptr(assoc), _ptr(status), _stream(stream)))


def rimg_register_workspace_bytes(src, dst, n_pairs, levels):
    b = _c_size(0)
    _check("rimg_register_workspace_bytes",
           _lib.rimg_register_workspace_bytes(src.ref(), dst.ref(), n_pairs, levels, ctypes.byref(b)))
    return b.value


def _iters(iters):
    return (_c_int * len(iters))(*[int(i) for i in iters])


def rimg_register(src, dst, n_pairs, src_range, dst_range, T_init, T_out, levels, iters, params, status=None,
                  workspace=None, stream=None):
    _check("rimg_register", _lib.rimg_register(
        src.ref(), dst.ref(), n_pairs, _ptr(src_range), _ptr(dst_range), _ptr(T_init), _ptr(T_out), levels,
        _iters(iters), ctypes.byref(params), _ptr(status), _ptr(workspace),
        workspace.numel() if workspace is not None else 0, _stream(stream)))


def rimg_register_last_sums(src, dst, n_pairs, levels, workspace, out32, stream=None):
    _check("rimg_register_last_sums", _lib.rimg_register_last_sums(
        src.ref(), dst.ref(), n_pairs, levels, _ptr(workspace), workspace.numel(), _ptr(out32), _stream(stream)))


def rimg_register_host_workspace_bytes(src, dst, n_pairs, levels, chunk_pairs=0):
    b = _c_size(0)
    _check("rimg_register_host_workspace_bytes", _lib.rimg_register_host_workspace_bytes(
        src.ref(), dst.ref(), n_pairs, levels, chunk_pairs, ctypes.byref(b)))
    return b.value


def rimg_register_host(src, dst, n_pairs, src_range_host, dst_range_host, T_init_host, T_out_host, levels, iters,
                       params, status_host=None, chunk_pairs=0, workspace=None, stream=None):
    """Host tensors (ideally pinned) in and out; synchronises the stream."""
    _check("rimg_register_host", _lib.rimg_register_host(
        src.ref(), dst.ref(), n_pairs, _ptr(src_range_host), _ptr(dst_range_host), _ptr(T_init_host),
        _ptr(T_out_host), levels, _iters(iters), ctypes.byref(params), _ptr(status_host), int(chunk_pairs),
        _ptr(workspace), workspace.numel() if workspace is not None else 0, _stream(stream)))


def rimg_register_host_async(src, dst, n_pairs, src_range_host, dst_range_host, T_init_host, T_out_host, levels,
                             iters, params, status_host=None, chunk_pairs=0, workspace=None, stream=None):
    """Queue the host-buffer registration without synchronising; the caller
    synchronises `stream` before reading outputs or reusing any buffer."""
    _check("rimg_register_host_async", _lib.rimg_register_host_async(
        src.ref(), dst.ref(), n_pairs, _ptr(src_range_host), _ptr(dst_range_host), _ptr(T_init_host),
        _ptr(T_out_host), levels, _iters(iters), ctypes.byref(params), _ptr(status_host), int(chunk_pairs),
        _ptr(workspace), workspace.numel() if workspace is not None else 0, _stream(stream)))


class Groups:
    """A C array of rimg_group built from Python descriptions; keeps every
    referenced object (sensors, parameters, schedules, tensors) alive."""

    def __init__(self, groups):
        self._keep = []
        self.array = (rimg_group * max(len(groups), 1))()
        self.n = len(groups)
        for i, g in enumerate(groups):
            it = _iters(g["iters"])
            prm = g["params"]
            self._keep += [g, it, prm]
            self.array[i] = rimg_group(ctypes.pointer(g["src"].struct), ctypes.pointer(g["dst"].struct),
                                       int(g["n_pairs"]), int(g["levels"]), it, ctypes.pointer(prm),
                                       _ptr(g["src_range"]), _ptr(g["dst_range"]), _ptr(g["T_init"]),
                                       _ptr(g["T_out"]), _ptr(g.get("status")))


def rimg_register_groups_workspace_bytes(groups):
    b = _c_size(0)
    _check("rimg_register_groups_workspace_bytes",
           _lib.rimg_register_groups_workspace_bytes(groups.n, groups.array, ctypes.byref(b)))
    return b.value


def rimg_register_groups(groups, workspace, stream=None):
    _check("rimg_register_groups", _lib.rimg_register_groups(groups.n, groups.array, _ptr(workspace),
                                                             workspace.numel(), _stream(stream)))


def rimg_autotune(groups, workspace, stream=None):
    n = _lib.rimg_autotune(groups.n, groups.array, _ptr(workspace), workspace.numel(), _stream(stream))
    if n < 0:
        raise RimgError("rimg_autotune", n)
    return n


def rimg_autotune_register(src, dst, n_pairs, src_range, dst_range, T_init, T_out, levels, iters, params,
                           workspace, stream=None):
    n = _lib.rimg_autotune_register(
        src.ref(), dst.ref(), n_pairs, _ptr(src_range), _ptr(dst_range), _ptr(T_init), _ptr(T_out), levels,
        _iters(iters), ctypes.byref(params), _ptr(workspace), workspace.numel(), _stream(stream))
    if n < 0:
        raise RimgError("rimg_autotune_register", n)
    return n


def rimg_autotune_clear():
    _check("rimg_autotune_clear", _lib.rimg_autotune_clear())


def rimg_autotune_set(H_l, W_l, n_pairs, threads, blocks_per_pair, schedule=-1):
    _check("rimg_autotune_set", _lib.rimg_autotune_set(H_l, W_l, n_pairs, threads, blocks_per_pair, schedule))


def rimg_gemm_bf16(A, B, C, C_bf16=None, bias=None, relu=False, splits=1, err=None, stream=None):
    """C = A @ B^T on the tcgen05 tensor cores; A [M, K] and B [N, K] bfloat16,
    C float32 [M, N] (or [splits, M, N] with splits > 1)."""
    M, K = A.shape
    N = B.shape[0]
    _check("rimg_gemm_bf16", _lib.rimg_gemm_bf16(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(C),
                                                 C.stride(-2), _ptr(C_bf16), _ptr(bias), int(relu), int(splits),
                                                 _ptr(err), _stream(stream)))


def rimg_sdf_integrate(sensor, level, range_l, T_world_to_sensor, dims, origin, voxel, sdf, weight, trunc=0.0,
                       params=None, n_scans=None, stream=None):
    """Projective SDF integration of n_scans level-`level` range images into
    the dense grid (sdf, weight float32 [nz, ny, nx], updated in place)."""
    n = range_l.shape[0] if n_scans is None else n_scans
    g = rimg_grid(int(dims[0]), int(dims[1]), int(dims[2]), float(voxel), (ctypes.c_float * 3)(*[float(o) for o in origin]))
    _check("rimg_sdf_integrate", _lib.rimg_sdf_integrate(
        sensor.ref(), level, n, _ptr(range_l), _ptr(T_world_to_sensor), ctypes.byref(g), float(trunc), _ptr(sdf),
        _ptr(weight), ctypes.byref(params) if params is not None else None, _stream(stream)))


def rimg_points_to_range(sensor, level, xyz, range_l, counts=None, T_cloud_to_sensor=None, params=None, stream=None):
    """Range images [n, H_l, W_l] of point clouds xyz float32 [n, max_points, 3]
    (nearest point per pixel, +inf where no point lands)."""
    n, m = xyz.shape[0], xyz.shape[1]
    _check("rimg_points_to_range", _lib.rimg_points_to_range(
        sensor.ref(), level, n, m, _ptr(xyz), _ptr(counts), _ptr(T_cloud_to_sensor), _ptr(range_l),
        ctypes.byref(params) if params is not None else None, _stream(stream)))


def rimg_center_init(src, dst, level, src_range_l, dst_range_l, T_out, status=None, stream=None):
    """Initial poses [n, 16] = [I | centre of the target's valid points -
    centre of the source's] from level-l range images [n, H_l, W_l]."""
    n = src_range_l.shape[0] if src_range_l.dim() == 3 else 1
    _check("rimg_center_init", _lib.rimg_center_init(src.ref(), dst.ref(), level, n, _ptr(src_range_l),
                                                     _ptr(dst_range_l), _ptr(T_out), _ptr(status), _stream(stream)))


# ---------------------------------------------------------------------------
# Learned pose proposal

def rimg_cnn_param_count():
    b = _c_size(0)
    _check("rimg_cnn_param_count", _lib.rimg_cnn_param_count(ctypes.byref(b)))
    return b.value


def rimg_cnn_state_bytes():
    b = _c_size(0)
    _check("rimg_cnn_state_bytes", _lib.rimg_cnn_state_bytes(ctypes.byref(b)))
    return b.value


def rimg_cnn_workspace_bytes(n):
    b = _c_size(0)
    _check("rimg_cnn_workspace_bytes", _lib.rimg_cnn_workspace_bytes(int(n), ctypes.byref(b)))
    return b.value


def _images(src, dst):
    H, W = src.shape[-2], src.shape[-1]
    if dst.shape[-2:] != src.shape[-2:]:
        raise ValueError("source and target images differ in size")
    stride = H // RIMG_CNN_IN_H
    return H, W, stride


class ProposalNet:
    """Device state of the proposal network (master FP32 parameters, Adam
    moments, BF16 weight copies) and per-batch-size workspaces."""

    def __init__(self, seed=None, params=None, device="cuda"):
        import torch
        self.n_params = rimg_cnn_param_count()
        self.state = torch.zeros(rimg_cnn_state_bytes(), dtype=torch.uint8, device=device)
        self._ws = {}
        self.err = torch.zeros(1, dtype=torch.int32, device=device)
        if params is not None:
            self.load(params)
        else:
            self.init(0 if seed is None else seed)

    @property
    def params(self):
        """The master parameters (a float32 view into the state)."""
        import torch
        return self.state[:4 * self.n_params].view(torch.float32)

    def init(self, seed, stream=None):
        rimg_cnn_init(self.state, seed, stream)

    def load(self, params, stream=None):
        rimg_cnn_load(self.state, params, stream)

    def workspace(self, n):
        import torch
        ws = self._ws.get(n)
        if ws is None:
            ws = torch.empty(rimg_cnn_workspace_bytes(n), dtype=torch.uint8, device=self.state.device)
            self._ws[n] = ws
        return ws


def rimg_cnn_init(state, seed, stream=None):
    _check("rimg_cnn_init", _lib.rimg_cnn_init(_ptr(state), state.numel(), int(seed) & (2 ** 64 - 1),
                                               _stream(stream)))


def rimg_cnn_load(state, params, stream=None):
    _check("rimg_cnn_load", _lib.rimg_cnn_load(_ptr(state), state.numel(), _ptr(params), _stream(stream)))


def rimg_propose(net, src, dst, n=None, index=None, pred=None, T_out=None, workspace=None, stream=None):
    """Proposals for n pairs: src, dst float32 [*, 8 s, 128 s] device images
    (s = 8 for 64 x 1024 scans); index (int32 [n]) picks the pairs."""
    H, W, stride = _images(src, dst)
    n = (index.numel() if index is not None else src.shape[0]) if n is None else n
    ws = workspace if workspace is not None else net.workspace(n)
    _check("rimg_propose", _lib.rimg_propose(_ptr(net.state), n, H, W, stride, _ptr(src), _ptr(dst), _ptr(index),
                                             _ptr(pred), _ptr(T_out), _ptr(net.err), _ptr(ws), ws.numel(),
                                             _stream(stream)))


def rimg_cnn_grad(net, src, dst, T_label, grad, n=None, index=None, loss=None, pred=None, workspace=None,
                  stream=None):
    H, W, stride = _images(src, dst)
    n = (index.numel() if index is not None else src.shape[0]) if n is None else n
    ws = workspace if workspace is not None else net.workspace(n)
    _check("rimg_cnn_grad", _lib.rimg_cnn_grad(_ptr(net.state), n, H, W, stride, _ptr(src), _ptr(dst), _ptr(index),
                                               _ptr(T_label), _ptr(loss), _ptr(grad), _ptr(pred), _ptr(net.err),
                                               _ptr(ws), ws.numel(), _stream(stream)))


def rimg_cnn_train_step(net, src, dst, T_label, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, n=None,
                        index=None, loss=None, workspace=None, stream=None):
    H, W, stride = _images(src, dst)
    n = (index.numel() if index is not None else src.shape[0]) if n is None else n
    ws = workspace if workspace is not None else net.workspace(n)
    opt = rimg_adam(lr, beta1, beta2, eps)
    _check("rimg_cnn_train_step", _lib.rimg_cnn_train_step(
        _ptr(net.state), net.state.numel(), n, H, W, stride, _ptr(src), _ptr(dst), _ptr(index), _ptr(T_label),
        ctypes.byref(opt), int(step), _ptr(loss), _ptr(net.err), _ptr(ws), ws.numel(), _stream(stream)))


def rimg_profile_begin(max_launches):
    _check("rimg_profile_begin", _lib.rimg_profile_begin(max_launches))


def rimg_profile_end(cap=100000):
    """Returns a list of (kernel_id, level, n_pairs, start_ms, ms) records."""
    kid = (_c_int * cap)()
    lvl = (_c_int * cap)()
    npr = (_c_int * cap)()
    t0 = (ctypes.c_float * cap)()
    ms = (ctypes.c_float * cap)()
    n = _lib.rimg_profile_end(cap, kid, lvl, npr, t0, ms)
    if n < 0:
        raise RimgError("rimg_profile_end", n)
    return [(kid[i], lvl[i], npr[i], t0[i], ms[i]) for i in range(n)]


KERNEL_NAMES = {0: "unproject", 1: "pyramid", 2: "normals", 3: "icp_step", 4: "src_pyramid", 5: "solve", 6: "sdf", 7: "points",
                8: "icp_iters", 9: "icp_queue", 10: "icp_cluster"}

__all__ = [n for n in dir() if n.startswith("rimg_")] + ["Sensor", "Groups", "ProposalNet", "RimgError", "KERNEL_NAMES",
                                                          "RIMG_MAX_LEVELS", "RIMG_FLAG_DEGENERATE", "lib"]
