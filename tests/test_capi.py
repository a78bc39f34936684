"""The C ABI on the CPU: the library loads, exports every function the header
declares, its structs match the Python mirrors, and host-side argument checks
reject bad input before any CUDA call (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from tests.conftest import ROOT

R = pytest.importorskip("paper_2112_02779_b300.rimg")
from paper_2112_02779_b300 import _abi  # noqa: E402

HEADER = os.path.join(ROOT, "include", "rimg.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(rimg_\w+)\s*\(", txt, flags=re.M)))


def test_header_declarations_are_exported():
    names = _declared()
    assert sorted(names) == sorted(_abi.HEADER_FUNCTIONS)
    out = subprocess.run(["nm", "-D", "--defined-only", R.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(rimg_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(R.lib(), n)


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "rimg.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(rimg_level), sizeof(rimg_sensor), sizeof(rimg_params));
  printf("%zu %zu %zu %zu\n", offsetof(rimg_level, off_rows), offsetof(rimg_level, off_bins),
         offsetof(rimg_sensor, d_tables), offsetof(rimg_sensor, level));
  printf("%zu %zu %zu\n", offsetof(rimg_params, proj_iters), offsetof(rimg_params, kahan),
         offsetof(rimg_params, streams));
  printf("%zu %zu %zu %zu\n", sizeof(rimg_group), offsetof(rimg_group, iters), offsetof(rimg_group, params),
         offsetof(rimg_group, status));
  printf("%zu %zu %zu\n", sizeof(rimg_grid), offsetof(rimg_grid, voxel), offsetof(rimg_grid, origin));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    L, S, P, G, Gr = _abi.rimg_level, _abi.rimg_sensor, _abi.rimg_params, _abi.rimg_group, _abi.rimg_grid
    assert vals == [ctypes.sizeof(L), ctypes.sizeof(S), ctypes.sizeof(P),
                    L.off_rows.offset, L.off_bins.offset, S.d_tables.offset, S.level.offset,
                    P.proj_iters.offset, P.kahan.offset, P.streams.offset,
                    ctypes.sizeof(G), G.iters.offset, G.params.offset, G.status.offset,
                    ctypes.sizeof(Gr), Gr.voxel.offset, Gr.origin.offset]


def test_default_params_and_status_strings():
    p = R.rimg_default_params()
    assert p.huber_delta == pytest.approx(0.5) and p.max_corr_dist == 0.0
    assert p.normal_rel_jump == pytest.approx(0.1) and p.proj_iters == 3 and p.kahan == 1 and p.streams == 2
    for code in _abi.STATUS_NAMES:
        assert R.rimg_status_string(code)
    assert R.rimg_status_string(12345) == "unknown status"


def test_table_bytes_size_rules():
    lib = R.lib()
    b = ctypes.c_size_t()
    assert lib.rimg_sensor_table_bytes(64, 1024, 4, ctypes.byref(b)) == 0 and b.value > 0
    assert lib.rimg_sensor_table_bytes(64, 1000, 4, ctypes.byref(b)) == -3      # W % (4 << 3)
    assert lib.rimg_sensor_table_bytes(4, 1024, 4, ctypes.byref(b)) == -3       # H >> 3 < 2
    assert lib.rimg_sensor_table_bytes(64, 1024, 9, ctypes.byref(b)) == -1      # too many levels
    assert lib.rimg_sensor_table_bytes(64, 1024, 4, None) == -1


def _build_raw(phi, theta, r0=0.0, H=None, W=64, levels=1, dptr=4096, nbytes=1 << 20):
    H = len(phi) if H is None else H
    phi = np.ascontiguousarray(phi, np.float64)
    theta = np.ascontiguousarray(theta, np.float64)
    s = _abi.rimg_sensor()
    return R.lib().rimg_sensor_build(H, W, levels, phi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     theta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), r0, dptr, nbytes,
                                     ctypes.byref(s))


def test_sensor_build_rejects_bad_tables_before_touching_the_device():
    # the device pointer is fake: these calls must fail in host-side checks
    H = 8
    good = np.deg2rad(np.linspace(10, -20, H))
    bad = good.copy()
    bad[3] = bad[2]                                   # not strictly monotone
    assert _build_raw(bad, np.zeros(H)) == -2
    nan = good.copy()
    nan[1] = np.nan
    assert _build_raw(nan, np.zeros(H)) == -2
    assert _build_raw(good, np.full(H, 4.0)) == -2    # |theta| >= pi
    assert _build_raw(good, np.zeros(H), r0=-1.0) == -1
    assert _build_raw(good, np.zeros(H), dptr=4097) == -4      # misaligned tables
    assert _build_raw(good, np.zeros(H), nbytes=16) == -4      # too small


def test_entry_points_reject_null_and_bad_arguments():
    lib = R.lib()
    p = R.rimg_default_params()
    iters = (ctypes.c_int * 1)(1)
    assert lib.rimg_register(None, None, 1, None, None, None, None, 1, iters, ctypes.byref(p), None, None, 0,
                             None) == -1
    assert lib.rimg_icp_step(None, None, 0, 1, None, None, None, None, ctypes.byref(p), 1, None, None, None,
                             None, 0, None) == -1
    assert lib.rimg_pyramid(1, 64, 64, 2, 3, 4096, None, None) == -1       # channels must be 1 or 4
    assert lib.rimg_pyramid(1, 63, 64, 2, 1, 4096, None, None) == -3       # H not divisible
    bad = R.rimg_default_params(normal_rel_jump=0.7)
    assert lib.rimg_normals(None, 1, None, ctypes.byref(bad), None, None, None) == -1
    assert lib.rimg_profile_begin(-1) == -1
    fake = 1 << 20                                    # never dereferenced: the checks come first
    assert lib.rimg_gn_update(-1, fake, fake, None, None) == -1
    assert lib.rimg_gn_update(0, None, None, None, None) == 0     # no pairs: no-op
    assert lib.rimg_gn_update(1, None, fake, None, None) == -1
    assert lib.rimg_gn_update(1, fake + 4, fake, None, None) == -1   # sums not 8-byte aligned


def test_autotune_set_takes_the_cluster_schedules():
    """Schedules -1 (leave), 0 (per-iteration launches), 1 (one block per
    pair), 2, 4 and 8 (clusters of that many blocks per pair); nothing else.
    The table is host memory: no device is touched."""
    lib = R.lib()
    try:
        for s in (-1, 0, 1, 2, 4, 8):
            assert lib.rimg_autotune_set(32, 512, 7, 0, 0, s) == 0, s
        for s in (-2, 3, 5, 6, 7, 9, 16):
            assert lib.rimg_autotune_set(32, 512, 7, 0, 0, s) == -1, s
        assert lib.rimg_autotune_set(32, 512, 7, 128, 33, 2) == -1      # blocks per pair above H_l
    finally:
        assert lib.rimg_autotune_clear() == 0


def test_normals_entry_point_rejects_misaligned_buffers_on_the_host():
    """rimg_normals reads ranges and writes planes 16 bytes at a time: a
    range or plane pointer off a 16-byte boundary is refused before any launch."""
    lib = R.lib()
    s = _abi.rimg_sensor()
    fake = 1 << 20                                    # never dereferenced: the checks come first
    s.d_tables = fake
    s.H, s.W, s.levels = 16, 64, 2
    s.level[0].H, s.level[0].W = 16, 64
    s.level[1].H, s.level[1].W = 8, 32
    p = R.rimg_default_params()
    vp = ctypes.c_void_p
    good = (vp * _abi.RIMG_MAX_LEVELS)(fake, fake + 4096)
    assert lib.rimg_normals(ctypes.byref(s), 1, fake + 4, ctypes.byref(p), good, None, None) == -1
    bad = (vp * _abi.RIMG_MAX_LEVELS)(fake, fake + 4104)
    assert lib.rimg_normals(ctypes.byref(s), 1, fake, ctypes.byref(p), bad, None, None) == -1
    assert lib.rimg_normals(ctypes.byref(s), 0, fake + 4, ctypes.byref(p), good, None, None) == 0   # no-op


def test_cnn_entry_points_check_arguments_on_the_host():
    lib = R.lib()
    n = ctypes.c_size_t()
    assert lib.rimg_cnn_param_count(ctypes.byref(n)) == 0 and n.value == 280550
    assert lib.rimg_cnn_state_bytes(ctypes.byref(n)) == 0 and n.value >= 3 * 4 * 280550
    assert lib.rimg_cnn_workspace_bytes(-1, ctypes.byref(n)) == -1
    assert lib.rimg_cnn_workspace_bytes(_abi.RIMG_CNN_MAX_BATCH + 1, ctypes.byref(n)) == -1
    assert lib.rimg_cnn_workspace_bytes(64, ctypes.byref(n)) == 0 and n.value > 0
    fake = 1 << 20                                    # never dereferenced: the checks come first
    # state misaligned / too small
    assert lib.rimg_cnn_init(fake + 4, 1 << 30, 1, None) == -4
    assert lib.rimg_cnn_init(fake, 16, 1, None) == -4
    # image size must be 8 s x 128 s
    assert lib.rimg_propose(fake, 4, 64, 1000, 8, fake, fake, None, None, None, None, fake, 1 << 40, None) == -3
    assert lib.rimg_propose(fake, 4, 64, 1024, 0, fake, fake, None, None, None, None, fake, 1 << 40, None) == -1
    # workspace too small
    assert lib.rimg_propose(fake, 4, 64, 1024, 8, fake, fake, None, None, None, None, fake, 16, None) == -4
    # n = 0 is a no-op
    assert lib.rimg_propose(fake, 0, 8, 128, 1, None, None, None, None, None, None, None, 0, None) == 0
    opt = _abi.rimg_adam(1e-3, 0.9, 1.5, 1e-8)     # beta2 >= 1
    assert lib.rimg_cnn_train_step(fake, 1 << 30, 4, 8, 128, 1, fake, fake, None, fake, ctypes.byref(opt), 1, None,
                                   None, fake, 1 << 40, None) == -1
    opt = _abi.rimg_adam(1e-3, 0.9, 0.999, 1e-8)
    assert lib.rimg_cnn_train_step(fake, 1 << 30, 4, 8, 128, 1, fake, fake, None, fake, ctypes.byref(opt), 0, None,
                                   None, fake, 1 << 40, None) == -1


def test_sdf_entry_point_checks_arguments_on_the_host():
    lib = R.lib()
    phi = np.deg2rad(np.linspace(10, -20, 16))
    s = _abi.rimg_sensor()
    # a sensor struct built against a fake device pointer (host checks only)
    assert R.lib().rimg_sensor_build(16, 64, 2, phi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     np.zeros(16).ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0.0, 4096, 16,
                                     ctypes.byref(s)) == -4
    g = _abi.rimg_grid(4, 4, 4, 0.1, (ctypes.c_float * 3)(0, 0, 0))
    fake = 1 << 20
    assert lib.rimg_sdf_integrate(None, 0, 1, fake, fake, ctypes.byref(g), 0.0, fake, fake, None, None) == -1
    bad = _abi.rimg_grid(4, 4, 4, 0.0, (ctypes.c_float * 3)(0, 0, 0))
    s.d_tables = fake
    s.H, s.W, s.levels = 16, 64, 1
    s.level[0].H, s.level[0].W = 16, 64
    assert lib.rimg_sdf_integrate(ctypes.byref(s), 0, 1, fake, fake, ctypes.byref(bad), 0.0, fake, fake, None,
                                  None) == -1                       # voxel size <= 0
    assert lib.rimg_sdf_integrate(ctypes.byref(s), 1, 1, fake, fake, ctypes.byref(g), 0.0, fake, fake, None,
                                  None) == -1                       # level out of range
    assert lib.rimg_sdf_integrate(ctypes.byref(s), 0, 1, None, fake, ctypes.byref(g), 0.0, fake, fake, None,
                                  None) == -1                       # missing images
    assert lib.rimg_sdf_integrate(ctypes.byref(s), 0, 0, None, None, ctypes.byref(g), 0.0, None, None, None,
                                  None) == 0                        # no scans: no-op
