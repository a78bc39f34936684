"""Host-side logic of bench.py, on the CPU: the pose check that reads the
GPU-vs-oracle differences with the oracle's own end-of-schedule motion, and
the committed ncu summaries it takes traffic and instruction counts from."""
import importlib.util
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_pose_check_reads_settled_and_moving_pairs():
    b = _bench()
    # pair 0: settled, within the bar; pair 1: moving (last 2e-4 / 3e-4, previous 3e-4 / 4e-4),
    # beyond 1e-4 but inside 1e-4 + 3 x tail; pair 2: moving, within 1e-4
    err = [(1e-6, 2e-6), (2e-4, 3e-4), (5e-5, 1e-5)]
    last = [(1e-6, 1e-6), (2e-4, 3e-4), (1e-4, 1e-4)]
    prev = [(2e-6, 2e-6), (3e-4, 4e-4), (1e-4, 1e-4)]
    r = b.pose_check(err, last, prev)
    assert r["pairs"] == 3 and r["within_1e-4"] == 2 and r["settled_pairs"] == 1
    assert r["settled_within_1e-4"] and r["beyond_1e-4_all_unsettled_within_tail_bar"]
    assert r["max_err_settled"] == [1e-6, 2e-6]
    # a settled pair beyond the bar fails the check
    r = b.pose_check([(2e-4, 0.0)], [(1e-6, 1e-6)], [(1e-6, 1e-6)])
    assert not r["settled_within_1e-4"] and not r["beyond_1e-4_all_unsettled_within_tail_bar"]
    # a moving pair beyond its tail bar fails it too: last 1e-5, previous 1e-4 -> rho 0.1,
    # tail = max(last, last rho / (1 - rho)) = 1e-5, bar 1.3e-4
    r = b.pose_check([(2e-4, 0.0)], [(1e-5, 1e-4)], [(1e-4, 1e-4)])
    assert not r["beyond_1e-4_all_unsettled_within_tail_bar"]
    r = b.pose_check([(1.25e-4, 0.0)], [(1e-5, 1e-4)], [(1e-4, 1e-4)])
    assert r["beyond_1e-4_all_unsettled_within_tail_bar"]


def test_committed_profiles_carry_the_keys_bench_reads():
    for name, keys in (("icp_step_level0_64x1024.md", ("dram_bytes_per_pair_per_launch", "instructions_per_pixel")),
                       ("sdf_integrate_512x512x64.md", ("instructions_per_update",))):
        txt = open(os.path.join(ROOT, "profiles", name)).read()
        assert re.search(r"kernel_source_hash:\s*[0-9a-f]{16}", txt), name
        for k in keys:
            m = re.search(re.escape(k) + r":\s*([0-9.eE+-]+)", txt)
            assert m and float(m.group(1)) > 0, (name, k)


def test_kernel_source_hash_is_stable_and_file_sensitive():
    b = _bench()
    h1 = b.kernel_source_hash()
    h2 = b.kernel_source_hash()
    assert h1 == h2 and re.fullmatch(r"[0-9a-f]{16}", h1)
    assert b.kernel_source_hash(("kernel_sdf.cu", "rimg_device.cuh", "rimg_internal.h")) != h1
