"""Host-side logic of bench.py, on the CPU: the summary of the per-level
GPU-vs-oracle pose check, and the committed ncu summaries it takes traffic
and instruction counts from."""
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


def test_pose_check_summarises_the_per_level_report():
    b = _bench()
    rep = {"pairs": 3, "levels_checked": 12, "max_err": [2e-4, 3e-4], "explained": 1, "unexplained": 1,
           "by_kind": {"near-tie": 1},
           "beyond": [dict(pair=1, level_index=3, err=[2e-4, 3e-4], split=4, split_ties=2, split_off_tie=0,
                           step_err_given_max=[1e-7, 2e-7], explained=True, kind="near-tie"),
                      dict(pair=2, level_index=2, err=[1e-4, 1.5e-4], split=None, split_ties=0, split_off_tie=0,
                           step_err_given_max=[1e-3, 1e-3], explained=False)]}
    whole = [(1e-6, 2e-6), (2e-4, 3e-4), (5e-5, 1e-5)]
    r = b.pose_check(rep, whole)
    assert r["pairs"] == 3 and r["levels_checked"] == 12 and r["levels_within_1e-4"] == 10
    assert r["levels_beyond_1e-4_explained"] == 1 and r["levels_beyond_1e-4_unexplained"] == 1
    assert r["whole_registration_within_1e-4"] == 2
    assert r["whole_registration_median_err"] == [5e-5, 1e-5]
    assert [x["pair"] for x in r["beyond"]] == [1, 2]
    assert r["explained_by_kind"] == {"near-tie": 1} and [x["kind"] for x in r["beyond"]] == ["near-tie", None]


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
