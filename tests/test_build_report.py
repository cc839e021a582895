"""The compiled kernels' resources (ptxas -v, recorded by the build): the frequency-resident
IP+EM kernels for M = 3, 4 run at their 96-register cap without spilling, the benchmark's
M = 4, N = 6 instantiation among them.  A change elsewhere (a larger argument struct, one
more live value) can push them into local memory; this catches it without a GPU."""
import json
import os
import re
import shutil

import pytest

from paper_2101_08563_gb300 import build


@pytest.fixture(scope="module")
def report():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    build.build()
    if not os.path.exists(build.REPORT_PATH):
        build.build(force=True)
    with open(build.REPORT_PATH) as f:
        return json.load(f)


def test_ip_em_kernels_for_m3_m4_do_not_spill(report):
    found = {}
    for name, res in report.items():
        m = re.search(r"fastfca_em_kernelILi([34])ELi(\d)ELb0ELb0E", name)
        if m:
            found[(int(m.group(1)), int(m.group(2)))] = res
    assert len(found) == 14                              # M 3..4 x N 2..8
    for key, res in found.items():
        assert res["spill_stores"] == 0 and res["spill_loads"] == 0, (key, res)
        assert res["registers"] <= 96, (key, res)


def test_bench_kernel_is_present_at_its_register_cap(report):
    names = [n for n in report if "fastfca_em_kernelILi4ELi6ELb0ELb0E" in n]
    assert len(names) == 1
    res = report[names[0]]
    assert res["registers"] <= 96 and res["stack"] == 0
