"""The launch geometry of every kernel, for every shape the library accepts, against the
GB300 limits (CPU).  `launch_geometry.cu` includes the library's launch headers and calls their
host functions (threads per CTA, frames per thread, shared memory per CTA, cluster shapes);
it is compiled with nvcc and run on the host, with no CUDA call."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_every_shape_fits_the_launch_limits(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "launch_geometry")
    build = subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                            "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "launch_geometry.cu"),
                            "-o", exe], capture_output=True, text=True)
    assert build.returncode == 0, build.stdout + build.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0 and run.stdout.strip() == "ok", run.stdout + run.stderr
