"""The TSQR planner on the host (no GPU): tests/plan_check.cu includes the planner and the
autotuner's candidate list, plans every candidate for widths 1-1024 and row counts 1-9M in
both precisions, and checks that planning a block again (the tuner's choice after the
rule) gives the same plan as planning a fresh block, and that every launch of the plan
fits its kernel's shared-memory limit.  A plan that kept the fold flags of the rule's plan
after switching to the thread-block-per-tile path launched the fold kernel with the tile's
shared memory, which the device refuses."""
import os
import shutil
import subprocess

import pytest

from paper_2204_00525_gb300 import build_lib

HERE = os.path.dirname(os.path.abspath(__file__))


def test_replanned_blocks_equal_fresh_plans_and_fit_shared_memory(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    build_lib.build()                    # the leaf objects the planner's translation unit calls
    objs = [os.path.join(build_lib.BUILD, f) for f in ("tsqr_tc.o", "tsqr_reg_f32.o", "tsqr_reg_f64.o")]
    exe = str(tmp_path / "plan_check")
    cmd = ([nvcc] + build_lib.ARCH_FLAGS + ["-O1", "-std=c++17", "-I" + build_lib.INCLUDE, "-I" + build_lib.CSRC,
                                            os.path.join(HERE, "plan_check.cu")] + objs + ["-o", exe])
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert " 0 failed" in r.stdout
