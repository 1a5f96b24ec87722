"""Host-side helpers of bench.py that need no GPU: the instruction-issue roofline and the
source check of the committed ncu counters."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_issue_roofline_arithmetic():
    r = bench.issue_roofline(1.2e9, 2.0, 152, 2000.0)
    # 1.2e9 warp instructions in 2 ms = 600 G/s against 152 x 4 x 2.0 GHz = 1216 G/s
    assert r["achieved"] == pytest.approx(600.0) and r["peak"] == pytest.approx(1216.0)
    assert r["frac"] == pytest.approx(600.0 / 1216.0, abs=1e-4)
    assert bench.issue_roofline(None, 2.0, 152, 2000.0) is None
    assert bench.issue_roofline(1.2e9, 2.0, 152, None) is None


def test_ncu_counters_are_withheld_for_other_sources(monkeypatch):
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda: "0000000000000000")
    assert bench.ncu_traffic("mixed", 256) is None
    assert bench._ncu_per_launch("mixed_warp_inst_per_launch_256", 256) is None


def test_kernel_hash_ignores_comments_and_whitespace(tmp_path, monkeypatch):
    """A comment or formatting edit keeps the identity of the kernel code; a code edit changes it."""
    import shutil
    src = os.path.join(bench.ROOT, "paper_2508_16387_gb300", "csrc")
    dst = tmp_path / "paper_2508_16387_gb300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench._kernel_source_hash()
    f = dst / "m2c_stage.cuh"
    text = f.read_text()
    f.write_text("// a new comment\n" + text.replace("\n", "\n\n", 3) + "\n/* and another */\n")
    assert bench._kernel_source_hash() == h0
    f.write_text(text.replace("kReinitChunk", "kReinitChunk ", 1).replace("const int tid = threadIdx.x",
                                                                         "const int tid = (int)threadIdx.x", 1))
    assert bench._kernel_source_hash() != h0


def test_launch_count_matches_the_launch_list():
    """The 256^3 launch list (ncu, mixed part of `bench.py --steps 10 --warmup 3 --no-cpu --no-e2e
    --l1-steps 0`) holds 72 stage, 72 FIVER, 72 finish, 36 phase-update, 36 end-of-step, 20
    reinitialisation and 4 copy launches = 312 for the step indices that run executes: warm-up
    0-2, the profiled pass 3-12, the timed steps 3-12 again from the restored state, then the
    FP32-start line's warm-up 13-15, profiled pass 16-20 and timed steps 16-20."""
    idx = list(range(0, 13)) + list(range(3, 13)) + list(range(13, 21)) + list(range(16, 21))
    assert len(idx) == 36
    assert sum(bench.launches_per_step(i, 10, 5) for i in idx) == 72 * 3 + 36 * 2 + 20 + 4
    assert sum(bench.launches_per_step(i, 10, 5) for i in range(100)) == 860
    assert bench.launches_per_step(9, 0, 5) == 8 and bench.launches_per_step(9, 10, 0) == 8

