"""bench.py's own arithmetic, on the CPU: the algorithmic bytes per node update
(the figures the roofline divides by), the kernel launches that one lbm_step
call makes in each step form (the line's gpu_launches), and the kernel-source
hash that gates the stored ncu traffic."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_per_update():
    # D2Q9 flow + D2Q5 PCM + D2Q5 metal: 19 populations read and written once,
    # plus the exchange history
    assert bench.bytes_per_update(5, 1, 1) == 160
    assert bench.bytes_per_update(5, 1, 2) == bench.bytes_per_update(5, 1, 3) == 84
    assert bench.bytes_per_update(5, 1, 0) == 320
    assert bench.bytes_per_update(9, 1, 1) == 224
    # the implementation's extra planes are reported apart
    assert bench.stored_bytes_per_update(5, 1, 1) - bench.bytes_per_update(5, 1, 1) == 8
    assert bench.stored_bytes_per_update(5, 1, 2) - bench.bytes_per_update(5, 1, 2) == 8


@pytest.mark.parametrize("form,steps,launches", [
    (1, 64, 64), (2, 20000, 20000),
    (3, 64, 32),                    # one graph of 32 two-step launches
    (3, 20000, 10000),              # 312 graphs, then 32 steps as 8 pairs of launches
    (3, 70, 32 + 2 + 2),            # a graph, one pair of two-step launches, two single steps
    (3, 6, 2 + 2),
])
def test_launches_per_lbm_step_call(form, steps, launches):
    assert bench.launches_per_call(form, steps) == launches


def test_source_hash_ignores_comments(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1701_00702_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in ("lbm_kernels.cuh", "lbm_launch.cuh", "lbm_kernels_f32.cu"):
        (csrc / name).write_text((bench.ROOT / "paper_1701_00702_gb300" / "csrc" / name).read_text())
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    h0 = bench.kernel_sources_hash()
    k = csrc / "lbm_kernels.cuh"
    k.write_text(k.read_text() + "\n// a comment changes no code\n\n")
    assert bench.kernel_sources_hash() == h0
    k.write_text(k.read_text() + "constexpr int kAnotherConstant = 1;\n")
    assert bench.kernel_sources_hash() != h0
