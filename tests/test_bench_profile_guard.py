"""bench.py reports the step kernel's DRAM traffic and pipe fractions only
while the kernel sources hash to the ones the committed ncu capture was
taken on: any edit to them turns the figures into null."""
import importlib.util
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module(root):
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(root, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_profile_figures_follow_the_source_hash(tmp_path):
    b = _bench_module(ROOT)
    prof = b.step_kernel_profile()
    assert prof is not None, "committed profile does not match the committed kernel sources"
    assert b.step_kernel_traffic(10.0) == prof["dram_bytes_per_event_cycle"] * 10.0
    pipes = b.pipe_fractions()
    assert 0.0 < pipes["fp64_pipe_of_active_cycles"] <= 1.0 and 0.0 < pipes["issue_slots_of_active_cycles"] <= 1.0

    # a copy of the tree with one kernel source edited: the guard drops the figures
    copy = tmp_path / "tree"
    shutil.copytree(os.path.join(ROOT, "profiles"), copy / "profiles")
    shutil.copytree(os.path.join(ROOT, "paper_2403_08692_gb300", "csrc"), copy / "paper_2403_08692_gb300" / "csrc")
    shutil.copy(os.path.join(ROOT, "bench.py"), copy / "bench.py")
    b2 = _bench_module(str(copy))
    assert b2.step_kernel_profile() is not None
    src = copy / "paper_2403_08692_gb300" / "csrc" / "shower_cycle.cuh"
    src.write_text(src.read_text() + "\n// edited\n")
    assert b2.step_kernel_profile() is None
    assert b2.step_kernel_traffic(10.0) is None and b2.pipe_fractions() is None
