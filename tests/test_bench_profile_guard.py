"""bench.py reports the step kernel's DRAM traffic and pipe fractions only
while the kernel sources hash to the ones the committed ncu capture was
taken on: any edit to them turns the figures into null.  Checked on a copy
of the tree, stamped with its own sources."""
import importlib.util
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module(root):
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(root, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _stamp(root):
    """Rewrite the profile's source hash to the tree's current sources."""
    import hashlib
    import re
    path = os.path.join(root, "profiles", "k_step_deferred_1e5.md")
    text = open(path).read()
    files = re.search(r"sources:\s*(.+)", text).group(1).split()
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(root, f), "rb").read())
    text = re.sub(r"source_sha256:\s*[0-9a-f]+", "source_sha256: " + h.hexdigest(), text)
    open(path, "w").write(text)


def test_profile_figures_follow_the_source_hash(tmp_path):
    # a copy of the tree whose profile is stamped with its own sources
    copy = tmp_path / "tree"
    shutil.copytree(os.path.join(ROOT, "profiles"), copy / "profiles")
    shutil.copytree(os.path.join(ROOT, "paper_2403_08692_gb300", "csrc"), copy / "paper_2403_08692_gb300" / "csrc")
    shutil.copy(os.path.join(ROOT, "paper_2403_08692_gb300", "build.py"), copy / "paper_2403_08692_gb300" / "build.py")
    shutil.copy(os.path.join(ROOT, "bench.py"), copy / "bench.py")
    _stamp(str(copy))
    b = _bench_module(str(copy))
    prof = b.step_kernel_profile()
    assert prof is not None
    assert b.step_kernel_traffic(10.0) == prof["dram_bytes_per_event_cycle"] * 10.0
    pipes = b.pipe_fractions()
    assert 0.0 < pipes["fp64_pipe_of_active_cycles"] <= 1.0 and 0.0 < pipes["issue_slots_of_active_cycles"] <= 1.0
    # one kernel source edited: the guard drops the figures
    src = copy / "paper_2403_08692_gb300" / "csrc" / "shower_cycle.cuh"
    src.write_text(src.read_text() + "\n// edited\n")
    assert b.step_kernel_profile() is None
    assert b.step_kernel_traffic(10.0) is None and b.pipe_fractions() is None
    # and so does a change of the build flags
    _stamp(str(copy))
    assert b.step_kernel_profile() is not None
    assert b.step_kernel_traffic(10.0, warm=True) == b.step_kernel_profile()["dram_bytes_per_event_cycle_warm"] * 10.0
    flags = copy / "paper_2403_08692_gb300" / "build.py"
    flags.write_text(flags.read_text().replace('"-fmad=false", ', ""))
    assert b.step_kernel_profile() is None
