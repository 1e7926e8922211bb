"""Host logic of bench.py (CPU only): a kernel's DRAM traffic is taken from its committed ncu
summary only while the summary names the same workload and the same source file content."""
import hashlib
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_needs_the_same_workload_and_source(tmp_path):
    bench = _bench()
    csrc = tmp_path / "paper_1812_05264_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = csrc / "k.cu"
    src.write_text("__global__ void k() {}\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles" / "k_w.md").write_text(
        "# k\n\n- workload: w1\n- k.cu sha256[:16]: %s\n- dram bytes per launch (full size): 12345\n" % sha)
    bench.ROOT = str(tmp_path)
    assert bench.traffic_from_profile("k_w.md", "k.cu", "w1") == 12345.0
    assert bench.traffic_from_profile("k_w.md", "k.cu", "w2") is None        # another workload
    assert bench.traffic_from_profile("missing.md", "k.cu", "w1") is None    # no summary
    src.write_text("__global__ void k() { }\n")                             # the source changed
    assert bench.traffic_from_profile("k_w.md", "k.cu", "w1") is None


def test_committed_profiles_state_their_workload_and_source():
    """Every summary that carries traffic names its workload and a source hash in the form the
    bench reads."""
    prof = os.path.join(ROOT, "profiles")
    for name in os.listdir(prof):
        text = open(os.path.join(prof, name)).read()
        if "dram bytes per launch (full size):" not in text:
            continue
        lines = [ln.strip()[2:] for ln in text.splitlines() if ln.strip().startswith("- ")]
        keys = {ln.split(": ", 1)[0] for ln in lines if ": " in ln}
        assert "workload" in keys, name
        assert any(k.endswith(".cu sha256[:16]") for k in keys), name
