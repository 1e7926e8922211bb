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


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler(bench, lines):
    cs = bench.ClockSampler(0)
    cs.proc = _FakeProc()
    cs.lines = list(lines)
    return cs.stop()


def test_clock_summary_reads_nvidia_smi_lines():
    """The clocks record: median SM clock under load, the maximum, and every throttle reason seen
    active ('Not Active' is not active); malformed lines are skipped."""
    bench = _bench()
    na = "Not Active"
    lines = [f"0, {mhz}, 2070, 900.5, 0x0000000000000000, {na}, {na}, {na}, {na}" for mhz in
             (2070, 2055, 2070, 1980, 2070)]
    lines.append(f"0, 1965, 2070, 1398.0, 0x0000000000000004, {na}, {na}, {na}, Active")
    lines += ["", "garbage", "0, [N/A], 2070, 1, 0x0, a, b, c, d"]
    out = _sampler(bench, lines)
    assert out["sm_mhz"] == 2062.5 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 6
    assert out["reasons"] == ["sw_power_cap"]
    out = _sampler(bench, [f"0, 1500, 2070, 700, 0x68, Active, Active, {na}, {na}"])
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    off = bench.ClockSampler(0, enabled=False)
    off.start()
    assert off.stop()["reasons"] == ["not sampled (--no-clocks)"]


def test_bench_order_rule_and_default_workload():
    """The bench takes the library's order rule and, by default, the 10,000-atom fcc workload at
    kT = 0.025 eV with 512 probes."""
    from paper_1812_05264_gb300 import api
    bench = _bench()
    for W, kT in ((120.0, 0.025), (40.0, 0.5), (10.0, 3.0)):
        assert bench.order_rule(W, kT) == api.order_for(W, kT)
    wk = bench.make_workload("fcc10k")
    assert wk.n_atoms == 10000 and wk.n_probes == 512 and wk.kT == 0.025 and wk.n_orb == 9
    assert wk.mixed and wk.name.startswith("fcc10000")
    assert bench.make_workload("fcc10k", rank=1).probe_seed == wk.probe_seed + 1   # replicas


def test_reference_arm_prints_one_contract_line(capsys):
    """`bench.py --impl reference` times the oracle on the host: one JSON line with the contract's
    keys, its own value as cpu_baseline and e2e, no host-device bytes; other ranks print nothing."""
    import argparse
    import json
    bench = _bench()
    bench.oracle_sample.__defaults__ = (30,)           # a 30-atom sample keeps this test short
    args = argparse.Namespace(workload="fcc1k", atom_order="radial", probes=None, warmup=1,
                              steps=2, gpus=1)
    assert bench.run_reference(args, 1, 2) == 0
    assert capsys.readouterr().out == ""
    assert bench.run_reference(args, 0, 1) == 0
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 2
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1 and "30 atoms" in line["cpu_baseline"]["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("fcc30") and line["config"]["sample_of"] == "fcc1k"
