"""CPU checks of bench.py's bookkeeping (no GPU): the DRAM traffic of the
roofline comes from profiles/traffic.txt only while the kernel sources it
was measured on are unchanged."""
import importlib.util
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def fake_tree(tmp_path):
    csrc = tmp_path / "paper_2309_07270_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("xd_types.cuh", "xd_device.cuh", "xd_lockstep16.cuh"):
        shutil.copy(os.path.join(ROOT, "paper_2309_07270_gb300", "csrc", f), csrc / f)
    (tmp_path / "profiles").mkdir()
    return csrc


def test_traffic_is_used_only_for_the_measured_sources(tmp_path):
    bench = load_bench()
    csrc = fake_tree(tmp_path)
    bench.ROOT = str(tmp_path)
    sha = bench.kernel_source_sha()
    assert len(sha) == 16
    (tmp_path / "profiles" / "traffic.txt").write_text(
        f"kernel=lockstep16_kernel<4,8> source_sha={sha} dram_bytes_per_launch=123\n"
        f"kernel=lockstep16_kernel<8,8> source_sha=0000000000000000 dram_bytes_per_launch=456\n")
    assert bench.traffic_from_profile("lockstep16_kernel<4,8>") == 123.0
    assert bench.traffic_from_profile("lockstep16_kernel<8,8>") is None  # other sources
    assert bench.traffic_from_profile("lockstep_kernel<4,16>") is None   # not measured
    # any change to the kernel sources drops the number
    with open(csrc / "xd_lockstep16.cuh", "a") as f:
        f.write("\n")
    assert bench.kernel_source_sha() != sha
    assert bench.traffic_from_profile("lockstep16_kernel<4,8>") is None


def test_committed_traffic_file_parses():
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    for line in open(path):
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        assert f["kernel"].startswith("lockstep")
        assert len(f["source_sha"]) == 16
        assert float(f["dram_bytes_per_launch"]) > 0


def test_committed_traffic_matches_the_current_kernel_sources():
    """The DRAM traffic in profiles/traffic.txt was measured on the kernel
    sources as they are, for the first-tier kernel the default bench line
    runs (packed 2 lanes x 32 cells at X = 50): the line can use it."""
    bench = load_bench()
    assert bench.traffic_from_profile("lockstep16_kernel<2,16>") is not None


def test_seed_discovery_failure_is_reported_not_raised(monkeypatch):
    """A seed-discovery run that fails (here: its child process exits 1)
    becomes an error entry of the line's seed_discovery object."""
    bench = load_bench()

    class Done:
        returncode = 1
        stdout = "build ok\n"
        stderr = "Traceback ...\nRuntimeError: no device\n"

    monkeypatch.setattr(bench.subprocess, "run", lambda *a, **k: Done())
    out = bench.seed_discovery_runs(genome=1000, timeout_s=5)
    assert out["sort"] == {"error": "exit 1: RuntimeError: no device"}
    assert out["rowwise"]["error"].startswith("exit 1")

    assert out["products_agree"] is None

    class Good:
        returncode = 0
        stdout = ('{"value": 5.0, "unit": "occurrences/s", "ms_per_step": 2.0, "product": "sort", '
                  '"candidates_sha256": "00ff"}\n')
        stderr = ""

    monkeypatch.setattr(bench.subprocess, "run", lambda *a, **k: Good())
    out = bench.seed_discovery_runs(genome=1000, timeout_s=5)
    assert out["sort"]["value"] == 5.0 and out["rowwise"]["ms_per_step"] == 2.0
    assert out["products_agree"] is True
