"""Host logic of bench.py: per-launch counters recorded in a profile summary
are read only while the summary's source hash equals the kernel sources'
hash, and each counter by its own key."""
import os

import bench


def test_recorded_counters_follow_the_source_hash(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for f in bench.KERNEL_SOURCES:                       # the real kernel sources, copied
        dst = tmp_path / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(here, f), "rb").read())
    h = bench.kernel_source_hash()
    (prof / "s.md").write_text(f"source_sha256: {h}\n"
                               "traffic_bytes_per_launch[k_sweep_B]: 1234\n"
                               "warp_instructions_per_launch[k_sweep_B]: 99\n")
    assert bench.recorded_traffic("s.md", "k_sweep_B") == 1234
    assert bench.recorded_traffic("s.md", "k_sweep_B", "warp_instructions_per_launch") == 99
    assert bench.recorded_traffic("s.md", "k_sweep_C") is None
    assert bench.recorded_traffic("missing.md", "k_sweep_B") is None
    # a comment does not change the code the counters were taken on; a
    # changed line of code invalidates every recorded counter
    src = tmp_path / bench.KERNEL_SOURCES[0]
    src.write_bytes(src.read_bytes() + b"\n// a comment\n")
    assert bench.kernel_source_hash() == h
    src.write_bytes(src.read_bytes() + b"\nconstexpr int kChanged = 1;\n")
    assert bench.kernel_source_hash() != h
    assert bench.recorded_traffic("s.md", "k_sweep_B") is None


def test_committed_profile_matches_the_sources():
    # the committed summary carries the counters the bench line reports
    got = bench.recorded_traffic("sweeps_oscillating_3d_f32_list.md", "k_sweep_B")
    assert got is not None and got > 0
    assert bench.recorded_traffic("sweeps_oscillating_3d_f32_list.md", "k_sweep_B",
                                  "warp_instructions_per_launch") > 0



def test_hbm_roof_reads_the_measured_peak_else_the_fallback(tmp_path):
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6000.0}')
    r = bench.hbm_roof(3 * 10**8, 1e-4, root=str(tmp_path))           # 300 MB in 0.1 ms = 3000 GB/s
    assert r["achieved"] == 3000.0 and r["peak"] == 6000.0 and r["frac"] == 0.5
    assert r["peak_source"].startswith("measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text("{}")
    r = bench.hbm_roof(3 * 10**8, 1e-4, root=str(tmp_path))
    assert r["peak"] == bench.HBM_FALLBACK_GBS and r["peak_source"].startswith("fallback")


def test_reference_arm_prints_its_line_on_the_host():
    # the reference arm times the oracle on the host cores only; on the 2D
    # static drop (7.4k particles) one timed step takes a few seconds
    import json
    import subprocess
    import sys
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "laplace_2d",
                        "--steps", "1", "--warmup", "3"], cwd=here, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == "laplace_2d" and line["higher_is_better"] is True
