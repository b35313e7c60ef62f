"""Host-side logic of bench.py, on the CPU: the clock summary that decides
whether a run is kept, the nearest-rank percentiles of the latency figures,
the code hash that ties the committed DRAM traffic record to the traversal
sources it was measured on, and the reference (oracle) arm's JSON line."""
import os

import pytest

import bench


def test_clock_summary_median_max_and_active_reasons():
    lines = [
        "2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "[N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active\n",   # unreadable sample
        "garbage\n",
    ]
    out = bench.summarize_clocks(lines)
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_summary_names_a_thermal_slowdown_and_a_low_clock():
    lines = ["1200, 2070, 800, 0x40, Not Active, Active, Not Active, Not Active\n"] * 4
    out = bench.summarize_clocks(lines)
    assert out["reasons"] == ["hw_thermal_slowdown"]
    assert out["sm_mhz"] == 1200.0 and out["sm_max_mhz"] == 2070.0


def test_clock_summary_without_samples_is_none():
    assert bench.summarize_clocks([]) is None
    assert bench.summarize_clocks(["only, three, fields\n"]) is None


def test_nearest_rank_percentiles():
    xs = list(range(1, 101))
    assert bench.pct(xs, 0.5) == 50
    assert bench.pct(xs, 0.99) == 99
    assert bench.pct(xs, 1.0) == 100
    assert bench.pct([7.0], 0.99) == 7.0
    assert bench.pct([4, 1, 3, 2], 0.5) == 2   # order of the input does not matter


def test_code_hash_ignores_comments_and_blank_lines(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    a.write_text("int f(int x) {\n    return x + 1;\n}\n")
    b.write_text("// a comment\nint f(int x) {   \n\n    return x + 1;  // trailing comment\n}\n")
    assert bench.code_sha(str(a)) == bench.code_sha(str(b))
    b.write_text("int f(int x) {\n    return x + 2;\n}\n")
    assert bench.code_sha(str(a)) != bench.code_sha(str(b))
    # file order and boundaries count
    assert bench.code_sha(str(a), str(b)) != bench.code_sha(str(b), str(a))


def test_traffic_record_only_for_the_sources_it_was_measured_on(tmp_path, monkeypatch):
    txt = open(os.path.join(bench.ROOT, "profiles", "trace_pair_medium.md")).read()
    assert "traversal_code_sha256_16:" in txt and "dram_bytes_per_traversal_launch:" in txt
    # a source set other than the measured one gives no record
    other = tmp_path / "other.cu"
    other.write_text("__global__ void k() {}\n")
    monkeypatch.setattr(bench, "TRAVERSAL_SOURCES", [str(other)])
    assert bench.traffic_record() is None


def test_traffic_record_value_is_a_plausible_byte_count():
    rec = bench.traffic_record()
    if rec is None:
        pytest.skip("traversal sources changed since the DRAM capture (the bench then reports traffic null)")
    # per launch: more than the rays read, far less than the algorithmic bytes (the BVH is in L2)
    assert 1e6 < rec < 1.33e9


def test_clock_sampler_stop_reads_and_removes_its_file(tmp_path):
    """The sampler's stop path: signal the sampling process, summarise its CSV
    file, delete it (a stand-in process object replaces nvidia-smi)."""
    class Proc:
        signals = []

        def send_signal(self, sig):
            self.signals.append(sig)

        def wait(self, timeout=None):
            return 0

    path = tmp_path / "clocks.csv"
    path.write_text("2070, 2070, 1000, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "2055, 2070, 1300, 0x4, Not Active, Not Active, Not Active, Active\n")
    cs = bench.ClockSampler(0)
    cs.proc, cs.path = Proc(), str(path)
    out = cs.stop()
    assert out == {"sm_mhz": 2062.5, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 2}
    assert Proc.signals and not path.exists()
    assert bench.ClockSampler(0).stop() is None   # never started (no nvidia-smi): no clocks


def _run_bench(args, env_extra=None, timeout=300):
    import json
    import subprocess
    import sys
    env = dict(os.environ)
    env.update(env_extra or {})
    p = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), *args], capture_output=True, text=True,
                       env=env, timeout=timeout)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(l) for l in p.stdout.splitlines() if l.startswith("{")]
    return lines


def test_reference_arm_prints_one_contract_line():
    """The oracle arm on the host cores: one JSON line with the metric of the
    native arm, the oracle named as the baseline and an end-to-end figure
    equal to the line's own (no host<->device copies)."""
    lines = _run_bench(["--impl", "reference", "--steps", "2", "--warmup", "1"])
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "Mrays/s"
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None and d["scaling"] == "weak"
    assert d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only():
    assert _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"],
                      {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_l2_figures_come_from_the_committed_captures():
    b = bench.l2_record(False)
    assert 0 < b["l2_sector_hit_pct"] <= 100 and 0 < b["l1_sector_hit_pct"] <= 100
    assert 0 < b["l2_throughput_pct_of_peak"] <= 100 and "trace_pair_medium.md" in b["source"]
    w = bench.l2_record(True)
    assert 0 < w["l2_sector_hit_pct"] <= 100 and "trace8_medium.md" in w["source"]


def test_profile_summaries_name_committed_commands():
    """Every ncu summary gives the command that made it: ncu with the clocks
    left alone, run on committed files only."""
    import glob
    import re
    files = sorted(glob.glob(os.path.join(bench.ROOT, "profiles", "*.md")))
    assert len(files) >= 3
    for path in files:
        lines = open(path).read().splitlines()
        cmds = []
        for k, line in enumerate(lines):
            if re.match(r"\s+ncu ", line):
                c = line
                while c.endswith("\\") and k + 1 < len(lines):
                    k += 1
                    c = c[:-1] + lines[k]
                cmds.append(c)
        assert cmds, path
        for c in cmds:
            assert "--clock-control none" in c, (path, c[:80])
            assert "python bench.py" in c and "_work" not in c, (path, c[:80])


def test_large_profile_carries_the_values_the_bench_reads():
    txt = open(os.path.join(bench.ROOT, "profiles", "trace_large.md")).read()
    for key in ("traversal_code_sha256_16:", "dram_bytes_per_closest_launch:", "warp_inst_per_closest_ray:"):
        assert key in txt, key
    rec = bench.traffic_record("trace_large.md", "dram_bytes_per_closest_launch")
    if rec is None:
        pytest.skip("traversal sources changed since the capture (the bench then reports traffic null)")
    # more than the rays read and the hit records written, far less than the counted bytes
    assert (1 << 24) * (32 + 20) < rec < 51.7e9


def test_ray_bytes_counts_ray_hit_nodes_triangles_and_instances():
    cst = {"closest_rays": 10, "node_visits": 30, "tri_tests": 20, "inst_entries": 10,
           "shadow_rays": 5, "any_node_visits": 5, "any_tri_tests": 0, "any_inst_entries": 5}
    assert bench.ray_bytes(cst, 64, False) == 32 + 20 + 64 * 3 + 48 * 2 + 80 * 1
    assert bench.ray_bytes(cst, 80, True) == 32 + 20 + 80 * 1 + 0 + 80 * 1


def test_hit_error_summary_counts_differing_ids_and_relative_errors():
    import numpy as np
    miss = np.uint32(0xFFFFFFFF)
    ref = {"inst": np.array([0, 1, 2, miss], np.uint32), "prim": np.array([5, 6, 7, miss], np.uint32),
           "t": np.array([10.0, 20.0, 30.0, np.inf]), "u": np.array([0.5, 0.0001, 0.2, 0.0]),
           "v": np.array([0.25, 0.5, 0.3, 0.0]), "ambiguous": np.array([False, False, True, False])}
    h = {"inst": np.array([0, 1, 3, miss], np.uint32), "prim": np.array([5, 6, 7, miss], np.uint32),
         "t": np.array([10.0001, 20.0, 31.0, np.inf], np.float32), "u": np.array([0.5, 0.0001 + 1e-9, 0.2, 0.0], np.float32),
         "v": np.array([0.25, 0.5, 0.3, 0.0], np.float32)}
    e = bench.hit_error_vs_oracle(h, ref)
    assert e["rays"] == 4 and e["hits"] == 2 and e["id_differ"] == 1 and e["id_differ_flagged"] == 1
    assert abs(e["t_rel"]["max"] - 1e-5) < 1e-7          # 10.0001 vs 10 (float32 rounding of 10.0001)
    assert e["u_rel"]["max"] < 2e-6                        # 1e-9 against max(1e-4, 1e-3)
