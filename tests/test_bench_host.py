"""Host-side logic of bench.py and of the workload recipes, on CPU: which
kernel each workload runs on, the algorithmic figures its roofline uses, the
lookup of recorded DRAM traffic, and the bounds that keep the bench short."""
import json
import os

import pytest

import bench
import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_workload_recipes_have_the_stated_sizes_and_time_steps():
    sizes = {"b1_hedgehog_48": 48, "b4_cubic_128": 128, "b4_sextic_128": 128,
             "b4_lightly_bound_128": 128, "b8_cluster_256": 256, "b32_cluster_512": 512}
    for name, n in sizes.items():
        wl = workloads.ALL[name]()
        assert wl.n == (n, n, n) and wl.interior_sites == (n - 4) ** 3
        # dt = 0.05 h (the largest stable Courant number), 0.025 h for the dense 512^3 cluster
        courant = 0.025 if name == "b32_cluster_512" else workloads.COURANT
        assert wl.dt == pytest.approx(courant * wl.h)
    sides = [w.n[0] for w in workloads.batched_noise(count=64, steps=10)]
    assert len(sides) == 64 and set(sides) <= {64, 80, 96, 112, 128}


def test_each_workload_runs_on_the_kernel_its_model_needs():
    std, pot, sext = (workloads.ALL[k]() for k in
                      ("b4_cubic_128", "b4_lightly_bound_128", "b4_sextic_128"))
    assert not std.extended and pot.extended and sext.extended
    assert std.streaming and pot.streaming and sext.streaming
    assert bench.step_kernel_key(std, 32) == "step_f32_b4_cubic_128"
    assert bench.step_kernel_key(pot, 32) == "step_f32_b4_lightly_bound_128"
    assert bench.step_kernel_key(sext, 32) == "step_f32_b4_sextic_128"
    assert bench.step_kernel_key(std, 64) == "step_f64_b4_cubic_128"
    assert bench.step_kernel_key(pot, 64) == "step_tile_f64_b4_lightly_bound_128"
    assert bench.flops_per_site(std) == bench.FLOPS_PER_SITE
    assert bench.flops_per_site(pot) == bench.FLOPS_PER_SITE_POT
    assert bench.flops_per_site(sext) == bench.FLOPS_PER_SITE_EXT
    assert bench.FLOPS_PER_SITE < bench.FLOPS_PER_SITE_POT < bench.FLOPS_PER_SITE_EXT


def test_recorded_traffic_is_keyed_by_source_and_scaled_by_sites(tmp_path, monkeypatch):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        table = json.load(f)
    for key, rec in table.items():
        if key.startswith("_"):
            continue
        assert rec["dram_bytes_per_launch"] > 0 and rec["sites"] > 0 and rec["source"]
    # a record of the current sources scales with the sites; another fingerprint reads as unknown
    key = "step_f32_b4_cubic_128"
    fake = {key: {"fingerprint": bench.kernel_fingerprint(key), "sites": 1000,
                  "dram_bytes_per_launch": 64000.0, "source": "test"},
            "step_f64_b1_hedgehog_48": {"fingerprint": "0" * 16, "sites": 10,
                                        "dram_bytes_per_launch": 1.0, "source": "test"}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(fake))
    real = {k: bench.kernel_fingerprint(k) for k in fake}
    monkeypatch.setattr(bench, "kernel_fingerprint", lambda k: real.get(k, "f" * 16))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic(key, 2000) == pytest.approx(128000.0)
    assert bench.recorded_traffic("step_f64_b1_hedgehog_48", 10) is None
    assert bench.recorded_traffic("step_f32_no_such_workload", 10) is None


def test_kernel_fingerprints_follow_the_kernel_sources():
    f32 = bench.kernel_fingerprint("step_f32_b4_cubic_128")
    assert f32 == bench.kernel_fingerprint("step_f32_b8_cluster_256")
    tile = bench.kernel_fingerprint("step_tile_f32_b4_sextic_128")
    assert tile == bench.kernel_fingerprint("step_f64_b1_hedgehog_48") and tile != f32
    assert len(f32) == 16 and int(f32, 16) >= 0


def test_run_to_tolerance_leg_is_bounded():
    # the default workload is relaxed; the 256^3 and 512^3 ones are skipped
    assert workloads.b4_cubic_128().interior_sites <= bench.UNTIL_MAX_SITES
    assert workloads.b8_cluster_256().interior_sites > bench.UNTIL_MAX_SITES
    out = bench.run_variants(None, None, None, workloads.b32_cluster_512(), 6778.0)
    assert set(out) == {"skipped"}
    # at the measured rates the capped relaxations end within a minute
    assert bench.UNTIL_MAX_STEPS[32] * 60e-6 < 5 and bench.UNTIL_MAX_STEPS[64] * 1.7e-3 < 15


def test_workload_config_names_the_workload_and_the_l2_rule():
    cfg = bench.workload_config(workloads.b4_cubic_128())
    assert cfg["workload"] == "b4_cubic_128" and cfg["lattice"] == [128, 128, 128]
    assert "larger than L2" in cfg["l2"]
    cfg = bench.workload_config(workloads.b4_lightly_bound_128())
    assert cfg["m_w"] == 1.0 and cfg["c6"] == 0.0
    assert "smaller than L2" in bench.l2_note(workloads.b1_hedgehog_48())


def test_fingerprints_ignore_comments_and_layout_but_not_code():
    code = "int f(int a) {\n    return a + 1;  // one more\n}\n"
    assert bench.source_code_only(code) == bench.source_code_only(
        "/* a block\n comment */ int f(int a)\n{ return a + 1; }")
    assert bench.source_code_only(code) != bench.source_code_only(code.replace("+ 1", "+ 2"))


def test_a_smaller_batch_is_the_head_of_the_batched_recipe():
    """`bench.py --batched-only COUNT` (a batch for profiling) runs the first
    COUNT lattices of the 64-lattice recipe, so its profile describes the
    same size mix."""
    head = [(w.n, w.seed, w.dt) for w in workloads.batched_noise(count=16, steps=200)]
    full = [(w.n, w.seed, w.dt) for w in workloads.batched_noise(count=64, steps=200)]
    assert head == full[:16]
