"""The host-side arms of bench.py on CPU: the reference arm's JSON line and
its bounded sample, and the oracle baseline that rides on the GPU line."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1805_01443_gb300 import inputs  # noqa: E402


class Args:
    steps = 2
    warmup = 1


def test_reference_sample_keeps_the_full_mesh_when_it_fits():
    import bench
    cfg = inputs.disc_planet_512()
    got, note = bench.reference_sample(cfg, 100, 0.5)
    assert got is cfg
    assert "512x512" in note


def test_reference_sample_shrinks_to_the_budget():
    import bench
    cfg = inputs.disc_planet_512()
    got, note = bench.reference_sample(cfg, 1000, 0.5)  # 500 s of full steps against 120 s
    assert got is not cfg and cfg["mesh"]["nx"] == 512  # the caller's configuration stays
    n = got["mesh"]["nx"]
    assert n == got["mesh"]["ny"] and n % 2 == 0
    assert (n / 512) ** 2 * 500 <= 120 < ((n + 2) / 512) ** 2 * 500
    assert got["order"] == cfg["order"] and got["mesh"]["x0"] == cfg["mesh"]["x0"]
    assert "%dx%d" % (n, n) in note


def test_reference_sample_never_grows_a_small_mesh():
    import bench
    cfg = inputs.disc_planet(16, 2)
    got, _ = bench.reference_sample(cfg, 10 ** 6, 1.0)
    assert got is cfg


def test_reference_arm_line(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    cfg = inputs.disc_planet(16, 2)
    assert bench.run_reference(Args(), cfg) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT and line["higher_is_better"]
    assert line["steps"] == 2 and line["value"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert "16x16" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_takes_the_coarse_sample_over_budget(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    cfg = inputs.disc_planet(80, 1)
    assert bench.run_reference(Args(), cfg, budget_s=0.0) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert "64x64" in line["cpu_baseline"]["sample"] and line["value"] > 0


def test_cpu_baseline_sample_fields():
    import bench
    import oracle
    cfg = inputs.disc_planet(16, 2)
    cb = bench.cpu_baseline_sample(cfg, seconds=0.05)
    assert cb["kind"] == "oracle" and cb["unit"] == bench.UNIT and cb["value"] > 0
    assert cb["cores"] == oracle.nthreads()
    assert cb["one_core"]["cores"] == 1 and cb["one_core"]["value"] > 0
    assert oracle.nthreads() == cb["cores"]  # the thread count is restored
    assert "16x16" in cb["sample"]


def test_clock_summary_reads_the_median_and_the_throttle_reasons():
    """The clocks record of the bench line: the median SM clock of the samples
    taken under load, the maximum clock, and every throttle reason seen Active
    (nvidia-smi csv,noheader,nounits lines in the sampler's field order)."""
    import bench
    c = bench.ClockSampler(0)
    c.lines = [
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines = ["0, 1200, 2070, 300, 0x8, Active, Not Active, Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.lines = []
    assert c.summary()["reasons"] == ["unsampled"]


def test_design_bytes_count_the_static_data_apart_from_the_algorithmic_bytes():
    """800 B per element and stage launch is the algorithmic figure (FP32 state:
    reads of delta^(s) and delta^n, one write, averaged over the three stages);
    the design bytes add R_b where it is kept, the background averages and the
    damping offsets of the zone tiles, all from the handle's tile counts."""
    import bench
    assert bench.BYTES_PER_ELEM_STAGE_PREC == (2 + 3 + 3) / 3 * 75 * 4
    assert bench.design_bytes(100, 0, 0) == 800.0 + 12.0 / 3.0
    assert bench.design_bytes(100, 100, 100) == 800.0 + 300.0 + (12.0 + 300.0) / 3.0
    assert 800.0 < bench.design_bytes(8192, 782, 4380) < 900.0
