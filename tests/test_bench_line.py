"""The benchmark's headline record: one short JSON line that a log tail still holds whole."""
import json

import bench


def _line(extra_serving: int = 0) -> dict:
    return {
        "metric": bench.METRIC, "value": 3.861234567e10, "unit": "trees/s", "n_gpus": 1, "steps": 20, "warmup": 5,
        "ms_per_step": 1.32512345, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "points_per_s": 386400.123456,
        "config": {"workload": "sin_2d: " + "x" * 120, "points": 512, "trees_per_point": 100000, "K": 10},
        "roofline": {"bound": "alu", "achieved": 10.55123456, "peak": 40.2712345, "unit": "Tinst/s",
                     "frac": 0.262123456, "traffic": 203612345, "graph_ms_per_step": 1.3181234},
        "e2e": {"value": 3.73e10, "unit": "trees/s", "h2d_bytes_per_step": 12288, "d2h_bytes_per_step": 6144},
        "gpu_launches": 40, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []},
        "workloads_trees_per_s": {"uneven_2d": 3.27e10, "pdd_3d": 2.72e10},
        "pdd_3d_pipeline_ms": {"point_solves": 63.6, "pdd_stage": 7.6},
        "serving": {"p50_ms": 4.8, "p99_ms": 285.0, "note": "y" * extra_serving,
                    "at_configured_rate": {"p50_ms": 13.7, "p99_ms": 1920.0, "points_per_s": 1.2e5}},
        "cpu_baseline": {"value": 8.19e7, "unit": "trees/s", "cores": 16, "kind": "oracle", "sample": "z" * 60},
    }


def test_headline_is_one_short_parseable_line():
    text = bench.headline_json(_line())
    assert "\n" not in text and len(text) <= bench.HEADLINE_MAX_BYTES
    d = json.loads(text)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "roofline", "e2e", "clocks", "cpu_baseline", "gpu_launches", "config"):
        assert key in d
    assert d["value"] == 3.8612e10 and d["roofline"]["frac"] == 0.26212
    assert d["serving"]["at_configured_rate"]["p99_ms"] == 1920.0


def test_optional_keys_go_before_the_required_ones():
    text = bench.headline_json(_line(extra_serving=2000))
    d = json.loads(text)
    assert len(text) <= bench.HEADLINE_MAX_BYTES
    assert "serving" not in d and "workloads_trees_per_s" not in d
    assert d["roofline"]["frac"] == 0.26212 and d["cpu_baseline"]["cores"] == 16
