"""Host-side pieces of the benchmark on CPU: the workload meshes, and the
reference arm's JSON line (the CPU oracle timed on a bounded sample of the
GPU arm's workload, whose configuration the line carries)."""
import argparse
import contextlib
import io
import json

import numpy as np
import pytest

import bench
from paper_2208_11630_gb300 import inputs


@pytest.mark.parametrize("name,scale", [("sod2d", 4), ("kh3d", 2), ("sedov_amr", 2),
                                        ("advection3d", 2)])
def test_workload_mesh_is_the_workload_mesh(name, scale):
    m = inputs.workload_mesh(name, scale)
    w, W, gamma, cfl = inputs.workload(name, scale)
    assert np.array_equal(m.level, w.level) and np.array_equal(m.origin, w.origin)
    assert np.array_equal(m.parent, w.parent) and W.shape == w.shape
    assert name in bench.REFERENCE_SAMPLE_SCALE


def test_reference_arm_line():
    args = argparse.Namespace(workload="sod2d", scale=None, precision="f64", steps=2, warmup=3,
                              gpus=1)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(args) == 0
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    full = inputs.workload_mesh("sod2d")
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["config"]["workload"] == bench.workload_name("sod2d", full)
    assert line["config"]["cells"] == full.leaf_zones()
    sample = inputs.workload_mesh("sod2d", bench.REFERENCE_SAMPLE_SCALE["sod2d"])
    assert line["config"]["ran"]["cells"] == sample.leaf_zones()   # what the oracle stepped
    assert line["config"]["ran"]["sample_of"] == line["config"]["workload"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_cpu_baseline_all_cores_and_one_thread():
    import oracle
    before = oracle.get_threads()
    cb = bench.oracle_sample("sod2d", target_s=0.05, max_steps=2, single_s=0.05)
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] == before
    one = cb["single_thread"]
    assert one["cores"] == 1 and one["value"] > 0 and one["unit"] == bench.UNIT
    assert oracle.get_threads() == before   # the thread count is restored


def test_reference_arm_other_ranks_do_no_work(monkeypatch):
    """Under torchrun only rank 0 times the oracle and prints; the others
    exit 0 without work or output."""
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = argparse.Namespace(workload="kh3d", scale=None, precision="f64", steps=2, warmup=3,
                              gpus=2)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(args) == 0
    assert buf.getvalue() == ""
