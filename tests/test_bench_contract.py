"""The JSON line bench.py prints: every key the benchmark contract names, with consistent
values. The reference arm (the FP64 oracle on the host cores) runs on the CPU; our arm
runs on the GPU at a small size with the extras and the CPU leg skipped."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
             "scaling", "vs_baseline", "dtype", "data", "config")


def _run(*args, timeout=600):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                       text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def _check_base(d, steps, warmup):
    for k in BASE_KEYS:
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["steps"] == steps and d["warmup"] == warmup and d["n_gpus"] == 1
    assert d["scaling"] == "weak" and d["vs_baseline"] is None and d["data"] == "synthetic"
    assert "workload" in d["config"]
    cpu = d["cpu_baseline"]
    if cpu is not None:
        assert cpu["kind"] == "oracle" and cpu["unit"] == "MLUPS" and cpu["cores"] >= 1 and cpu["sample"]
    e2e = d["e2e"]
    if e2e is not None:
        for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
            assert k in e2e, k


def test_reference_arm_line():
    d = _run("--impl", "reference", "--steps", "3", "--warmup", "1", "--n", "32")
    _check_base(d, 3, 1)
    assert d["impl"] == "reference" and d["dtype"] == "f64"
    assert d["cpu_baseline"]["value"] == d["value"]
    # one timed step = one oracle step on the named slab: the line's time is the time spent
    slab = d["config"]["slab_cells"]
    assert d["value"] == pytest.approx(slab / (d["ms_per_step"] * 1e-3) / 1e6)
    assert d["ms_per_step"] * 1e-3 * d["steps"] <= 3.0 * d["cpu_baseline"]["seconds"]
    assert "z-slab" in d["config"]["workload"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.gpu
def test_our_arm_line_at_64cube():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = _run("--n", "64", "--steps", "4", "--warmup", "3", "--no-cpu", "--no-extras", "--forms", "mixed,bgk_f32")
    _check_base(d, 4, 3)
    roof = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in roof, k
    # the NCO is bound by the tensor roof: achieved = algorithmic flops per launch / the step time
    assert roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s"
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert roof["achieved"] == pytest.approx(47920 * 64 ** 3 / (d["ms_per_step"] * 1e-3) / 1e12, rel=1e-6)
    # and its HBM view: algorithmic bytes per launch / the step time
    hbm = roof["hbm"]
    assert hbm["achieved"] == pytest.approx(108 * 64 ** 3 / (d["ms_per_step"] * 1e-3) / 1e9, rel=1e-6)
    assert hbm["frac"] == pytest.approx(hbm["achieved"] / hbm["peak"])
    assert d["gpu_launches"] == d["steps"]
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    assert d["e2e"]["value"] > 0 and d["e2e"]["d2h_bytes_per_step"] == 8
    assert d["forms"]["mixed"]["mlups"] == pytest.approx(d["value"])
