"""The benchmark's output contract, checked on the CPU through its reference arm (the oracle on
host cores): one JSON line with the contract's keys, the GPU arm's config, and a CPU baseline
that names what it timed.  The GPU arm itself needs a GB300 and runs in the GPU job."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2", "--warmup", "1",
         "--ref-rows", "2048"],
        capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["value"] > 0
    bench = _bench_module()
    assert d["metric"] == bench.METRIC
    assert d["config"] == bench.main_config(bench.M_DEFAULT, bench.N_DEFAULT, 0, 1)  # the GPU arm's config
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert "Q^T b" in cb["sample"] and "2048 rows" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_flop_counts_and_job_value():
    """The metric's flop counts are the LAPACK ones (factor and thin Q 2mn^2 - 2n^3/3 each, Q^T b
    4mn - 2n^2) and the job value sums the ranks' work over the slowest rank's time."""
    bench = _bench_module()
    m, n = 1 << 22, 64
    f = bench.flops(m, n)
    assert f["factor"] == 2.0 * m * n * n - 2.0 * n ** 3 / 3
    assert f["form_q"] == f["factor"]
    assert f["apply_qt"] == 4.0 * m * n - 2.0 * n * n
    per = sum(f.values())
    assert abs(bench.job_value(per, 4, 100.0) - 4 * per / 0.1 / 1e9) <= 1e-9 * bench.job_value(per, 4, 100.0)


def test_host_cpu_names_the_processor():
    h = _bench_module().host_cpu()
    assert isinstance(h["model"], str) and h["model"]
    assert h["cpu_count"] == os.cpu_count()


def test_usv_family_equals_usv():
    """The benchmark's conditioning grid draws U and V once for all kappa; each matrix must be the
    one usv() draws for that kappa, bit for bit."""
    import numpy as np

    from paper_0809_2407_gb300 import inputs

    ks = (0.0, 4.0, 12.0)
    fam = inputs.usv_family(500, 12, ks, 31)
    for k, A in zip(ks, fam):
        assert np.array_equal(A, inputs.usv(500, 12, k, 31))
