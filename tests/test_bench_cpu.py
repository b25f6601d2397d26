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


def test_launches_per_step_matches_the_launch_lists():
    """gpu_launches counts the kernels of a step as the committed ncu launch lists show them at
    m = 2^22, n = 64 (leaf height 96, 43691 leaves, 304 chains, 9 tree levels): FP64 12 (factor,
    9 tree levels, thin-Q chains, Q^T b), the Ozaki form 14 (three thin-Q chain kernels), FP32
    storage 15 (also the widening of A)."""
    bench = _bench_module()
    full = dict(np_=64, leaf_h=96, leaves=43691, chains=304)
    assert bench.launches_per_step(1, 9, 0, False, **full) == 12
    assert bench.launches_per_step(1, 9, 1, False, **full) == 12
    assert bench.launches_per_step(1, 9, 2, False, **full) == 14
    assert bench.launches_per_step(1, 9, 3, False, **full) == 14
    assert bench.launches_per_step(1, 9, 0, True, **full) == 15
    # every leaf starts a chain: no leaf-products launch; padded width 32: the one chain kernel
    assert bench.launches_per_step(1, 4, 2, False, np_=64, leaf_h=96, leaves=16, chains=16) == 8
    assert bench.launches_per_step(1, 9, 2, False, np_=32, leaf_h=256, leaves=16384, chains=304) == 12
