"""Host-side pieces of bench.py that need no GPU: the CPU-oracle baseline
(its one-thread child process) and the algorithmic work models behind the
roofline figures."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_oracle_sample_child_prints_one_json_line():
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-sample", "1"],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["n"] == 2 and d["dt"] > 0


def test_work_models_scale_with_iterations_and_batch():
    import bench
    ps = bench.workload(2, 0)
    outs = [{"iters": 10, "M": 128, "D": 20} if p.is_box else {"iters": 0} for p in ps]
    w1 = bench.fp64_flops_per_step(ps, outs)
    for o in outs:
        if "M" in o:
            o["iters"] = 20
    w2 = bench.fp64_flops_per_step(ps, outs)
    assert set(w1) >= {"k_rr", "k_gemm_tn", "k_gemm_nn", "k_band_solve", "k_fft", "k_fblocks_eig"}
    for k in ("k_rr", "k_gemm_tn", "k_gemm_nn", "k_band_solve", "k_fft"):
        assert w2[k] > w1[k]
    assert w2["k_fblocks_eig"] == w1["k_fblocks_eig"]           # periodic work has no iterations
    w4 = bench.fp64_flops_per_step(ps + ps, outs + outs)
    for k in w2:
        assert np.isclose(w4[k], 2 * w2[k])
    # the band solve model: 4 L (D+1) m0^2 kb flops per application
    box = ps[0]
    kb = box.k_eig + max(4, box.k_eig // 8)
    one = bench.fp64_flops_per_step([box], [{"iters": 1, "M": 128, "D": 20}])
    assert one["k_band_solve"] == 4 * box.L[0] * 21 * 64 * kb


def test_latency_summary_per_kind():
    import bench
    lat = [1.0, 2.0, 3.0, 100.0, 200.0]
    kind = [False, False, False, True, True]
    s = bench.latency_summary(lat, kind)
    assert s["p50_ms"] == 3.0 and s["p50_ms_periodic"] == 2.0 and s["p50_ms_structured"] == 150.0
    assert s["n_periodic"] == 3 and s["n_structured"] == 2
    only = bench.latency_summary([5.0, 7.0], [False, False])
    assert "p50_ms_structured" not in only and only["p99_ms_periodic"] == np.percentile([5.0, 7.0], 99)


def test_poll_all_deadline():
    import time

    import bench

    class Srv:
        def __init__(self, ready):
            self.ready = ready

        def poll(self, t, timeout_ms):
            return {"t": t} if t in self.ready else None

    assert bench._poll_all(Srv({1, 2}), [1, 2], time.perf_counter() + 5) == [{"t": 1}, {"t": 2}]
    import pytest
    with pytest.raises(TimeoutError):
        bench._poll_all(Srv({1}), [1, 2], time.perf_counter() + 0.01)
