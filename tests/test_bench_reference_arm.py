"""The reference arm of bench.py (the oracle timed on the host) prints one
JSON line with the contract keys, on a bounded sample (k = 2 only); the GPU
arm's contract line, built from stub timings, has its keys and stays a few
KB; and the batched leg runs the variants its options ask for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_reference_arm_prints_contract_line():
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "0", "--ks", "2"], capture_output=True, text=True, timeout=600, env=env)
    assert res.returncode == 0, res.stderr[-2000:]
    line = json.loads(res.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "dtype", "config", "cpu_baseline", "e2e"]:
        assert key in line
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    # the timed interval is real: steps x ms_per_step fits in the run
    assert line["steps"] * line["ms_per_step"] < 600e3
    assert line["full_step_estimate_ms"] > line["ms_per_step"]


def test_headline_line_keys_and_size():
    import bench
    per_k = {str(k): {"dofs_per_s": 1e9, "ms_per_call": 10.0, "tflops": 1.2, "frac_fp64_peak": 0.95}
             for k in bench.KS}
    roofline = {"bound": "alu", "kernel": "patch_smooth_kernel<3,16,vertex,double> (k=7)", "achieved": 1.2,
                "peak": 1.2586, "unit": "TFLOP/s", "frac": 0.95, "peak_source": "derived", "per": "one call",
                "traffic": 3.1e10, "traffic_unit": "bytes per call", "algorithmic_bytes": 2.1e9}
    e2e = {"value": 9e8, "unit": "DoF/s", "h2d_bytes_per_step": 1, "d2h_bytes_per_step": 1, "note": "x"}
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 10, "reasons": []}
    cpu = {"value": 1e6, "unit": "DoF/s", "cores": 16, "kind": "oracle", "sample": "s" * 300, "timed_s": 3.0,
           "full_step_estimate_ms": 2.4e4, "nproc": 16, "cpu_model": "Neoverse-V2",
           "per_degree_s": {str(k): 0.5 for k in bench.KS},
           "one_core": {"value": 1e5, "degrees": [2, 3, 4], "cores": 1, "all_cores_same_degrees": 1e6},
           "dense_lu_one_core": {"value": 5e3, "degree": 2, "sample": "24 random vertex patches"}}
    line = bench.headline_line(9.6e8, 350.0, 1, 20, 5, roofline, e2e, clocks, per_k, cpu, 960)
    text = json.dumps(line)
    assert len(text) < 6000
    for key in ["impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "dtype", "config", "roofline", "cpu_baseline", "e2e", "clocks", "per_degree",
                "gpu_launches"]:
        assert key in line
    assert line["impl"] == "tpss" and line["roofline"]["algorithmic_bytes"] > 0
    failed = bench.headline_line(9.6e8, 350.0, 1, 20, 5, roofline, e2e, clocks, per_k, {"error": "boom"}, 960)
    assert failed["cpu_baseline"]["value"] is None and "boom" in failed["cpu_baseline"]["sample"]


def test_batched_leg_variants_with_stub_runs():
    # the batched leg's composition (which variants run, the speedup keys)
    # with the GPU parts replaced by stubs
    import contextlib
    import types
    import bench
    from paper_1910_11239_gb300 import workloads

    class Event:
        def __init__(self, enable_timing=False):
            pass

        def record(self, stream=None):
            pass

        def elapsed_time(self, other):
            return 10.0

    class Tensor:
        def __init__(self, a):
            self.a = a

        def to(self, *args, **kwargs):
            return self

    cuda = types.SimpleNamespace(Stream=lambda: None, stream=lambda s: contextlib.nullcontext(), Event=Event,
                                 synchronize=lambda: None)
    torch_stub = types.SimpleNamespace(cuda=cuda, from_numpy=Tensor, empty_like=lambda t: t)

    class Problem:
        def __init__(self, *args, **kwargs):
            pass

        def mg_setup(self, *args, **kwargs):
            pass

        def ndofs(self, level):
            return 10

        def pcg_solve(self, *args, **kwargs):
            return {"iters": 40}

        def close(self):
            pass

    tpss_stub = types.SimpleNamespace(Problem=Problem, FP64=0)
    calls = []

    def one(tpss, wl, torch, steps, prec, columns=True):
        calls.append((prec, columns))
        return {"pcg": {"time_s": 2.0}}

    saved = bench.run_batch_one
    bench.run_batch_one = one
    try:
        out = bench.run_batch(tpss_stub, workloads, None, torch_stub, 3)
        assert calls == [("bf16", True), ("fp32", True)]
        assert set(out) == {"workload", "bf16", "fp32", "one_at_a_time_fp64"}
        calls.clear()
        out = bench.run_batch(tpss_stub, workloads, None, torch_stub, 3, True)
        assert calls == [("bf16", True), ("bf16", False), ("fp32", True)]
        for key in ("bf16", "bf16_persistent", "fp32"):
            assert out[key]["speedup_time_to_solution_vs_fp64_one_at_a_time"] > 0
    finally:
        bench.run_batch_one = saved
