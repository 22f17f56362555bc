"""The bench's default-line records on the CPU: the compact records of the
batched, differentiable and serving workloads keep the figures the line must
carry (value, per-step time, roofline with kernel and traffic, clocks,
accuracy against the oracle, the workload's own comparison) and drop the rest;
the three workloads run with bounded settings and their own autotuning; the
DRAM traffic the line declares stays within its kernels' algorithmic bytes.
No GPU is needed."""
import argparse

import bench


def _full(workload, **extra):
    r = {"metric": "m", "value": 1.0, "unit": "u", "n_gpus": 1, "steps": 5, "warmup": 3,
         "ms_per_step": 2.0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
         "dtype": "f32", "data": "synthetic", "config": {"workload": workload, "x": 1},
         "roofline": {"bound": "hbm", "achieved": 1.0, "peak": 2.0, "unit": "GB/s",
                      "frac": 0.5, "traffic": 3.0, "kernel": "k"},
         "clocks": {"sm_mhz": 2070.0, "reasons": []}, "gpu_launches": 7, "peaks": "measured"}
    r.update(extra)
    return r


def test_compact_record_keeps_the_line_figures():
    acc = {"rel_l2": 1e-7, "max_abs_over_peak": 1e-7}
    full = _full("batched_uneven_512src",
                 vs_per_source={"ratio": 1.6}, autotune={"64": {"mac_staging": 2}},
                 cpu_baseline={"value": 5.0, "unit": "u", "cores": 16, "kind": "oracle",
                               "sample": "s", "seconds": 2.0, "accuracy": acc})
    c = bench.compact_record("batched", full, 8.25)
    assert c["workload"] == "batched_uneven_512src"
    for k in ("metric", "value", "unit", "ms_per_step", "roofline", "clocks", "gpu_launches",
              "vs_per_source", "autotune", "accuracy", "cpu_baseline"):
        assert k in c, k
    assert c["accuracy"] == acc and c["roofline"]["traffic"] == 3.0
    assert set(c["cpu_baseline"]) == {"value", "unit", "cores", "sample"}
    assert "config" not in c and "peaks" not in c and "data" not in c
    assert abs(c["wall_s"] - 8.25) <= 0.051          # rounded to 0.1 s


def test_compact_record_of_the_differentiable_and_serving_workloads():
    grad = {"dP_max_abs_over_peak": 1e-8, "dx_rel_l2": 1e-7}
    c = bench.compact_record("adjoint", _full("differentiable_16ch", gradient_accuracy=grad,
                                              segmented_k32_ms_per_step=2.1), 1.0)
    assert c["accuracy"] == grad and c["segmented_k32_ms_per_step"] == 2.1
    lat = {"ticks": 2000, "host_to_host_ms_p99": 0.2, "missed_deadline": 0}
    streams = {"dropped": 0, "live_during_latency": {"min": 1000}}
    c = bench.compact_record("serve", _full("serving_1000_streams", latency=lat, streams=streams,
                                            stages_ms_per_tick={"mac": 0.1}), 1.0)
    assert c["latency"] == lat and c["streams"] == streams and "stages_ms_per_tick" in c


def test_subrecords_are_bounded(monkeypatch):
    seen = {}

    def fake(name):
        def run(a):
            seen[name] = (a.steps, a.warmup, a.serve_ticks, a.staging)
            return _full(name)
        return run

    for name, fn, _ in bench.SUBRECORD_RUNS:
        monkeypatch.setattr(bench, fn, fake(name))

    class _Cuda:
        @staticmethod
        def empty_cache():
            pass

    import torch
    monkeypatch.setattr(torch, "cuda", _Cuda)
    args = argparse.Namespace(steps=20, warmup=5, serve_ticks=10000, staging=1)
    out = bench.workload_subrecords(args)
    assert set(out) == {"batched", "adjoint", "serve"}
    assert seen["batched"][:2] == (5, 3) and seen["adjoint"][:2] == (5, 3)
    assert seen["serve"][2] == 2000
    assert all(v[3] is None for v in seen.values())      # the autotuner, not a fixed staging
    assert args.steps == 20 and args.staging == 1         # the caller's settings are untouched


def test_declared_dram_traffic_is_within_the_algorithmic_bytes():
    """The DRAM bytes the default line declares for the multiply-accumulate
    (scaled from an ncu capture at 32 channels) stay within the bytes its
    launch must move at least once: X read, the bank read and Y written,
    each once. Traffic above them would mean re-reads; far below, a capture of
    the wrong kernel or size. The same for the fused adjoint (P read, dP
    written)."""
    from synth import workloads as W
    ch, L, M, n_ir = 64, 256, 94, 8
    P = 2 * L
    nb = W.blocks_for(480000, L)
    algo = 2 * ch * nb * P * 8 + ch * n_ir * M * P * 8
    assert 0.8 * algo < bench.MAC_TRAFFIC_BYTES <= algo
    # differentiable workload: 16 channels, 240000 samples, M = 47
    nb16 = W.blocks_for(240000, L)
    params = 16 * nb16 * 47 * P * 8
    assert 0.8 * 2 * params < bench.ADJ_TRAFFIC_BYTES <= 2 * params
