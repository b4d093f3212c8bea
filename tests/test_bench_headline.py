"""bench.py's one stdout line: the contract's keys, the summary ratios, and a size that a
reader keeping only the last few KB of output still sees whole (CPU only)."""
import json
import math

import bench

MiB = 1 << 20


def _study():
    """A study object of the full shape and size (28 sweep rows, 20 host rows, serving,
    batched, windows, Jacobi and lifecycle payloads of realistic length)."""
    sweep = []
    for k, n in enumerate(bench.SIZES):
        sweep.append({"bytes": n, "in_sweep_us": 1.0, "in_sweep_gbs": 100.0 + k, "mode": "graph",
                      "plan": [[2, 65536, n, 2432, 0]], "tuned_vs_best_single": 1.0 + 0.01 * (k % 3),
                      "b2b_tuned_vs_best_single": 0.99, "b2b_gbs": {"x": 1.0, "y": 2.0}})
    host = []
    for k in range(12, 32):
        n = 1 << k
        host.append({"bytes": n, "h2d_tuned_gbs": 210.0, "h2d_best_single_gbs": 200.0,
                     "d2h_tuned_gbs": 190.0, "d2h_best_single_gbs": 190.0, "h2d_plan": [[1, 65536, n]] * 3})
    return {
        "metric": "multi-path GB/s vs best single path by msg size; batched p99 latency", "value": 3241.5,
        "unit": "GB/s", "n_gpus": 1, "steps": 20, "warmup": 5, "ms_per_step": 0.6627, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": bench.workload_config(1),
        "roofline": {"bound": "hbm", "achieved": 6772.0, "peak": 6658.3, "unit": "GB/s", "frac": 1.017,
                     "traffic": 2090000000, "kernel": "k_sm_copy_vec",
                     "launch": "1 GiB message, 2 GiB algorithmic HBM bytes", "launch_ms": 0.3171,
                     "peak_source": "measured hbm_gbs (burst)"},
        "e2e": {"value": 136.0, "unit": "GB/s", "h2d_bytes_per_step": 4294967296, "d2h_bytes_per_step": 4294967296,
                "steps": 10, "pipelined": "2 device arena sets; step k down while step k+1 comes up",
                "link_plans": "ce", "link_chunk_mib": "whole leg"},
        "cpu_baseline": {"value": 12.6, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "13 passes over the 28 sweep sizes 8 B..1 GiB (oracle plan + numpy memcpy, one thread)",
                         "all_cores": {"value": 146.0, "unit": "GB/s", "cores": 16, "sample": "x" * 160}},
        "gpu_launches": 560, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 300},
        "parity_ok": True,
        "batched": {"transfers_per_s": 436000.0, "p99_us": 9200.0, "eager_transfers_per_s": 99900.0,
                    "eager_p99_us": 40600.0, "latency_origin": "host clock before the submitting call",
                    "dma_lanes": [{"x": "y" * 200}] * 3},
        "serving_replay": [{"rate_per_s": r, "seconds": 2.0, "p50_us": 40.0, "p99_us": 300.0, "x": "y" * 300}
                           for r in (1000.0, 10000.0, 50000.0)],
        "copy64MiB_ce_sm_50_50": {"split_vs_best_single": 0.86},
        "host_sweep": {"rows": host, "parity_ok": True},
        "windows": {"rows": [{"dir": "d2d", "gbs": 1.0}] * 96, "parity_ok": True},
        "sweep": sweep, "jacobi": {"x": "y" * 5000}, "graph_lifecycle": [{"x": 1}] * 9,
    }


def test_headline_is_small_and_complete():
    study = _study()
    assert len(json.dumps(study)) > 20000
    line = bench.headline(study, "out/study.json")
    text = json.dumps(line)
    assert len(text) <= bench.HEADLINE_MAX_BYTES, len(text)
    for k in bench.HEADLINE_KEYS:
        assert k in line, k
    assert line["roofline"]["frac"] == 1.017 and line["roofline"]["traffic"] == 2090000000
    assert line["e2e"]["h2d_bytes_per_step"] == 4294967296
    assert line["study"] == "out/study.json"
    assert "sweep" not in line and "host_sweep" not in line
    assert json.loads(text) == line
    assert line["summary"]["serving"]["p99_us"]["50000"] == 300.0
    assert line["cpu_baseline"]["all_cores"] == {"value": 146.0, "cores": 16}
    # the study object itself is left as it was
    assert "sample" in study["cpu_baseline"]["all_cores"] and "pipelined" in study["e2e"]


def test_summary_ratios():
    s = bench.summary_ratios(_study())
    # isolated launches: messages of 4 MiB and more only (2^22 .. 2^30, k = 19 .. 27)
    r = [1.0 + 0.01 * (k % 3) for k, n in enumerate(bench.SIZES) if n >= 4 * MiB]
    assert len(r) == 9
    want = math.exp(sum(math.log(x) for x in r) / len(r))
    d2d = s["d2d_tuned_vs_best_single"]
    assert abs(d2d["isolated_ge4MiB_geomean"] - want) < 1e-4 and d2d["isolated_ge4MiB_min"] == 1.0
    assert d2d["back_to_back_geomean"] == 0.99 and d2d["back_to_back_min"] == 0.99
    # host rows of 64 MiB and more only: 2^26 .. 2^31 (six sizes), 210/200 and 190/190
    assert s["h2d_ge64MiB_tuned_vs_best_single"] == {"geomean": 1.05, "min": 1.05, "max": 1.05}
    assert s["d2h_ge64MiB_tuned_vs_best_single"]["geomean"] == 1.0
    assert s["copy64MiB_split_vs_best_single"] == 0.86
    assert s["batched"]["transfers_per_s_vs_eager"] == round(436000.0 / 99900.0, 3)
    assert s["serving"]["p99_us"] == {"1000": 300.0, "10000": 300.0, "50000": 300.0}
    assert s["windows_parity_ok"] is True


def test_headline_of_a_sparse_study():
    line = bench.headline({"metric": "m", "value": 1.0, "unit": "GB/s"})
    assert line == {"metric": "m", "value": 1.0, "unit": "GB/s", "summary": {}}


def test_fair_share_finish_times_by_hand():
    """The serving bound's processor-sharing server against cases worked by hand: a job alone
    takes its work; two jobs arriving together share the rate (works 1 and 2 finish at 2 and
    3); a job arriving while another is half done (works 2 at t=0 and 1 at t=1: from t=1 both
    run at half rate, the second finishes at 3, the first's last 0 at 3 too); and a job that
    arrives after the server emptied starts afresh."""
    assert bench._fair_share_finish([5.0], [2.0]) == [7.0]
    assert bench._fair_share_finish([0.0, 0.0], [1.0, 2.0]) == [2.0, 3.0]
    f = bench._fair_share_finish([0.0, 1.0], [2.0, 1.0])
    assert abs(f[0] - 3.0) < 1e-12 and abs(f[1] - 3.0) < 1e-12
    f = bench._fair_share_finish([0.0, 1.0, 10.0], [0.5, 4.0, 1.0])
    assert f == [0.5, 5.0, 11.0]


def test_serving_bounds_orders_and_alone_case():
    """No-queue and fair-share references: with one request they agree with fixed cost plus
    bytes at the rate; fair sharing never beats running alone."""
    one = [(0.0, 2 << 20, 1)]
    b = bench.serving_bounds(one, 10.0, 20.0, link_gbs=(200.0, 100.0), dev_gbs=1000.0)
    want = 20.0 + (2 << 20) / 200e3
    assert abs(b["no_queue_p99_us"] - round(want, 1)) < 1e-9 and abs(b["fair_share_p99_us"] - round(want, 1)) < 1e-9
    import payload
    sched = payload.serving_schedule(50000, 0.2)
    b = bench.serving_bounds(sched, 14.0, 16.0)
    assert b["fair_share_p99_us"] >= b["no_queue_p99_us"] and b["fair_share_p50_us"] >= b["no_queue_p50_us"]
