"""Host-side helpers of bench.py: the code digest that decides whether the
recorded DRAM traffic still describes the kernel."""
import bench


def test_code_only_ignores_comments_and_whitespace():
    a = "int f(int x) {  // add one\n  return x + 1; /* done */\n}\n"
    b = "/* header */\nint f(int x) {\n\treturn x + 1;\n}  // changed comment\n"
    assert bench.code_only(a) == bench.code_only(b) == "int f(int x) { return x + 1; }"


def test_code_only_sees_code_changes_and_keeps_literals():
    a = 'const char *p = "a // b /* c */"; char q = \'"\'; int k = 2;'
    assert bench.code_only(a) == a
    assert bench.code_only(a) != bench.code_only(a.replace("k = 2", "k = 3"))
    # a block comment separates tokens like whitespace does
    assert bench.code_only("int/**/x;") == "int x;"


def test_traffic_only_for_the_captured_workload():
    assert bench.measured_traffic("rmat18", 10000) is None
    assert bench.measured_traffic("rmat20", 1000) is None


def test_batched_cpu_baseline_runs_the_oracle_on_every_instance_in_parallel():
    import oracle
    from paper_2511_01235_gb300 import workloads as W
    gs = [W.erdos_renyi(300 + 50 * k, 2000, seed=900 + k, cap_hi=50) for k in range(6)]
    rate, threads, vals = bench.cpu_baseline_batched(gs)
    assert rate > 0 and threads >= 1
    assert vals == [oracle.maxflow(g.n, g.src, g.dst, g.cap, g.s, g.t).value for g in gs]


def test_roofline_nominal_peak_is_the_parts_bandwidth():
    assert bench.HBM_NOMINAL_GBS == 7900.0 and bench.HBM_FALLBACK_GBS < bench.HBM_NOMINAL_GBS


def test_cpu_baseline_sample_is_bounded_by_its_budget():
    import numpy as np
    from paper_2511_01235_gb300 import workloads as W
    g = W.erdos_renyi(300, 2000, seed=31, cap_hi=50)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(32)
    batches = []
    for _ in range(4):
        b = W.mixed_batch(es, 50, rng, ins_cap_hi=50)
        es.apply(b.u, b.v, b.cap)
        batches.append(b)
    assert len(bench.cpu_baseline_sample(g, batches, budget_s=0.0)) == 1       # stops after the first batch
    times = bench.cpu_baseline_sample(g, batches, budget_s=60.0)
    assert len(times) == 4 and all(t > 0 for t in times)


def test_serving_service_time_follows_the_timed_sizes():
    """The offered load of the serving run: a calibration of small requests
    scales up to the timed requests' mean size; a calibration of large ones
    keeps its own per-request mean."""
    import bench
    per_req, svc = bench.service_time(0.1, [1000] * 10, [5000, 15000])      # 10 ms per 1 K updates
    assert abs(per_req - 0.01) < 1e-12 and abs(svc - 0.1) < 1e-12          # 10 K mean size -> 100 ms
    per_req, svc = bench.service_time(1.0, [50000] * 10, [10, 30])
    assert abs(per_req - 0.1) < 1e-12 and abs(svc - 0.1) < 1e-12           # never below the per-request mean
    assert bench.service_time(0.5, [100], [])[1] == 0.5


def test_per_batch_jsonl_records(tmp_path):
    """--log-jsonl: one record per timed batch, its rate and GB/s from its own
    latency, kernel time and algorithmic bytes."""
    import json
    import bench
    recs = bench.step_records([2.0, 1.0], [1.5, 0.5], [[1.5, 2, 11, 100, 7], [0.5, 1, 5, 40, 3]], [26, 19],
                              [3.0e8, 1.0e8], 10000)
    assert [r["step"] for r in recs] == [0, 1]
    assert recs[0]["updates_per_s"] == 10000 / 2e-3 and recs[1]["updates_per_s"] == 10000 / 1e-3
    assert abs(recs[0]["alg_gbs"] - 3.0e8 / 1.5e6) < 1e-9 and recs[1]["iterations"] == 1
    assert recs[0]["barriers"] == 26 and recs[1]["relabels"] == 3
    path = tmp_path / "steps.jsonl"
    bench.write_jsonl(str(path), recs)
    back = [json.loads(line) for line in path.read_text().splitlines()]
    assert back == recs


def test_phase_roofline_arithmetic():
    """Per-phase rate: algorithmic bytes over the phase's device time, and its
    fraction of the peak; a phase that took no time reports 0."""
    import bench

    class FakeStats:
        def __init__(self, rows):
            self.rows = iter(rows)

        def stats(self):
            return next(self.rows)

    calls = [{"bytes_bfs": 3.0e8, "ms_bfs": 0.5, "bytes_discharge": 1.0e8, "ms_discharge": 0.25,
              "bytes_fix": 0, "ms_fix": 0.0, "bytes_apply": 1.0e6, "ms_apply": 0.1}] * 2
    S = FakeStats(calls)
    totals = {}
    bench._phase_rates(S, totals)
    bench._phase_rates(S, totals)
    assert totals["bfs"] == [6.0e8, 1.0] and totals["discharge"] == [2.0e8, 0.5]
    out = bench.phase_roofline(totals, hbm=6000.0)
    assert abs(out["bfs"]["gbs"] - 600.0) < 1e-9 and abs(out["bfs"]["frac"] - 0.1) < 1e-12
    assert abs(out["discharge"]["gbs"] - 400.0) < 1e-9
    assert out["fix"]["gbs"] == 0.0 and out["fix"]["frac"] == 0.0
    assert abs(out["apply"]["gbs"] - 10.0) < 1e-9
