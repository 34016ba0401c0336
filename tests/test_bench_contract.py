"""bench.py's reference arm (the oracle on the host cores) prints the contract's JSON line,
and only rank 0 prints it.  A tiny UDV case keeps this a CPU test of seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--m", "4096", "--n", "64", "--kappa", "1e3", "--steps", "2",
        "--warmup", "0", "--cpu-iters", "2"]


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *ARGS], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_the_contract_line():
    out = _run({"LSQ_REF_ITERS": "500"})
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in rec, key
    assert rec["impl"] == "reference" and rec["n_gpus"] == 1 and rec["steps"] == 2
    assert rec["higher_is_better"] is True and rec["unit"] == "solves/s" and rec["vs_baseline"] is None
    assert rec["config"]["workload"] == "udv_dense_4096x64_kappa1000"
    assert rec["value"] > 0 and abs(rec["value"] * rec["ms_per_step"] / 1e3 - 1.0) < 1e-9
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == rec["value"] and "500" in cb["sample"]
    e2e = rec["e2e"]
    assert e2e["value"] == rec["value"] and e2e["unit"] == rec["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_runs_on_rank_zero_only():
    out = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out.returncode == 0 and not out.stdout.strip()


def test_roofline_bytes_of_the_benchmark_launch():
    """The algorithmic bytes bench.py divides by the kernel time: per PCG iteration one pass
    over A (m n elem) and one over the n x n SGS operator, plus the FP64 residual passes.
    At 262144 x 512 in double-float pairs that is 1,075,838,976 B per iteration, which at
    the measured 278.6 us per iteration is the 3.86 TB/s quoted for the benchmark."""
    import types
    sys.path.insert(0, ROOT)
    import bench
    m, n, it = 262144, 512, 110802
    info = types.SimpleNamespace(iters=[it], outer=[1])
    byts, flops = bench.pcg_algorithmic(None, m, n, info, 8, 8, 8)
    per_iter = m * n * 8 + n * n * 8
    assert per_iter == 1_075_838_976
    residual = 2 * (m * n * 8 + 8 * m)             # h = Â^T b and the final true residual
    assert byts == it * per_iter + residual
    assert abs(per_iter / 278.6e-6 / 1e12 - 3.86) < 0.005
    assert flops == it * (4.0 * m * n + 2.0 * n * n) + 2 * 4.0 * m * n


def test_sweep_latency_bound_arithmetic():
    """The sparse lines' `sweep` object: ms per sweep = one preconditioner application over 2t,
    and the latency bound = levels x (half the SM-to-SM round trip + one dependent L2 load).
    A fake library and tensor layer stand in for the GPU (no device is touched)."""
    import types
    sys.path.insert(0, ROOT)
    import bench

    class FakeEvent:
        def __init__(self, enable_timing=True):
            self.t = 0.0

        def record(self):
            FakeTorch.clock += 0.0
            self.t = FakeTorch.clock

        def elapsed_time(self, other):
            return 6.0   # ms for the timed applications

    class FakeTorch:
        clock = 0.0
        float64 = "f64"
        cuda = types.SimpleNamespace(synchronize=lambda: None, Event=FakeEvent)

        @staticmethod
        def randn(n, dtype=None, device=None):
            return [0.0] * n

    api = types.SimpleNamespace(measure_latency=lambda: {"l2_load_ns": 150.0, "sm_round_trip_ns": 320.0,
                                                         "cluster_barrier_ns": 190.0, "dsmem_load_ns": 100.0,
                                                         "sm_round_trip_fenced_ns": 800.0})
    P = types.SimpleNamespace(apply=lambda R: R)
    saved = sys.modules.get("torch")
    sys.modules["torch"] = FakeTorch
    try:
        out = bench.sweep_latency_bound(api, P, 40000, 1, 1583, reps=3)
    finally:
        if saved is not None:
            sys.modules["torch"] = saved
        else:
            del sys.modules["torch"]
    assert abs(out["ms_per_sweep"] - 6.0 / 3 / 2) < 1e-12
    assert abs(out["bound_ms_per_sweep"] - 1583 * (160.0 + 150.0) / 1e6) < 1e-12
    assert abs(out["frac"] - out["bound_ms_per_sweep"] / out["ms_per_sweep"]) < 1e-12
    assert out["bound"] == "latency" and out["levels"] == 1583


def test_paper_tables_match_the_golden_printed_counts():
    """The printed iteration counts the GPU paper-tables run sets its results beside (Sec. 5.1
    and 5.2) are the ones the oracle's pins use (tests/golden/paper_iterations.txt): CG's
    count and RS's mean over ten runs, row by row."""
    sys.path.insert(0, ROOT)
    import bench
    gold = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_iterations.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            fam, n, m, it_cg, it_rs, rs_mean, rs_std = line.split()
            gold[(fam, int(m), int(n))] = (int(it_cg), float(rs_mean))
    for fam, key in (("gaussian", "gauss"), ("semi_gaussian", "semi")):
        rows = bench.PAPER_TABLES[fam]
        assert len(rows) == 5
        for (m, n), cg, rs in rows:
            assert gold[(key, m, n)] == (cg, rs), (fam, m, n)


def test_paper_tables_of_the_ill_conditioned_families_match_the_printed_counts():
    """The UDV (Sec. 5.4) and random graph Laplacian (Sec. 5.5) rows of the GPU paper-tables
    run against tests/golden/paper_iterations_udv_graph.txt: the printed kappa(A^T A) of each
    UDV matrix, the graph sizes (two Chung-Lu graphs of n vertices glued on 5 give 2 n - 5,
    the printed vertex counts up to one), CG's count and RS's ten-run mean."""
    sys.path.insert(0, ROOT)
    import bench
    gold = {"udv": [], "graph": []}
    with open(os.path.join(ROOT, "tests", "golden", "paper_iterations_udv_graph.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            fam, key, m, n, it_cg, it_rs, rs_mean, rs_std = line.split()
            gold[fam].append((float(key), int(it_cg), float(rs_mean)))
    udv = bench.PAPER_TABLES["udv_linear_90000x300"]
    assert [(float(k), cg, float(rs)) for k, cg, rs in udv] == gold["udv"]
    graph = bench.PAPER_TABLES["graph_laplacian_chung_lu"]
    assert len(graph) == len(gold["graph"]) == 5
    for (n_each, cg, rs), (verts, g_cg, g_rs) in zip(graph, gold["graph"]):
        assert abs((2 * n_each - 5) - verts) <= 1 and (cg, float(rs)) == (g_cg, g_rs)
