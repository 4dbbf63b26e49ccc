"""bench.py's main path on CPU: the library, the workload object and CUDA
timing are replaced by stubs with fixed timings, so the glue that turns
measurements into the one JSON line (keys, units, the whole-job rate, the
roofline, the end-to-end copies, the optional sub-measurements) runs without
a GPU and is checked against the numbers the stubs produced."""
import json
import sys
import types

import numpy as np
import pytest

import bench

CLASSES = ["ntt_fwd", "ntt_inv", "modup_bconv", "ks_inner_product", "moddown_bconv", "moddown_final", "tensor",
           "rescale", "automorph", "mask_mul", "accumulate", "other", "ks_ntt_fwd", "ks_ntt_inv"]
STEP_MS = 2000.0


class FakeEvent:
    clock = 0.0

    def __init__(self, enable_timing=True):
        self.t = 0.0

    def record(self):
        FakeEvent.clock += STEP_MS
        self.t = FakeEvent.clock

    def elapsed_time(self, other):
        return other.t - self.t


class SpfheError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(msg)
        self.status = status


def fake_library():
    sp = types.SimpleNamespace()
    sp.SpfheError = SpfheError
    sp.launches = 0
    sp.spfhe_prof_alu_rates = lambda ctx: (1.1e12, 1.2e12, 1.15e12, 2.0e13, 7.2e12, 1.1e13)
    sp.spfhe_prof_enable = lambda ctx, on: None
    sp.spfhe_launch_count = lambda ctx: sp.launches

    def prof_all(ctx):
        d = {c: {"launches": 0, "ms": 0.0, "bytes": 0.0, "work": 0.0} for c in CLASSES}
        d["ks_ntt_fwd"] = {"launches": 100, "ms": 600.0, "bytes": 2.0e12, "work": 4.0e11,
                           "limbs": (400.0, 250.0, 150.0)}
        d["modup_bconv"] = {"launches": 50, "ms": 200.0, "bytes": 3.0e11, "work": 1.0e11}
        d["ks_inner_product"] = {"launches": 50, "ms": 100.0, "bytes": 5.0e11, "work": 0.0}
        return d
    sp.spfhe_prof_all = prof_all
    sp.spfhe_prof_keyswitch = lambda ctx: (1000, 7.5e10)
    sp.spfhe_ct_export = lambda ctx, h, n, out=None: out
    sp.spfhe_ct_import = lambda ctx, ptr, level, scale: ("ct", ptr)
    sp.matmul_req = lambda *a: a
    sp.spfhe_matmul_graph_create = lambda ctx, req, variant: "graph"
    sp.spfhe_matmul_graph_launch = lambda gr: None
    sp.spfhe_matmul_graph_results = lambda gr, n_c: (["c"] * n_c, {"launches": 40180})
    sp.spfhe_ct_free = lambda h: None
    sp.spfhe_matmul_graph_free = lambda gr: None
    sp.spfhe_tune_rotation_base = lambda *a: (256, 48014, 37251710976)
    sp.spfhe_keys_free = lambda k: None
    sp.spfhe_ctx_destroy = lambda ctx: None
    return sp


class FakeMatmul:
    def __init__(self, case, rot_base, stream, ntt_chunk=-1, ntt_variant=0):
        self.sp = SP
        self.case = case
        self.rec = case.ring
        self.ctx, self.keys = "ctx", "keys"
        self.K = 7
        self.n = 1 << 6                   # small buffers for the host copies
        self.n_c = 1
        self.A_cts, self.B_cts = ["a0"], ["b0"]
        self.Am = self.Bm = None
        self.rows, self.inner, self.cols = case.A.shape[0], case.A.shape[1], case.B.shape[1]
        self.nnz = (np.count_nonzero(case.A), np.count_nonzero(case.B))
        self.ntt_chunk, self.ntt_tune = (4, 8, 0), None
        self.keygen_s = 1.0
        self.last_frobenius = 0.0

    def step(self, A_cts=None, B_cts=None, grouped=False):
        SP.launches += 40180
        st = {"matches": 21310, "ks_relin": 21310, "ks_align": 5483, "ks_final": 42531, "rescales": 42620}
        if grouped:
            st = {"matches": 21310, "ks_relin": 11403, "ks_align": 3003, "ks_final": 11423, "rescales": 22806}
        return ["c"], st

    def free(self, outs):
        pass

    def check(self, outs):
        self.last_frobenius = 5e-6
        return 4e-7


SP = fake_library()


@pytest.fixture
def stubbed(monkeypatch):
    torch = pytest.importorskip("torch")
    FakeEvent.clock = 0.0
    SP.launches = 0
    monkeypatch.setattr(torch.cuda, "set_device", lambda i: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: types.SimpleNamespace(cuda_stream=0))
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda.profiler, "start", lambda: None)
    monkeypatch.setattr(torch.cuda.profiler, "stop", lambda: None)
    from paper_2604_11659_gb300 import build as gbuild
    monkeypatch.setattr(gbuild, "build", lambda *a, **k: None)
    monkeypatch.setattr(bench, "GpuMatmul", FakeMatmul)
    monkeypatch.setattr(bench, "_pinned", lambda shape: np.zeros(shape, np.uint64))
    monkeypatch.setattr(bench, "batch_vs_plain", lambda *a, **k: {"speedup": 1.7})
    monkeypatch.setattr(bench, "serve_run", lambda *a, **k: {"served": {"p99_ms": 1.0}})
    monkeypatch.setattr(bench, "dense_layer_pt", lambda *a, **k: {"ms": 1.0})
    monkeypatch.setattr(bench, "naive_sweep", lambda *a, **k: {"rows": []})
    monkeypatch.setattr(bench, "accuracy_table2", lambda *a, **k: {"rows": []})
    monkeypatch.setattr(bench, "workload_16x16_end_to_end", lambda *a, **k: {"gpu_ms": 1.0})
    monkeypatch.setattr(bench, "cpu_baseline_line", lambda *a, **k: {"value": 2e-5, "unit": "matmuls/s",
                                                                      "cores": 8, "kind": "oracle", "sample": "s"})
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)


def _run(monkeypatch, capsys, argv):
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    bench.main()
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_default_line_carries_the_contract(stubbed, monkeypatch, capsys):
    line = _run(monkeypatch, capsys, ["--steps", "2", "--warmup", "3"])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "clocks", "roofline",
              "cpu_baseline"):
        assert k in line, k
    assert line["n_gpus"] == 1 and line["steps"] == 2 and line["warmup"] == 3 and line["scaling"] == "weak"
    assert line["higher_is_better"] is True and line["vs_baseline"] is None and line["dtype"] == "u64"
    # two timed steps between two event records: the stub clock advanced by one STEP_MS
    assert line["ms_per_step"] == pytest.approx(STEP_MS / 2)
    assert line["value"] == pytest.approx(2 / (STEP_MS / 1e3))
    assert line["gpu_launches"] == 2 * 40180
    assert line["config"]["workload"].startswith("128x128 ct x ct")
    e2e = line["e2e"]
    assert e2e["h2d_bytes_per_step"] == 2 * 2 * 24 * 64 * 8 and e2e["d2h_bytes_per_step"] == 2 * 22 * 64 * 8
    roof = line["roofline"]
    assert roof["kernel"] == "ks_ntt_fwd" and roof["bound"] == "alu"
    assert roof["achieved"] == pytest.approx(4.0e11 / 0.6 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert roof["traffic"] is None and "variant 4" in roof["traffic_source"]
    assert roof["alu_microbench"]["frac_of_butterfly_peak"] == pytest.approx(4.0e11 / 0.6 / 1.2e12)
    assert line["max_abs_err"] == 4e-7 and line["frobenius_err"] == 5e-6
    assert line["rotation_base"] == {"used": 256, "tuner_pick": 256, "key_budget_gib": 40.0,
                                     "tuner_rotation_key_switches": 48014,
                                     "tuner_key_gib": pytest.approx(37251710976 / 2 ** 30)}
    assert line["graph"]["vs_eager"] == pytest.approx(1.0)
    assert line["variant_grouped"]["ks_per_step"] == 11403 + 3003 + 11423
    for k in ("batch", "batch_128x128", "serve", "dense_layer_ct_pt", "naive_sweep_16x16", "accuracy_table2",
              "workload_16x16"):
        assert k in line


def test_skips_leave_their_keys_out(stubbed, monkeypatch, capsys):
    line = _run(monkeypatch, capsys, ["--steps", "1", "--warmup", "3", "--graph-steps", "0", "--grouped-steps", "0",
                                      "--batch-products", "0", "--batch128-products", "0", "--serve-requests", "0",
                                      "--dense-layer", "0", "--naive-sweep", "0",
                                      "--no-cpu-baseline"])
    assert line["graph"] is None and line["variant_grouped"] is None
    for k in ("batch", "batch_128x128", "serve", "dense_layer_ct_pt", "cpu_baseline", "naive_sweep_16x16",
              "accuracy_table2", "workload_16x16"):
        assert k not in line
    assert line["ms_per_step"] == pytest.approx(STEP_MS)


def test_reference_arm_line(monkeypatch, capsys):
    """--impl reference times the oracle (here on the small 16x16 workload so
    the test stays short) and prints the same metric and config as the
    library's arm, with impl, cpu_baseline and a zero-copy e2e."""
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    line = _run(monkeypatch, capsys, ["--impl", "reference", "--workload", "16x16", "--steps", "1", "--warmup", "0"])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "matmuls/s"
    assert line["higher_is_better"] is True and line["value"] > 0
    assert line["config"]["workload"].startswith("16x16 ct x ct, ") and "N=2^12, L=4" in line["config"]["workload"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "matmuls/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def _install_stubs(rank):
    """The fixture's stubs, installed directly in a spawned rank process; the
    rank's device clock runs (rank + 1) times slower."""
    import torch
    from paper_2604_11659_gb300 import build as gbuild

    class RankEvent(FakeEvent):
        def record(self):
            FakeEvent.clock += STEP_MS * (rank + 1)
            self.t = FakeEvent.clock

    torch.cuda.set_device = lambda i: None
    torch.cuda.synchronize = lambda *a: None
    torch.cuda.current_stream = lambda *a: types.SimpleNamespace(cuda_stream=0)
    torch.cuda.Event = RankEvent
    torch.cuda.profiler.start = lambda: None
    torch.cuda.profiler.stop = lambda: None
    gbuild.build = lambda *a, **k: None
    bench.GpuMatmul = FakeMatmul
    bench._pinned = lambda shape: np.zeros(shape, np.uint64)
    bench.batch_vs_plain = lambda *a, **k: {"speedup": 1.7}
    bench.serve_run = lambda *a, **k: {"served": {"p99_ms": 1.0}}
    bench.dense_layer_pt = lambda *a, **k: {"ms": 1.0}
    bench.naive_sweep = lambda *a, **k: {"rows": []}
    bench.accuracy_table2 = lambda *a, **k: {"rows": []}


def _bench_rank(rank, world, port, out_dir):
    import os
    os.environ.update({"WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    _install_stubs(rank)
    sys.argv = ["bench.py", "--gpus", str(world), "--steps", "2", "--warmup", "3"]
    with open(os.path.join(out_dir, "rank%d.out" % rank), "w") as f:
        old = sys.stdout
        sys.stdout = f
        try:
            bench.main()
        finally:
            sys.stdout = old


def test_two_ranks_print_one_line_with_the_slowest_time(tmp_path):
    """bench.py under two ranks (gloo, processes): rank 0 alone prints, the
    time is the slowest rank's, and the value counts both ranks' products."""
    import socket

    import torch.multiprocessing as mp
    pytest.importorskip("torch")
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_bench_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    out0 = [ln for ln in (tmp_path / "rank0.out").read_text().splitlines() if ln.strip()]
    assert (tmp_path / "rank1.out").read_text().strip() == ""
    assert len(out0) == 1
    line = json.loads(out0[0])
    # rank 1's clock is twice as slow: two steps took 2 * STEP_MS there
    assert line["n_gpus"] == 2 and line["scaling"] == "weak"
    assert line["ms_per_step"] == pytest.approx(2 * STEP_MS / 2)
    assert line["value"] == pytest.approx(2 * 2 / (2 * STEP_MS / 1e3))
    assert "cpu_baseline" not in line
    assert line["variant_grouped"]["ms_per_step"] == pytest.approx(2 * STEP_MS / 2)


def test_traffic_reported_for_the_captured_variant(stubbed, monkeypatch, capsys):
    """When the tuner runs the kernel variant the DRAM counters were captured
    on, roofline.traffic is the per-launch estimate from the library's limb
    counts by pass kind, with its ratio to the algorithmic bytes."""
    orig = FakeMatmul.__init__

    def init(self, *a, **k):
        orig(self, *a, **k)
        self.ntt_chunk = (bench.NTT_FWD_DRAM_VARIANT, 8, 0)
    monkeypatch.setattr(FakeMatmul, "__init__", init)
    line = _run(monkeypatch, capsys, ["--steps", "2", "--warmup", "3"])
    roof = line["roofline"]
    want = bench.ks_ntt_fwd_traffic((400.0, 250.0, 150.0), 100)
    assert roof["traffic"] == pytest.approx(want)
    assert roof["traffic_over_algorithmic"] == pytest.approx(want / (2.0e12 / 100))
