"""Host-side arithmetic of bench.py (no GPU): the DRAM-traffic estimate of
the key-switching forward transforms recovers the pass mix it is built from."""
import bench


def test_ks_ntt_fwd_traffic_weights_pass_kinds():
    """Per-launch DRAM traffic = the limbs of each pass kind times that kind's
    measured bytes per limb, over the class's launches."""
    la, lb, lf = 120.0, 70.0, 50.0          # pass-A, plain pass-B, fused pass-B limbs
    d = bench.NTT_FWD_DRAM_PER_LIMB
    want = (la * d["a"] + lb * d["b"] + lf * d["b_moddown"]) / 6
    assert abs(bench.ks_ntt_fwd_traffic((la, lb, lf), 6) - want) < 1e-6 * want
    assert bench.ks_ntt_fwd_traffic((64.0, 64.0, 0.0), 2) == (64 * d["a"] + 64 * d["b"]) / 2


def test_both_arms_share_the_config():
    c = bench.bench_config("w")
    assert c == bench.bench_config("w") and set(c) == {"workload", "l2", "parallelism"}


def test_alu_microbench_summary():
    meas = (1.5e12, 1.2e12, 1.4e12, 2.0e13, 1.0e13, 1.2e13)
    out = bench.alu_microbench(meas, 0.75e12, 2070.0)
    assert out["frac_of_butterfly_peak"] == 0.5
    meas2 = (1.0e12, 1.2e12, 1.5e12, 2.0e13, 1.0e13, 1.2e13)
    assert bench.alu_microbench(meas2, 0.75e12, 2070.0)["frac_of_butterfly_peak"] == 0.5
    assert abs(out["imad_per_clk_per_sm"] - 2.0e13 / (152 * 2070e6)) < 1e-9
    assert abs(out["imad_hi_per_clk_per_sm"] - 1.2e13 / (152 * 2070e6)) < 1e-9
    assert bench.alu_microbench(None, 1.0, 2070.0) is None
    assert "frac_of_butterfly_peak" not in bench.alu_microbench(meas, None, 2070.0)


def test_traffic_only_for_the_captured_variant():
    assert "variant 6, the tuner ran variant 4" in bench.traffic_source("ks_ntt_fwd", 4)
    assert bench.traffic_source("ks_ntt_fwd", bench.NTT_FWD_DRAM_VARIANT).startswith("ncu")
    assert bench.traffic_source("modup_bconv", 5).startswith("no DRAM")


def test_check_reports_max_abs_and_frobenius_errors():
    """GpuMatmul.check on a stub library: the decoded slots hold A B plus a
    known error, and both error measures come out of it."""
    import types

    import numpy as np
    A = np.array([[1.0, 0.0], [0.5, 2.0]])
    B = np.array([[0.0, 1.0], [1.0, 0.0]])
    err = np.array([3e-7, -4e-7, 0.0, 0.0])
    S = 8
    slots = np.zeros(S)
    slots[:4] = (A @ B).reshape(-1) + err
    sp = types.SimpleNamespace(spfhe_decrypt=lambda ctx, keys, h: h, spfhe_pt_free=lambda pt: None,
                               spfhe_decode=lambda ctx, pt, n: slots[:n].astype(complex))
    g = bench.GpuMatmul.__new__(bench.GpuMatmul)
    g.sp, g.ctx, g.keys, g.S, g.rows, g.cols = sp, None, None, S, 2, 2
    g.case = types.SimpleNamespace(A=A, B=B)
    assert abs(g.check(["chunk"]) - 4e-7) < 1e-15
    assert abs(g.last_frobenius - 5e-7) < 1e-15


def test_clock_summary_parses_samples_and_reasons(tmp_path):
    """The nvidia-smi samples taken during the timed region: median SM clock,
    the maximum, and every throttle reason seen Active."""
    path = tmp_path / "clocks.csv"
    path.write_text("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 1980, 2070, 1380.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                    "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "garbage line\n")
    c = bench.ClockSampler(0)
    c.path = str(path)
    out = c.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    assert not path.exists()
    empty = tmp_path / "empty.csv"
    empty.write_text("")
    c.path = str(empty)
    assert c.summary()["reasons"] == ["no samples"]
