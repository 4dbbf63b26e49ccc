"""The seeded input recipes: each generator draws what its workload names
(shapes, value ranges, sparsity structure, ring parameters), so the inputs
both the oracle and the CUDA path consume are the ones the design states."""
import numpy as np
import pytest

from paper_2604_11659_gb300 import synthetic


def test_bernoulli_sparse_density_and_range():
    rng = np.random.default_rng(0)
    M = synthetic.bernoulli_sparse(rng, 200, 300, 0.9)
    nz = M[M != 0]
    assert M.shape == (200, 300) and np.all(np.abs(nz) <= 1.0)
    n = M.size
    assert abs(nz.size / n - 0.1) < 5 * np.sqrt(0.09 / n)


@pytest.mark.parametrize("s", [0.5, 0.7, 0.95])
def test_structured_2_4(s):
    rng = np.random.default_rng(1)
    M = synthetic.structured_2_4(rng, 64, 128, s)
    groups = (M != 0).reshape(64, 32, 4).sum(axis=2)
    assert groups.max() <= 2
    n = M.size
    assert abs(np.count_nonzero(M) / n - (1 - s)) < 5 * np.sqrt((1 - s) * s / n) + 1e-9


def test_row_rescale_bounds_every_output():
    rng = np.random.default_rng(2)
    A = synthetic.bernoulli_sparse(rng, 16, 16, 0.3)
    B = synthetic.bernoulli_sparse(rng, 16, 16, 0.3)
    A2 = synthetic.rescale_rows_to_unit_output(A, B)
    C, C2 = A @ B, A2 @ B
    assert np.max(np.abs(C2)) <= 1.0 + 1e-12
    for i in range(16):
        if np.max(np.abs(C[i])) <= 1.0:
            assert np.array_equal(A2[i], A[i])
        else:
            assert abs(np.max(np.abs(C2[i])) - 1.0) < 1e-12


def test_small_and_bench_workloads():
    c = synthetic.case_16x16(seed=0)
    r = c.ring
    assert c.A.shape == c.B.shape == (16, 16)
    assert (r.log_n, r.q_bits, r.dnum, r.scale) == (12, [60, 40, 40, 40], 1, 2.0 ** 40)
    assert np.max(np.abs(c.A @ c.B)) <= 1.0 + 1e-12
    c = synthetic.case_128x128(seed=1)
    r = c.ring
    assert c.A.shape == c.B.shape == (128, 128)
    assert (r.log_n, r.L, r.q_bits[0], set(r.q_bits[1:]), r.dnum, r.scale) == (16, 24, 60, {45}, 3, 2.0 ** 45)
    for M in (c.A, c.B):
        assert abs(np.count_nonzero(M) / M.size - 0.1) < 0.02 and np.all(np.abs(M) <= 1.0)


def test_dense_layer_workload():
    c = synthetic.case_dense_layer(seed=3)
    r = c.ring
    assert c.A.shape == (64, 784) and c.B.shape == (784, 128)
    assert (r.log_n, r.L, r.q_bits[0], set(r.q_bits[1:]), r.dnum) == (17, 35, 60, {50}, 5)
    # ReLU-like activations: half exact zeros, the rest in [0, 1]
    assert abs(np.mean(c.A == 0) - 0.5) < 0.02 and c.A.min() >= 0.0 and c.A.max() <= 1.0
    # N(0, 0.05^2) weights magnitude-pruned to 90 %: exactly the largest 10 %
    # of the drawn weights survive, unchanged
    assert np.count_nonzero(c.B) == round(0.1 * c.B.size)
    W0 = np.random.default_rng(5).normal(0.0, 0.05, size=(784, 128))
    Wp = synthetic.pruned_weights(np.random.default_rng(5), 784, 128)
    keep = Wp != 0
    assert np.array_equal(Wp[keep], W0[keep])
    assert np.abs(W0[keep]).min() >= np.abs(W0[~keep]).max()
    # two-sided top 10 % of N(0, sigma^2): |w| above about 1.645 sigma
    assert abs(np.abs(W0[keep]).min() / 0.05 - 1.645) < 0.05


def test_batch_workload():
    cases = synthetic.batch64_cases(seed=2, count=64)
    assert len(cases) == 64
    for b, c in enumerate(cases):
        d, s = c.meta["d"], c.meta["sparsity"]
        assert d in (32, 64, 128, 256) and 0.70 <= s <= 0.95
        assert c.A.shape == c.B.shape == (d, d)
        assert (c.ring.log_n, c.ring.L, c.ring.dnum) == (16, 20, 4)
        if b % 2:
            assert (c.A != 0).reshape(d, d // 4, 4).sum(axis=2).max() <= 2
    assert {c.meta["d"] for c in cases} == {32, 64, 128, 256}


def test_serving_stream():
    reqs = synthetic.serving_stream(seed=4, count=400, rate_per_s=20.0)
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(np.mean(gaps) - 1 / 20.0) < 5 * (1 / 20.0) / np.sqrt(len(gaps))
    for r in reqs:
        assert r.case.meta["d"] in (64, 128, 256, 512) and 0.5 <= r.case.meta["sparsity"] <= 0.95
        assert 11 <= r.level <= 31 and 0 <= r.key_set < 4
        assert r.level <= r.case.ring.L
    assert {r.key_set for r in reqs} == {0, 1, 2, 3}
    assert (reqs[0].case.ring.log_n, reqs[0].case.ring.L, reqs[0].case.ring.dnum) == (16, 31, 4)
