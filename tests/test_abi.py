"""C-ABI checks that need no GPU: the library loads, exports every entry
point include/spfhe.h declares, and its host-only planner (Alg. 1) matches
the oracle's merge exactly and rejects malformed metadata."""
import os
import re

import numpy as np
import pytest

from oracle import spmspm
from paper_2604_11659_gb300 import synthetic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sp():
    from paper_2604_11659_gb300 import build, spfhe
    build.build()
    spfhe.lib()
    return spfhe


def _declared():
    text = open(os.path.join(ROOT, "include", "spfhe.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spfhe_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(sp):
    names = _declared()
    assert len(names) >= 30
    lib = sp.lib()
    for nm in names:
        assert hasattr(lib, nm), nm
    assert sorted(sp.EXPORTED) == names


@pytest.mark.parametrize("seed,rows,inner,cols,s", [(0, 6, 5, 4, 0.5), (1, 16, 16, 16, 0.75), (2, 9, 3, 7, 0.9),
                                                    (3, 5, 5, 5, 1.0), (4, 128, 128, 128, 0.9)])
def test_planner_matches_oracle(sp, seed, rows, inner, cols, s):
    rng = np.random.default_rng(seed)
    A = synthetic.bernoulli_sparse(rng, rows, inner, s)
    B = synthetic.bernoulli_sparse(rng, inner, cols, s)
    Aip, Aix, _ = spmspm.dense_to_csr(A)
    Bip, Bix, _ = spmspm.dense_to_csc(B)
    got = sp.spfhe_plan_matches(sp.sparse_meta(Aip, Aix, rows, inner), sp.sparse_meta(Bip, Bix, inner, cols))
    want = [(m.i, m.j, m.k, m.a_pos, m.b_pos) for m in spmspm.alg1_matches(Aip, Aix, Bip, Bix, rows, cols)]
    assert [tuple(int(v) for v in r) for r in got] == want


def test_planner_rejects_malformed_metadata(sp):
    ip = np.array([0, 2, 3], np.int32)
    ix = np.array([0, 1, 1], np.int32)
    good = sp.sparse_meta(ip, ix, 2, 2)
    bad_range = sp.sparse_meta(ip, np.array([0, 5, 1], np.int32), 2, 2)
    unsorted = sp.sparse_meta(ip, np.array([1, 0, 1], np.int32), 2, 2)
    non_mono = sp.sparse_meta(np.array([0, 3, 2], np.int32), ix, 2, 2)
    for bad in (bad_range, unsorted, non_mono):
        with pytest.raises(sp.SpfheError) as e:
            sp.spfhe_plan_matches(bad, good)
        assert e.value.status == -1
    with pytest.raises(sp.SpfheError):
        sp.spfhe_plan_matches(good, sp.sparse_meta(ip, ix, 3, 2))   # inner dims differ


def _plan_key_switches(A, B, S, base):
    """Key switches of Alg. 1 + Alg. 2's rotations for one rotation base,
    counted from the oracle's planner and rotation plan: each distinct
    alignment (operand, chunk, amount) once, every final rotation."""
    from oracle import ckks
    Aip, Aix, _ = spmspm.dense_to_csr(A)
    Bip, Bix, _ = spmspm.dense_to_csc(B)
    cols = B.shape[1]
    align, ks = set(), 0
    for m in spmspm.alg1_matches(Aip, Aix, Bip, Bix, A.shape[0], cols):
        sa, sb = m.a_pos % S, m.b_pos % S
        if sa < sb:
            align.add(("B", m.b_pos // S, sb - sa))
        elif sb < sa:
            align.add(("A", m.a_pos // S, sa - sb))
        ks += len(ckks.rotation_plan((min(sa, sb) - (m.i * cols + m.j) % S) % S, S, base))
    return ks + sum(len(ckks.rotation_plan(d, S, base)) for _, _, d in align)


@pytest.mark.parametrize("seed,log_n,d,s", [(0, 6, 6, 0.5), (1, 7, 9, 0.3), (2, 12, 16, 0.75), (3, 16, 64, 0.9),
                                          (4, 5, 6, 0.3)])
def test_rotation_base_tuner_matches_oracle_counts(sp, seed, log_n, d, s):
    """The host-only tuner picks, among the power-of-two bases whose keys fit
    the budget, the one with the fewest key switches (ties: fewer keys), with
    counts equal to the oracle planner's."""
    from oracle import ckks
    rng = np.random.default_rng(seed)
    A = synthetic.bernoulli_sparse(rng, d, d, s)
    B = synthetic.bernoulli_sparse(rng, d, d, s)
    Aip, Aix, _ = spmspm.dense_to_csr(A)
    Bip, Bix, _ = spmspm.dense_to_csc(B)
    L, K, dnum = 5, 2, 2
    S = 1 << (log_n - 1)
    per_key = dnum * 2 * (L + K) * (1 << log_n) * 8
    rows = []
    b = 2
    while b <= S:
        rows.append((b, _plan_key_switches(A, B, S, b), len(ckks.rotation_key_amounts(S, b)) * per_key))
        b *= 2
    for budget in (max(r[2] for r in rows), sorted(r[2] for r in rows)[len(rows) // 2], min(r[2] for r in rows)):
        fits = [r for r in rows if r[2] <= budget]
        want = min(fits, key=lambda r: (r[1], r[2]))
        got = sp.spfhe_tune_rotation_base(log_n, L, K, dnum, sp.sparse_meta(Aip, Aix, d, d),
                                          sp.sparse_meta(Bip, Bix, d, d), budget)
        assert got == want, (budget, got, want)
    with pytest.raises(sp.SpfheError) as e:
        sp.spfhe_tune_rotation_base(log_n, L, K, dnum, sp.sparse_meta(Aip, Aix, d, d),
                                    sp.sparse_meta(Bip, Bix, d, d), min(r[2] for r in rows) - 1)
    assert e.value.status == -2


def test_no_cpu_fallback_without_a_gpu(sp):
    """On a host without a usable GPU the library computes nothing: creating
    a context fails with SPFHE_ECUDA and a message, and calls given no context
    fail with SPFHE_EINVAL.  (On a GPU host this test has nothing to check.)"""
    import ctypes
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2604_11659_gb300 import params as gparams
    with pytest.raises(sp.SpfheError) as e:
        sp.spfhe_ctx_create(gparams.ctx_params(synthetic.ring_tiny()))
    assert e.value.status == -6 and str(e.value)
    lib = sp.lib()
    n = ctypes.c_size_t(0)
    assert lib.spfhe_keys_export(None, None, None, None, ctypes.byref(n), None, None) == -1
    assert lib.spfhe_prof_alu_peak(None, None, None, None, None) == -1
    assert lib.spfhe_rescale_noalloc(None, None, 2, None) == -1
    assert lib.spfhe_sync(None) == -1


def test_planner_fuzz_valid_or_refused(sp):
    """Random shapes and densities, some with one corrupted index or pointer
    (or mismatched inner dimensions): the host planner either returns the
    oracle's matches or refuses the metadata with SPFHE_EINVAL."""
    rng = np.random.default_rng(123)
    planned = refused = 0
    for _ in range(600):
        rows, inner, cols = (int(x) for x in rng.integers(1, 10, 3))
        A = (rng.random((rows, inner)) < rng.random()) * 1.0
        B = (rng.random((inner, cols)) < rng.random()) * 1.0
        Aip, Aix, _ = spmspm.dense_to_csr(A)
        Bip, Bix, _ = spmspm.dense_to_csc(B)
        Aip, Aix, Bip, Bix = (np.array(x, np.int32) for x in (Aip, Aix, Bip, Bix))
        mode = int(rng.integers(0, 5))
        b_inner = inner
        if mode == 1 and Aix.size:
            Aix[rng.integers(0, Aix.size)] = rng.integers(-3, inner + 3)
        elif mode == 2:
            Aip[rng.integers(1, Aip.size)] = rng.integers(0, max(1, Aix.size))
        elif mode == 3 and Bix.size:
            Bix[rng.integers(0, Bix.size)] = rng.integers(-3, inner + 3)
        elif mode == 4:
            b_inner = inner + 1
        Am = sp.sparse_meta(Aip, Aix, rows, inner)
        Bm = sp.sparse_meta(Bip, Bix, b_inner, cols)
        if Am.nnz > Aix.size:      # a pointer past the caller's index array: not the library's to detect
            continue
        valid = (np.all(np.diff(Aip) >= 0) and all(np.all(np.diff(Aix[Aip[i]:Aip[i + 1]]) > 0) for i in range(rows))
                 and np.all((Aix >= 0) & (Aix < inner)) and np.all((Bix >= 0) & (Bix < inner))
                 and all(np.all(np.diff(Bix[Bip[j]:Bip[j + 1]]) > 0) for j in range(cols)) and b_inner == inner)
        try:
            got = sp.spfhe_plan_matches(Am, Bm)
        except sp.SpfheError as e:
            assert e.status == -1 and not valid
            refused += 1
            continue
        assert valid
        want = [(m.i, m.j, m.k, m.a_pos, m.b_pos) for m in spmspm.alg1_matches(Aip, Aix, Bip, Bix, rows, cols)]
        assert [tuple(int(v) for v in r) for r in got] == want
        planned += 1
    assert planned > 200 and refused > 50


def test_bench_kernel_classes_exist_in_the_library(sp):
    """Every kernel class bench.py reads from the profiler is one the library
    reports (a renamed class would otherwise fail only on the GPU)."""
    import bench
    names = {sp.spfhe_prof_class_name(c) for c in range(sp.spfhe_prof_classes())}
    assert bench.ALU_CLASSES <= names and bench.NTT_CLASSES <= names and set(bench.KS_CLASSES) <= names
