"""GPU parity of the element-wise baselines of Sec. 4 (spfhe_naive_matmul_ct_ct:
Naive Dense, Naive Sparse with reading G15's skip rule, and the printed
"skip only when both are zero" rule): result chunks bit-identical to the
oracle's naive_ct_ct on the same keys, noise and densely packed operands,
key-switch counts equal, on a tiny ring (several operand and result chunks)
and on the 16x16 workload's ring (N = 2^12, the radix-16 transforms)."""
import os

import numpy as np
import pytest

from oracle import ckks, spmspm
from paper_2604_11659_gb300 import synthetic
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu

MODES = {"dense": spmspm.NAIVE_DENSE, "sparse": spmspm.NAIVE_SPARSE, "literal": spmspm.NAIVE_SPARSE_LITERAL}


def _run(case, mode, seed, rot_base=None):
    ckks.threads(os.cpu_count() or 1)
    p = Pair(case.ring, rot_base=rot_base)
    try:
        o, P, sp = p.o, p.P, p.spfhe
        rows, inner = case.A.shape
        cols = case.B.shape[1]
        amts = set()
        for a in spmspm.naive_rotation_amounts(rows, inner, cols, P.slots):
            amts.update(ckks.rotation_plan(a, P.slots, P.rot_base))
        keys = o.keygen(seed, rot_amounts=sorted(amts))
        gkeys = p.import_keys(keys)
        rng = np.random.default_rng(seed + 1)
        A_cts = [o.encrypt(o.encode(z, P.L, P.scale), keys, rng) for z in spmspm.dense_pack(case.A, P.slots)]
        B_cts = [o.encrypt(o.encode(z, P.L, P.scale), keys, rng) for z in spmspm.dense_pack(case.B, P.slots)]
        mask = spmspm.make_mask(o, 0, P.L - 1)
        counts = spmspm.OpCounts()
        want = spmspm.naive_ct_ct(o, keys, A_cts, B_cts, case.A != 0, case.B != 0, MODES[mode], mask_pt=mask,
                                  counts=counts)
        n_c = max(1, -(-(rows * cols) // P.slots))
        outs, st = sp.spfhe_naive_matmul_ct_ct(p.ctx, gkeys, MODES[mode], case.A != 0, case.B != 0,
                                               [p.import_ct(c) for c in A_cts], [p.import_ct(c) for c in B_cts],
                                               p.import_pt(mask), n_c)
        assert len(outs) == len(want) == n_c
        for h, w in zip(outs, want):
            p.assert_ct_equal(p.track("ct", h), w)
        assert (st["matches"], st["ks_relin"], st["ks_align"], st["ks_final"], st["rescales"]) == \
            (counts.matches, counts.ks_relin, counts.ks_align, counts.ks_final, counts.rescales)
        C = spmspm.decrypt_result(o, keys, want, rows, cols)
        assert np.max(np.abs(C - case.A @ case.B)) < 1e-4
        return st
    finally:
        p.close()


@pytest.mark.parametrize("mode", list(MODES))
def test_naive_tiny_ring_bit_exact(mode):
    """5 x 3 x 6 at n = 2^6 (32 slots) with 3 = dnum: 15 elements of A, 18 of B,
    a 30-slot result; 9 x 4 x 9 spills A, B and the result into two chunks."""
    for seed, (rows, inner, cols) in ((1, (5, 3, 6)), (2, (9, 4, 9))):
        case = synthetic.tiny_case(seed, 4, 0.5, log_n=6, L=5, dnum=3, rot_base=4, rows=rows, inner=inner, cols=cols)
        st = _run(case, mode, 10 + seed)
        if mode == "dense":
            assert st["matches"] == rows * inner * cols


def test_naive_sparse_workload_ring_bit_exact():
    """The 16x16 workload (N = 2^12, L = 4, dnum = 1, rotation base 16, 75 %
    sparsity): Naive Sparse computes Alg. 1's 2-operand-rotated products."""
    case = synthetic.case_16x16(seed=0)
    st = _run(case, "sparse", 40)
    Acsr, Bcsc = spmspm.dense_to_csr(case.A), spmspm.dense_to_csc(case.B)
    assert st["matches"] == len(spmspm.alg1_matches(Acsr[0], Acsr[1], Bcsc[0], Bcsc[1], 16, 16))


@pytest.mark.parametrize("mode", ["dense", "literal"])
def test_naive_workload_ring_small_matrix(mode):
    """Naive Dense and the literal rule at the 16x16 workload's ring on a 6x6
    product (216 products for Naive Dense)."""
    rng = np.random.default_rng(50)
    A = synthetic.bernoulli_sparse(rng, 6, 6, 0.5)
    B = synthetic.bernoulli_sparse(rng, 6, 6, 0.5)
    A = synthetic.rescale_rows_to_unit_output(A, B)
    case = synthetic.MatmulCase("naive6", A, B, synthetic.ring_small_16x16())
    _run(case, mode, 51)


def test_naive_errors():
    """Wrong chunk counts, an unknown mode and a missing pattern are refused."""
    case = synthetic.tiny_case(3, 4, 0.5, log_n=6, L=4, dnum=1, rot_base=4)
    p = Pair(case.ring)
    try:
        o, P, sp = p.o, p.P, p.spfhe
        keys = o.keygen(3, rot_amounts=ckks.rotation_key_amounts(P.slots, P.rot_base))
        gkeys = p.import_keys(keys)
        rng = np.random.default_rng(4)
        A_cts = [p.import_ct(o.encrypt(o.encode(z, P.L, P.scale), keys, rng)) for z in spmspm.dense_pack(case.A, P.slots)]
        B_cts = [p.import_ct(o.encrypt(o.encode(z, P.L, P.scale), keys, rng)) for z in spmspm.dense_pack(case.B, P.slots)]
        with pytest.raises(sp.SpfheError) as e:
            sp.spfhe_naive_matmul_ct_ct(p.ctx, gkeys, 7, case.A != 0, case.B != 0, A_cts, B_cts, None, 1)
        assert e.value.status == -1
        with pytest.raises(sp.SpfheError) as e:
            sp.spfhe_naive_matmul_ct_ct(p.ctx, gkeys, 0, case.A != 0, case.B != 0, A_cts + A_cts, B_cts, None, 1)
        assert e.value.status == -1
        with pytest.raises(sp.SpfheError) as e:
            sp.spfhe_naive_matmul_ct_ct(p.ctx, gkeys, 0, case.A != 0, case.B != 0, A_cts, B_cts, None, 2)
        assert e.value.status == -1
        # no rotation keys at all: EKEY before anything runs
        relin_only = p.track("keys", sp.spfhe_keys_import(p.ctx, keys.s, _ntt_key(p, keys.relin), {}))
        with pytest.raises(sp.SpfheError) as e:
            sp.spfhe_naive_matmul_ct_ct(p.ctx, relin_only, 0, case.A != 0, case.B != 0, A_cts, B_cts, None, 1)
        assert e.value.status == -4
    finally:
        p.close()


def _ntt_key(p, k):
    out = np.empty_like(k)
    mi = np.arange(p.M, dtype=np.int32)
    for j in range(k.shape[0]):
        for b in range(2):
            out[j, b] = p.o.rns_ntt(k[j, b], mi)
    return out
