"""Pins for the oracle's element-wise baselines of Sec. 4 (Naive Dense and
Naive Sparse, reading R16 for their packing, G15 for the skip rule): the
products each one computes against brute-force enumeration over the dense
matrices, the decrypted result against FP64 A @ B within 1e-4, key-switch
counts against an independent recount from the rotation plans, and the
degenerate cases (a 100 %-sparse pair: no work and an exact zero for Naive
Sparse, N^3 products of encrypted zeros for Naive Dense)."""
import itertools

import numpy as np
import pytest

from oracle import ckks, spmspm
from paper_2604_11659_gb300 import synthetic
from tests.oracle_util import oracle_params

MODES = {"dense": spmspm.NAIVE_DENSE, "sparse": spmspm.NAIVE_SPARSE, "literal": spmspm.NAIVE_SPARSE_LITERAL}


@pytest.mark.parametrize("seed,rows,inner,cols,s", [(0, 4, 5, 3, 0.5), (1, 6, 6, 6, 0.0), (2, 5, 4, 7, 0.9),
                                                    (3, 3, 3, 3, 1.0)])
def test_triples_brute_force(seed, rows, inner, cols, s):
    rng = np.random.default_rng(seed)
    A = synthetic.bernoulli_sparse(rng, rows, inner, s)
    B = synthetic.bernoulli_sparse(rng, inner, cols, s)
    allt = list(itertools.product(range(rows), range(cols), range(inner)))
    assert spmspm.naive_triples(A != 0, B != 0, spmspm.NAIVE_DENSE) == allt
    assert len(allt) == rows * inner * cols
    both = [(i, j, k) for i, j, k in allt if A[i, k] != 0 and B[k, j] != 0]
    assert spmspm.naive_triples(A != 0, B != 0, spmspm.NAIVE_SPARSE) == both
    either = [(i, j, k) for i, j, k in allt if A[i, k] != 0 or B[k, j] != 0]
    assert spmspm.naive_triples(A != 0, B != 0, spmspm.NAIVE_SPARSE_LITERAL) == either
    # Naive Sparse computes exactly Alg. 1's matches (in the same order)
    Aip, Aix, _ = spmspm.dense_to_csr(A)
    Bip, Bix, _ = spmspm.dense_to_csc(B)
    assert [(m.i, m.j, m.k) for m in spmspm.alg1_matches(Aip, Aix, Bip, Bix, rows, cols)] == both


def test_dense_pack_is_row_major():
    M = np.arange(12, dtype=float).reshape(3, 4) + 1
    chunks = spmspm.dense_pack(M, 8)
    assert len(chunks) == 2
    assert chunks[0].tolist() == [1, 2, 3, 4, 5, 6, 7, 8] and chunks[1].tolist() == [9, 10, 11, 12, 0, 0, 0, 0]


def _recount(A, B, mode, S, base):
    """Key switches an element-wise method needs, recounted from the rotation
    plans over the dense matrices."""
    rows, inner = A.shape
    cols = B.shape[1]
    align = final = n = 0
    for i, j, k in itertools.product(range(rows), range(cols), range(inner)):
        a, b = A[i, k] != 0, B[k, j] != 0
        if mode == "sparse" and not (a and b):
            continue
        if mode == "literal" and not (a or b):
            continue
        n += 1
        align += len(ckks.rotation_plan((i * inner + k) % S, S, base))
        align += len(ckks.rotation_plan((k * cols + j) % S, S, base))
        final += len(ckks.rotation_plan(-((i * cols + j) % S), S, base))
    return n, align, final


def _encrypted(case, rot_base, seed):
    P = oracle_params(case.ring, rot_base=rot_base)
    o = ckks.Oracle(P)
    rows, inner = case.A.shape
    cols = case.B.shape[1]
    keys = o.keygen(seed, rot_amounts=spmspm.naive_rotation_amounts(rows, inner, cols, P.slots)
                    if rot_base == 0 else ckks.rotation_key_amounts(P.slots, P.rot_base))
    rng = np.random.default_rng(seed + 1)
    A_cts = [o.encrypt(o.encode(z, P.L, P.scale), keys, rng) for z in spmspm.dense_pack(case.A, P.slots)]
    B_cts = [o.encrypt(o.encode(z, P.L, P.scale), keys, rng) for z in spmspm.dense_pack(case.B, P.slots)]
    return o, P, keys, A_cts, B_cts


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("rows,inner,cols,s", [(4, 4, 4, 0.5), (5, 3, 6, 0.3)])
def test_naive_products_match_fp64_and_counts(mode, rows, inner, cols, s):
    """5 x 3 x 6 at n = 2^5 (16 slots): the 30-slot result spans two chunks,
    A's 15 elements fit one, B's 18 spill into a second."""
    case = synthetic.tiny_case(7, 4, s, log_n=5, L=4, dnum=1, rot_base=4, rows=rows, inner=inner, cols=cols)
    o, P, keys, A_cts, B_cts = _encrypted(case, P_BASE, 11)
    counts = spmspm.OpCounts()
    res = spmspm.naive_ct_ct(o, keys, A_cts, B_cts, case.A != 0, case.B != 0, MODES[mode], counts=counts)
    C = spmspm.decrypt_result(o, keys, res, rows, cols)
    assert np.max(np.abs(C - case.A @ case.B)) < 1e-4
    n, align, final = _recount(case.A, case.B, mode, P.slots, P.rot_base)
    assert (counts.matches, counts.ks_align, counts.ks_final, counts.ks_relin) == (n, align, final, n)
    assert counts.rescales == 2 * n
    assert res[0].level == P.L - 2


P_BASE = 4


def test_naive_sparse_equals_alg2_values_not_work():
    """Naive Sparse and CSR/C compute the same products (Alg. 1's matches) and
    decrypt to the same matrix within 1e-4; CSR/C rotates at most one operand
    per match, Naive Sparse both (Sec. 3.2.2)."""
    case = synthetic.tiny_case(3, 4, 0.4, log_n=5, L=4, dnum=1, rot_base=4)
    o, P, keys, A_cts, B_cts = _encrypted(case, P_BASE, 21)
    cn = spmspm.OpCounts()
    rn = spmspm.naive_ct_ct(o, keys, A_cts, B_cts, case.A != 0, case.B != 0, spmspm.NAIVE_SPARSE, counts=cn)
    Acsr, Bcsc = spmspm.dense_to_csr(case.A), spmspm.dense_to_csc(case.B)
    rng = np.random.default_rng(22)
    Ac = [o.encrypt(o.encode(z, P.L, P.scale), keys, rng) for z in spmspm.pack_values(Acsr[2], P.slots)]
    Bc = [o.encrypt(o.encode(z, P.L, P.scale), keys, rng) for z in spmspm.pack_values(Bcsc[2], P.slots)]
    cc = spmspm.OpCounts()
    rc = spmspm.spmspm_ct_ct(o, keys, Acsr[:2], Ac, Bcsc[:2], Bc, 4, 4, counts=cc)
    Cn = spmspm.decrypt_result(o, keys, rn, 4, 4)
    Cc = spmspm.decrypt_result(o, keys, rc, 4, 4)
    assert np.max(np.abs(Cn - Cc)) < 1e-4
    assert cn.matches == cc.matches and cn.ks_relin == cc.ks_relin
    assert cn.ks_align > cc.ks_align


def test_fully_sparse_pair():
    """100 % sparsity: Naive Sparse does nothing and returns an exact zero;
    Naive Dense still multiplies all N^3 encrypted zeros (small, not exact)."""
    d = 3
    case = synthetic.MatmulCase("zeros", np.zeros((d, d)), np.zeros((d, d)), synthetic.ring_tiny(5, 4, 1, 4))
    o, P, keys, A_cts, B_cts = _encrypted(case, P_BASE, 31)
    cs = spmspm.OpCounts()
    rs = spmspm.naive_ct_ct(o, keys, A_cts, B_cts, case.A != 0, case.B != 0, spmspm.NAIVE_SPARSE, counts=cs)
    assert cs.matches == 0 and not rs[0].c0.any() and not rs[0].c1.any()
    cd = spmspm.OpCounts()
    rd = spmspm.naive_ct_ct(o, keys, A_cts, B_cts, case.A != 0, case.B != 0, spmspm.NAIVE_DENSE, counts=cd)
    assert cd.matches == d ** 3
    assert np.max(np.abs(spmspm.decrypt_result(o, keys, rd, d, d))) < 1e-4


def test_planted_rotation_direction_fails():
    """A Naive Dense that rotates the operands the wrong way (right instead of
    left) is caught by the FP64 check."""
    case = synthetic.tiny_case(5, 3, 0.0, log_n=5, L=4, dnum=1, rot_base=4)
    o, P, keys, A_cts, B_cts = _encrypted(case, P_BASE, 41)
    real_rotate = o.rotate
    o.rotate = lambda ct, r, k: real_rotate(ct, (-r) % P.slots, k) if r else ct
    try:
        res = spmspm.naive_ct_ct(o, keys, A_cts, B_cts, case.A != 0, case.B != 0, spmspm.NAIVE_DENSE)
    finally:
        o.rotate = real_rotate
    C = spmspm.decrypt_result(o, keys, res, 3, 3)
    assert np.max(np.abs(C - case.A @ case.B)) > 1e-2
