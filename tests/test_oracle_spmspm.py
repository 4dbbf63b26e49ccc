"""Pins for the oracle's Alg. 1 planner and the encrypted Alg. 1 + Alg. 2
product: brute-force enumeration, the complexity model's match count,
FP64 A @ B within 1e-4, and the paper's degenerate cases (Sec. 4.2, 4.3)."""
import itertools

import numpy as np
import pytest

from oracle import ckks, spmspm
from paper_2604_11659_gb300 import synthetic
from tests.oracle_util import oracle_params


def _csr(M):
    ip, ix, _ = spmspm.dense_to_csr(M)
    return ip, ix


def test_formats_round_trip():
    M = synthetic.bernoulli_sparse(np.random.default_rng(0), 7, 5, 0.6)
    ip, ix, d = spmspm.dense_to_csr(M)
    R = np.zeros_like(M)
    for i in range(7):
        for p in range(ip[i], ip[i + 1]):
            R[i, ix[p]] = d[p]
    assert np.array_equal(R, M)
    ip, ix, d = spmspm.dense_to_csc(M)
    R = np.zeros_like(M)
    for j in range(5):
        for p in range(ip[j], ip[j + 1]):
            R[ix[p], j] = d[p]
    assert np.array_equal(R, M)


@pytest.mark.parametrize("seed,rows,inner,cols,s", [(0, 6, 5, 4, 0.5), (1, 8, 8, 8, 0.0), (2, 9, 3, 7, 0.8), (3, 5, 5, 5, 1.0)])
def test_alg1_matches_brute_force(seed, rows, inner, cols, s):
    rng = np.random.default_rng(seed)
    A = synthetic.bernoulli_sparse(rng, rows, inner, s)
    B = synthetic.bernoulli_sparse(rng, inner, cols, s)
    Aip, Aix, _ = spmspm.dense_to_csr(A)
    Bip, Bix, _ = spmspm.dense_to_csc(B)
    got = spmspm.alg1_matches(Aip, Aix, Bip, Bix, rows, cols)
    want = [(i, j, k) for i, j, k in itertools.product(range(rows), range(cols), range(inner))
            if A[i, k] != 0 and B[k, j] != 0]
    assert [(m.i, m.j, m.k) for m in got] == want
    for m in got:
        assert Aix[m.a_pos] == m.k and Bix[m.b_pos] == m.k
        assert Aip[m.i] <= m.a_pos < Aip[m.i + 1] and Bip[m.j] <= m.b_pos < Bip[m.j + 1]
    # match count = sum_k nnz(col k of A) * nnz(row k of B)
    assert len(got) == int(sum(np.count_nonzero(A[:, k]) * np.count_nonzero(B[k, :]) for k in range(inner)))


def test_dense_case_has_d_cubed_matches():
    d = 6
    A = np.ones((d, d))
    Aip, Aix, _ = spmspm.dense_to_csr(A)
    Bip, Bix, _ = spmspm.dense_to_csc(A)
    assert len(spmspm.alg1_matches(Aip, Aix, Bip, Bix, d, d)) == d ** 3


def _run(case, rot_base=None, dnum=None, variant="ct_ct", seed=7):
    recipe = case.ring
    P = oracle_params(recipe, rot_base=rot_base)
    o = ckks.Oracle(P)
    A, B = case.A, case.B
    rows, cols = A.shape[0], B.shape[1]
    Aip, Aix, Ad = spmspm.dense_to_csr(A)
    Bip, Bix, Bd = spmspm.dense_to_csc(B)
    amts = ckks.rotation_key_amounts(P.slots, P.rot_base)
    keys = o.keygen(seed, rot_amounts=amts)
    rng = np.random.default_rng(seed + 1)
    A_cts = [o.encrypt(o.encode(z, P.L, P.scale), keys, rng) for z in spmspm.pack_values(Ad, P.slots)]
    counts = spmspm.OpCounts()
    if variant == "ct_ct":
        B_cts = [o.encrypt(o.encode(z, P.L, P.scale), keys, rng) for z in spmspm.pack_values(Bd, P.slots)]
        res = spmspm.spmspm_ct_ct(o, keys, (Aip, Aix), A_cts, (Bip, Bix), B_cts, rows, cols, counts=counts)
    elif variant.startswith("grouped"):
        B_cts = [o.encrypt(o.encode(z, P.L, P.scale), keys, rng) for z in spmspm.pack_values(Bd, P.slots)]
        res = spmspm.spmspm_ct_ct_grouped(o, keys, (Aip, Aix), A_cts, (Bip, Bix), B_cts, rows, cols,
                                          merge_digits=variant == "grouped", counts=counts)
    elif variant.startswith("ptgrouped"):
        res = spmspm.spmspm_ct_pt_grouped(o, keys, (Aip, Aix), A_cts, (Bip, Bix), Bd, rows, cols,
                                          merge_digits=variant == "ptgrouped", counts=counts)
    else:
        res = spmspm.spmspm_ct_pt(o, keys, (Aip, Aix), A_cts, (Bip, Bix), Bd, rows, cols, counts=counts)
    C = spmspm.decrypt_result(o, keys, res, rows, cols)
    return o, P, keys, res, C, counts, (Aip, Aix, Bip, Bix)


@pytest.mark.parametrize("seed,d,s", [(0, 4, 0.5), (1, 5, 0.3), (2, 4, 0.0)])
def test_encrypted_product_matches_fp64(seed, d, s):
    case = synthetic.tiny_case(seed, d, s, log_n=6)
    o, P, keys, res, C, counts, (Aip, Aix, Bip, Bix) = _run(case)
    ref = spmspm.matmul_fp64(case.A, case.B)
    assert np.max(np.abs(C - ref)) < 1e-4
    # op counts predicted by the planner
    ms = spmspm.alg1_matches(Aip, Aix, Bip, Bix, d, d)
    assert counts.matches == counts.ks_relin == len(ms)
    assert counts.rescales == 2 * len(ms)
    S = P.slots
    fin = sum(len(ckks.rotation_plan((min(m.a_pos, m.b_pos) - (m.i * d + m.j)) % S, S, P.rot_base)) for m in ms)
    assert counts.ks_final == fin
    deltas = {("B" if m.a_pos < m.b_pos else "A", abs(m.a_pos - m.b_pos)) for m in ms if m.a_pos != m.b_pos}
    assert counts.ks_align == sum(len(ckks.rotation_plan(dd, S, P.rot_base)) for _, dd in deltas)


def test_multi_chunk_operands_and_result():
    # S = 32 slots: 8x8 result spans 2 chunks; dense-ish operands span 2 chunks
    case = synthetic.tiny_case(4, 8, 0.35, log_n=6, rot_base=4)
    o, P, keys, res, C, counts, _ = _run(case, rot_base=4)
    assert len(res) == 2
    assert np.max(np.abs(C - spmspm.matmul_fp64(case.A, case.B))) < 1e-4


def test_rectangular_ct_pt():
    case = synthetic.tiny_case(5, 0, 0.5, log_n=6, rows=3, inner=7, cols=5)
    o, P, keys, res, C, counts, _ = _run(case, variant="ct_pt")
    assert counts.rescales == counts.matches
    assert np.max(np.abs(C - spmspm.matmul_fp64(case.A, case.B))) < 1e-4


def test_fully_sparse_gives_exact_zero():
    case = synthetic.tiny_case(6, 4, 1.0, log_n=6)
    o, P, keys, res, C, counts, _ = _run(case)
    assert counts.matches == 0
    assert all(not r.c0.any() and not r.c1.any() for r in res)
    assert np.array_equal(C, np.zeros((4, 4)))


def test_identity_rhs_returns_lhs():
    case = synthetic.tiny_case(8, 4, 0.4, log_n=6)
    case.B = np.eye(4)
    o, P, keys, res, C, counts, _ = _run(case)
    assert np.max(np.abs(C - case.A)) < 1e-4


@pytest.mark.slow
def test_16x16_workload_matches_fp64():
    case = synthetic.case_16x16(seed=0)
    o, P, keys, res, C, counts, _ = _run(case)
    ref = spmspm.matmul_fp64(case.A, case.B)
    assert np.max(np.abs(C - ref)) < 1e-4
    assert spmspm.frobenius(C, ref) < 1e-3


# ---- lazy accumulation (a reordering of Alg. 2, checked against FP64) -------
def _dense_groups(A, B, S):
    """(result chunk, final amount) -> match count, enumerated from the dense
    matrices with slot positions taken from running nonzero counts."""
    rows, inner = A.shape
    cols = B.shape[1]
    a_pos = np.cumsum((A != 0).ravel()).reshape(A.shape) - 1          # CSR order
    b_pos = np.cumsum((B.T != 0).ravel()).reshape(B.T.shape) - 1      # CSC order
    groups = {}
    for i in range(rows):
        for j in range(cols):
            for k in range(inner):
                if A[i, k] != 0 and B[k, j] != 0:
                    t = i * cols + j
                    r = (min(a_pos[i, k] % S, b_pos[j, k] % S) - t % S) % S
                    key = (t // S, r)
                    groups[key] = groups.get(key, 0) + 1
    return groups


def _dense_alignments(A, B, S):
    """(operand, chunk) -> set of alignment amounts, from the dense matrices."""
    rows, inner = A.shape
    cols = B.shape[1]
    a_pos = np.cumsum((A != 0).ravel()).reshape(A.shape) - 1
    b_pos = np.cumsum((B.T != 0).ravel()).reshape(B.T.shape) - 1
    need = {}
    for i in range(rows):
        for j in range(cols):
            for k in range(inner):
                if A[i, k] != 0 and B[k, j] != 0:
                    pa, pb = a_pos[i, k], b_pos[j, k]
                    sa, sb = pa % S, pb % S
                    if sa < sb:
                        need.setdefault(("B", pb // S), set()).add(sb - sa)
                    elif sb < sa:
                        need.setdefault(("A", pa // S), set()).add(sa - sb)
    return need


def _topdown_key_switches(need, S, b):
    """Key switches of rotating each source by all its amounts digit by
    digit from the top, sharing the higher digits: one per distinct
    (source, higher digits, nonzero digit)."""
    ks = 0
    for amts in need.values():
        w = 1
        while w * b < S:
            w *= b
        while w >= 1:
            ks += len({(a - a % (w * b), (a // w) % b) for a in amts if (a // w) % b})
            w //= b
    return ks


def _tree_key_switches(groups, S, b):
    """Digit-by-digit merge of the group amounts, simulated on the amounts."""
    ks = 0
    live = set()
    for rc, r in groups:
        if r % b:
            ks += 1
        live.add((rc, r - r % b))
    w = b
    while w < S:
        nxt = set()
        for rc, rem in live:
            d = (rem // w) % b
            ks += d != 0
            nxt.add((rc, rem - d * w))
        live = nxt
        w *= b
    return ks


@pytest.mark.parametrize("seed,d,s,rot_base", [(0, 4, 0.5, 2), (1, 6, 0.3, 4), (2, 5, 0.0, 4), (3, 8, 0.5, 8)])
def test_grouped_product_matches_fp64_and_counts(seed, d, s, rot_base):
    case = synthetic.tiny_case(seed, d, s, log_n=6, rot_base=rot_base)
    o, P, keys, res, C, counts, (Aip, Aix, Bip, Bix) = _run(case, rot_base=rot_base, variant="grouped")
    ref = spmspm.matmul_fp64(case.A, case.B)
    assert np.max(np.abs(C - ref)) < 1e-4
    groups = _dense_groups(case.A, case.B, P.slots)
    assert counts.matches == sum(groups.values())
    assert counts.ks_relin == len(groups) and counts.rescales == 2 * len(groups)
    assert counts.ks_final == _tree_key_switches(groups, P.slots, P.rot_base)
    assert (counts.ks_relin, counts.ks_final) == spmspm.grouped_key_switches(
        (Aip, Aix), (Bip, Bix), d, d, P.slots, P.rot_base)
    assert counts.ks_align == _topdown_key_switches(_dense_alignments(case.A, case.B, P.slots), P.slots,
                                                    P.rot_base)


def test_grouped_merges_matches_and_saves_key_switches():
    """A dense 8x8 product on 32 slots: many matches share (chunk, amount),
    so the lazy variant needs fewer relinearisations and final-rotation key
    switches than Alg. 2, with or without merging digits, and all three
    decrypt to the FP64 product."""
    case = synthetic.tiny_case(9, 8, 0.0, log_n=6, rot_base=4)
    ref = spmspm.matmul_fp64(case.A, case.B)
    _, _, _, _, C_lit, lit, _ = _run(case, rot_base=4)
    _, _, _, res_g, C_g, grp, _ = _run(case, rot_base=4, variant="grouped")
    _, _, _, _, C_n, nom, _ = _run(case, rot_base=4, variant="grouped_nomerge")
    for C in (C_lit, C_g, C_n):
        assert np.max(np.abs(C - ref)) < 1e-4
    assert grp.matches == lit.matches == 512
    assert grp.ks_relin < lit.ks_relin and grp.ks_relin == nom.ks_relin
    assert grp.ks_final < nom.ks_final < lit.ks_final
    # top-down alignment shares the higher digits: never more key switches
    assert grp.ks_align <= lit.ks_align
    assert len(res_g) == 2


def test_grouped_fully_sparse_gives_exact_zero():
    case = synthetic.tiny_case(6, 4, 1.0, log_n=6)
    o, P, keys, res, C, counts, _ = _run(case, variant="grouped")
    assert counts.matches == 0 and counts.ks_relin == 0
    assert all(not r.c0.any() and not r.c1.any() for r in res)
    assert np.array_equal(C, np.zeros((4, 4)))


def _dense_groups_pt(A, B, S):
    """ct x pt groups: (result chunk, a_slot - t) -> match count."""
    rows, inner = A.shape
    cols = B.shape[1]
    a_pos = np.cumsum((A != 0).ravel()).reshape(A.shape) - 1
    groups = {}
    for i in range(rows):
        for j in range(cols):
            for k in range(inner):
                if A[i, k] != 0 and B[k, j] != 0:
                    t = i * cols + j
                    key = (t // S, (a_pos[i, k] % S - t % S) % S)
                    groups[key] = groups.get(key, 0) + 1
    return groups


@pytest.mark.parametrize("seed,rows,inner,cols,s,rot_base", [(5, 3, 7, 5, 0.5, 2), (6, 8, 8, 8, 0.2, 4),
                                                             (7, 6, 9, 4, 0.0, 8)])
def test_ct_pt_grouped_matches_fp64_and_counts(seed, rows, inner, cols, s, rot_base):
    case = synthetic.tiny_case(seed, 0, s, log_n=6, rows=rows, inner=inner, cols=cols, rot_base=rot_base)
    o, P, keys, res, C, counts, _ = _run(case, rot_base=rot_base, variant="ptgrouped")
    assert np.max(np.abs(C - spmspm.matmul_fp64(case.A, case.B))) < 1e-4
    groups = _dense_groups_pt(case.A, case.B, P.slots)
    assert counts.matches == sum(groups.values()) and counts.rescales == len(groups)
    assert counts.ks_final == _tree_key_switches(groups, P.slots, P.rot_base)
    _, _, _, _, C_n, nom, _ = _run(case, rot_base=rot_base, variant="ptgrouped_nomerge")
    assert np.max(np.abs(C_n - spmspm.matmul_fp64(case.A, case.B))) < 1e-4
    assert nom.ks_final >= counts.ks_final


# ---- degenerate and boundary shapes -------------------------------------------
EDGE = synthetic.edge_cases()


def _dense_match_count(A, B):
    """Alg. 1's matches counted from the dense matrices: for every inner index
    k, each nonzero of column k of A meets each nonzero of row k of B."""
    return int(sum(np.count_nonzero(A[:, k]) * np.count_nonzero(B[k, :]) for k in range(A.shape[1])))


@pytest.mark.parametrize("variant", ["ct_ct", "grouped", "ct_pt", "ptgrouped"])
@pytest.mark.parametrize("name", list(EDGE))
def test_edge_shapes_match_fp64(name, variant):
    case = EDGE[name]
    o, P, keys, res, C, counts, _ = _run(case, rot_base=case.ring.rot_base, variant=variant)
    rows, cols = case.A.shape[0], case.B.shape[1]
    assert len(res) == max(1, -(-(rows * cols) // P.slots))
    assert counts.matches == _dense_match_count(case.A, case.B)
    assert np.max(np.abs(C - spmspm.matmul_fp64(case.A, case.B))) < 1e-4
