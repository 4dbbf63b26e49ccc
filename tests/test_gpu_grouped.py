"""GPU parity of the lazy-accumulation variants (spfhe_sparse_matmul_ct_ct_grouped,
spfhe_sparse_matmul_ct_pt_grouped) against the oracle's spmspm_ct_ct_grouped
and spmspm_ct_pt_grouped: result ciphertexts bit-exact on identical keys,
noise, operands, masks and weight plaintexts, with and without the
digit-by-digit rotation merge, at several batch sizes (the streaming tree
flushes differently); op counts equal to the oracle's; decrypted results
within 1e-4 of the FP64 product; error cases."""
import numpy as np
import pytest

from oracle import spmspm
from paper_2604_11659_gb300 import synthetic
from tests.test_gpu_spmspm import _setup

pytestmark = pytest.mark.gpu

CASES = {
    "tiny_4x4_b2": lambda: synthetic.tiny_case(0, 4, 0.5, log_n=6, rot_base=2),
    "dense_8x8_b4_two_chunks": lambda: synthetic.tiny_case(9, 8, 0.0, log_n=6, rot_base=4),
    "multi_chunk_8x8_b4": lambda: synthetic.tiny_case(4, 8, 0.35, log_n=6, rot_base=4),
    "rect_3x7x5_dnum3_b8": lambda: synthetic.tiny_case(5, 0, 0.4, log_n=7, L=6, dnum=3, rows=3, inner=7, cols=5,
                                                         rot_base=8),
}


def _run_grouped(p, merge, use_oracle_mask=True):
    o, P, sp = p.o, p.P, p.spfhe
    ell = p.A_cts[0].level
    mask = spmspm.make_mask_grouped(o, 0, ell)
    counts = spmspm.OpCounts()
    want = spmspm.spmspm_ct_ct_grouped(o, p.keys, p.Acsr[:2], p.A_cts, p.Bcsc[:2], p.B_cts, p.rows, p.cols,
                                       mask_pt=mask if use_oracle_mask else None, merge_digits=merge, counts=counts)
    gA = [p.import_ct(c) for c in p.A_cts]
    gB = [p.import_ct(c) for c in p.B_cts]
    gmask = p.import_pt(mask) if use_oracle_mask else None
    outs, stats = sp.spfhe_sparse_matmul_ct_ct_grouped(p.ctx, p.gkeys, p.Am, gA, p.Bm, gB, gmask, p.n_c,
                                                       merge_digits=merge)
    for h in outs:
        p.track("ct", h)
    return want, outs, stats, counts


@pytest.mark.parametrize("merge", [True, False])
@pytest.mark.parametrize("name", list(CASES))
def test_grouped_bit_exact_small(name, merge):
    case = CASES[name]()
    p = _setup(case, rot_base=case.ring.rot_base)
    try:
        want, outs, stats, counts = _run_grouped(p, merge)
        assert len(outs) == len(want)
        for h, w in zip(outs, want):
            p.assert_ct_equal(h, w)
        for k in ("matches", "ks_relin", "ks_align", "ks_final", "rescales"):
            assert stats[k] == getattr(counts, k), k
        C = spmspm.decrypt_result(p.o, p.keys, want, p.rows, p.cols)
        assert np.max(np.abs(C - spmspm.matmul_fp64(case.A, case.B))) < 1e-4
    finally:
        p.close()


def test_grouped_small_match_batches_and_big_groups():
    """One match per batch piece: groups larger than a piece are summed
    across pieces; still bit-exact."""
    case = CASES["dense_8x8_b4_two_chunks"]()
    p = _setup(case, rot_base=4)
    try:
        p.spfhe.spfhe_ctx_set_match_batch(p.ctx, 1)
        want, outs, stats, counts = _run_grouped(p, True)
        for h, w in zip(outs, want):
            p.assert_ct_equal(h, w)
    finally:
        p.close()


@pytest.mark.parametrize("batch", [2, 32])
def test_grouped_streamed_alignments_bit_exact(batch):
    """With an alignment-memory budget of zero every batch of groups computes
    the alignment rotations its matches use and frees them afterwards: the
    results are the oracle's bits, relinearisation and final-rotation counts
    unchanged, alignment key switches at least the kept-for-the-call count."""
    case = CASES["multi_chunk_8x8_b4"]()
    p = _setup(case, rot_base=4)
    try:
        p.spfhe.spfhe_ctx_set_align_budget(p.ctx, 0)
        p.spfhe.spfhe_ctx_set_match_batch(p.ctx, batch)
        want, outs, stats, counts = _run_grouped(p, True)
        for h, w in zip(outs, want):
            p.assert_ct_equal(h, w)
        for k in ("matches", "ks_relin", "ks_final", "rescales"):
            assert stats[k] == getattr(counts, k), k
        assert stats["ks_align"] >= counts.ks_align
    finally:
        p.close()


def test_grouped_library_mask_decrypts():
    """With the library's own mask (its encoder agrees with the oracle's to
    +-1 per coefficient, so no bit parity): within 1e-4 of FP64."""
    case = CASES["multi_chunk_8x8_b4"]()
    p = _setup(case, rot_base=4)
    try:
        want, outs, stats, counts = _run_grouped(p, True, use_oracle_mask=False)
        got = [p.export_ct(h) for h in outs]
        from oracle import ckks
        cts = [ckks.Ct(g[0].copy(), g[1].copy(), want[0].scale) for g in got]
        cts = [ckks.Ct(p.o.rns_intt(c.c0), p.o.rns_intt(c.c1), c.scale) for c in cts]
        C = spmspm.decrypt_result(p.o, p.keys, cts, p.rows, p.cols)
        assert np.max(np.abs(C - spmspm.matmul_fp64(case.A, case.B))) < 1e-4
    finally:
        p.close()


def test_grouped_16x16_workload_bit_exact():
    case = synthetic.case_16x16(seed=0)
    p = _setup(case)
    try:
        want, outs, stats, counts = _run_grouped(p, True)
        for h, w in zip(outs, want):
            p.assert_ct_equal(h, w)
        assert stats["ks_relin"] == counts.ks_relin < counts.matches
    finally:
        p.close()


def test_grouped_errors():
    case = CASES["tiny_4x4_b2"]()
    p = _setup(case, rot_base=2)
    sp = p.spfhe
    try:
        gA = [p.import_ct(c) for c in p.A_cts]
        gB = [p.import_ct(c) for c in p.B_cts]
        # a mask at level L-1 (the literal product's) is refused
        bad_mask = p.import_pt(spmspm.make_mask(p.o, 0, p.P.L - 1))
        with pytest.raises(sp.SpfheError) as e:
            sp.spfhe_sparse_matmul_ct_ct_grouped(p.ctx, p.gkeys, p.Am, gA, p.Bm, gB, bad_mask, p.n_c)
        assert e.value.status == -3
        # keys without rotation keys: EKEY before any launch
        relin_only = p.track("keys", sp.spfhe_keys_import(p.ctx, p.keys.s, _ntt_key(p, p.keys.relin), {}))
        with pytest.raises(sp.SpfheError) as e:
            sp.spfhe_sparse_matmul_ct_ct_grouped(p.ctx, relin_only, p.Am, gA, p.Bm, gB, None, p.n_c)
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


# ---- streaming tree with many digits, small batches ------------------------
@pytest.mark.parametrize("batch", [1, 3])
def test_grouped_base2_streaming_tree(batch):
    """Base 2 on 64 slots (six digit levels) with one or three groups per
    batch: tree sums complete and flush at every level while groups stream
    in; still bit-exact."""
    case = synthetic.tiny_case(12, 8, 0.3, log_n=7, L=5, dnum=1, rot_base=2)
    p = _setup(case, rot_base=2)
    try:
        p.spfhe.spfhe_ctx_set_match_batch(p.ctx, batch)
        want, outs, stats, counts = _run_grouped(p, True)
        for h, w in zip(outs, want):
            p.assert_ct_equal(h, w)
        assert stats["ks_final"] == counts.ks_final
    finally:
        p.close()


# ---- ct x pt ------------------------------------------------------------------
PT_CASES = {
    "rect_4x6x5_b2": lambda: synthetic.tiny_case(6, 0, 0.5, log_n=6, rows=4, inner=6, cols=5, rot_base=2),
    "multi_chunk_8x8_b4": lambda: synthetic.tiny_case(4, 8, 0.35, log_n=6, rot_base=4),
    "dense_6x9x4_b8": lambda: synthetic.tiny_case(7, 0, 0.0, log_n=6, rows=6, inner=9, cols=4, rot_base=8),
}


@pytest.mark.parametrize("batch", [0, 2])
@pytest.mark.parametrize("merge", [True, False])
@pytest.mark.parametrize("name", list(PT_CASES))
def test_ct_pt_grouped_bit_exact(name, merge, batch):
    case = PT_CASES[name]()
    p = _setup(case, rot_base=case.ring.rot_base)
    try:
        o, P, sp = p.o, p.P, p.spfhe
        if batch:
            sp.spfhe_ctx_set_match_batch(p.ctx, batch)
        Bd = p.Bcsc[2]
        base = [o.encode_onehot(float(v), 0, P.L, spmspm.weight_scale(o)) for v in Bd]
        counts = spmspm.OpCounts()
        want = spmspm.spmspm_ct_pt_grouped(o, p.keys, p.Acsr[:2], p.A_cts, p.Bcsc[:2], Bd, p.rows, p.cols,
                                           b_pts=base, merge_digits=merge, counts=counts)
        gA = [p.import_ct(c) for c in p.A_cts]
        gpts = [p.import_pt(b) for b in base]
        outs, stats = sp.spfhe_sparse_matmul_ct_pt_grouped(p.ctx, p.gkeys, p.Am, gA, p.Bm, None, gpts, p.n_c,
                                                           merge_digits=merge)
        assert len(outs) == len(want)
        for h, w in zip(outs, want):
            p.track("ct", h)
            p.assert_ct_equal(h, w)
        for k in ("matches", "ks_final", "rescales"):
            assert stats[k] == getattr(counts, k), k
        C = spmspm.decrypt_result(o, p.keys, want, p.rows, p.cols)
        assert np.max(np.abs(C - spmspm.matmul_fp64(case.A, case.B))) < 1e-4
        # the library's own weight encoding: the same product within tolerance
        outs2, _ = sp.spfhe_sparse_matmul_ct_pt_grouped(p.ctx, p.gkeys, p.Am, gA, p.Bm, Bd, None, p.n_c)
        vals = []
        for h in outs2:
            pt = p.track("pt", sp.spfhe_decrypt(p.ctx, p.gkeys, p.track("ct", h)))
            vals.append(sp.spfhe_decode(p.ctx, pt, P.slots).real)
        got = np.concatenate(vals)[: p.rows * p.cols].reshape(p.rows, p.cols)
        assert np.max(np.abs(got - spmspm.matmul_fp64(case.A, case.B))) < 1e-4
    finally:
        p.close()
