"""GPU parity of the encrypted sparse matmul (Alg. 1 + Alg. 2) against the
oracle: result ciphertexts bit-exact on identical keys, noise, operands and
mask, op counts equal to the oracle's, decrypted results within 1e-4 of the
FP64 product; degenerate and error cases."""
import numpy as np
import pytest

from oracle import ckks, spmspm
from paper_2604_11659_gb300 import synthetic
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu


def _setup(case, rot_base=None, seed=11):
    p = Pair(case.ring, rot_base=rot_base)
    o, P = p.o, p.P
    A, B = case.A, case.B
    p.rows, p.cols = A.shape[0], B.shape[1]
    p.Acsr = spmspm.dense_to_csr(A)
    p.Bcsc = spmspm.dense_to_csc(B)
    p.keys = o.keygen(seed, rot_amounts=ckks.rotation_key_amounts(P.slots, P.rot_base))
    p.gkeys = p.import_keys(p.keys)
    rng = np.random.default_rng(seed + 1)
    p.A_cts = [o.encrypt(o.encode(z, P.L, P.scale), p.keys, rng) for z in spmspm.pack_values(p.Acsr[2], P.slots)]
    p.B_cts = [o.encrypt(o.encode(z, P.L, P.scale), p.keys, rng) for z in spmspm.pack_values(p.Bcsc[2], P.slots)]
    sp = p.spfhe
    p.Am = sp.sparse_meta(p.Acsr[0], p.Acsr[1], p.rows, A.shape[1])
    p.Bm = sp.sparse_meta(p.Bcsc[0], p.Bcsc[1], B.shape[0], p.cols)
    p.n_c = max(1, -(-(p.rows * p.cols) // P.slots))
    return p


def _run_ct_ct(p, use_oracle_mask=True):
    o, P, sp = p.o, p.P, p.spfhe
    mask = spmspm.make_mask(o, 0, P.L - 1)
    counts = spmspm.OpCounts()
    want = spmspm.spmspm_ct_ct(o, p.keys, p.Acsr[:2], p.A_cts, p.Bcsc[:2], p.B_cts, p.rows, p.cols,
                               mask_pt=mask if use_oracle_mask else None, counts=counts)
    gA = [p.import_ct(c) for c in p.A_cts]
    gB = [p.import_ct(c) for c in p.B_cts]
    gmask = p.import_pt(mask) if use_oracle_mask else None
    outs, stats = sp.spfhe_sparse_matmul_ct_ct(p.ctx, p.gkeys, p.Am, gA, p.Bm, gB, gmask, p.n_c)
    for h in outs:
        p.track("ct", h)
    return want, outs, stats, counts


CASES = {
    "tiny_4x4": lambda: synthetic.tiny_case(0, 4, 0.5, log_n=6),
    "tiny_dense_5x5": lambda: synthetic.tiny_case(1, 5, 0.0, log_n=6),
    "multi_chunk_8x8": lambda: synthetic.tiny_case(4, 8, 0.35, log_n=6, rot_base=4),
    "rect_3x7x5_dnum3": lambda: synthetic.tiny_case(5, 0, 0.4, log_n=7, L=6, dnum=3, rows=3, inner=7, cols=5),
}


@pytest.mark.parametrize("name", list(CASES))
def test_ct_ct_bit_exact_small(name):
    case = CASES[name]()
    p = _setup(case, rot_base=case.ring.rot_base)
    try:
        want, outs, stats, counts = _run_ct_ct(p)
        assert len(outs) == len(want)
        for h, w in zip(outs, want):
            p.assert_ct_equal(h, w)
        assert stats["matches"] == counts.matches
        assert stats["ks_relin"] == counts.ks_relin
        assert stats["ks_align"] == counts.ks_align
        assert stats["ks_final"] == counts.ks_final
        assert stats["rescales"] == counts.rescales
        C = spmspm.decrypt_result(p.o, p.keys, want, p.rows, p.cols)
        assert np.max(np.abs(C - spmspm.matmul_fp64(case.A, case.B))) < 1e-4
    finally:
        p.close()


def test_ct_ct_16x16_workload_bit_exact():
    case = synthetic.case_16x16(seed=0)
    p = _setup(case)
    try:
        want, outs, stats, counts = _run_ct_ct(p)
        p.assert_ct_equal(outs[0], want[0])
        # decrypt on the GPU and compare with FP64
        sp = p.spfhe
        pt = p.track("pt", sp.spfhe_decrypt(p.ctx, p.gkeys, outs[0]))
        vals = sp.spfhe_decode(p.ctx, pt, 256).real.reshape(16, 16)
        ref = spmspm.matmul_fp64(case.A, case.B)
        assert np.max(np.abs(vals - ref)) < 1e-4
    finally:
        p.close()


def test_library_mask_encoding_agrees():
    """With the library's own mask encoding the result still decrypts to
    A B within 1e-4 (bits may differ only where a mask coefficient lands on a
    rounding tie; parity runs pass the oracle's mask)."""
    case = synthetic.tiny_case(2, 4, 0.3, log_n=6)
    p = _setup(case)
    try:
        want, outs, stats, counts = _run_ct_ct(p, use_oracle_mask=False)
        sp = p.spfhe
        pt = p.track("pt", sp.spfhe_decrypt(p.ctx, p.gkeys, outs[0]))
        vals = sp.spfhe_decode(p.ctx, pt, 16).real.reshape(4, 4)
        assert np.max(np.abs(vals - spmspm.matmul_fp64(case.A, case.B))) < 1e-4
    finally:
        p.close()


def test_ct_pt_bit_exact_and_own_encoding():
    case = synthetic.tiny_case(6, 0, 0.5, log_n=6, rows=4, inner=6, cols=5)
    p = _setup(case)
    try:
        o, P, sp = p.o, p.P, p.spfhe
        Bd = p.Bcsc[2]
        base = [o.encode_onehot(float(v), 0, P.L, spmspm.weight_scale(o)) for v in Bd]
        counts = spmspm.OpCounts()
        want = spmspm.spmspm_ct_pt(o, p.keys, p.Acsr[:2], p.A_cts, p.Bcsc[:2], Bd, p.rows, p.cols,
                                   b_pts=base, counts=counts)
        gA = [p.import_ct(c) for c in p.A_cts]
        gpts = [p.import_pt(b) for b in base]
        outs, stats = sp.spfhe_sparse_matmul_ct_pt(p.ctx, p.gkeys, p.Am, gA, p.Bm, None, gpts, p.n_c)
        for h, w in zip(outs, want):
            p.track("ct", h)
            p.assert_ct_equal(h, w)
        assert stats["ks_final"] == counts.ks_final and stats["matches"] == counts.matches
        # library's own weight encoding: same product within tolerance
        outs2, _ = sp.spfhe_sparse_matmul_ct_pt(p.ctx, p.gkeys, p.Am, gA, p.Bm, Bd, None, p.n_c)
        pt = p.track("pt", sp.spfhe_decrypt(p.ctx, p.gkeys, p.track("ct", outs2[0])))
        vals = sp.spfhe_decode(p.ctx, pt, p.rows * p.cols).real.reshape(p.rows, p.cols)
        assert np.max(np.abs(vals - spmspm.matmul_fp64(case.A, case.B))) < 1e-4
    finally:
        p.close()


def test_fully_sparse_is_exact_zero():
    case = synthetic.tiny_case(7, 4, 1.0, log_n=6)
    p = _setup(case)
    try:
        want, outs, stats, counts = _run_ct_ct(p)
        assert stats["matches"] == 0
        assert not p.export_ct(outs[0]).any()
        p.assert_ct_equal(outs[0], want[0])
    finally:
        p.close()


def test_missing_rotation_key_is_ekey():
    case = synthetic.tiny_case(8, 4, 0.2, log_n=6)
    p = _setup(case)
    try:
        sp = p.spfhe
        only_relin = p.track("keys", sp.spfhe_keys_import(p.ctx, p.keys.s, _ntt_key(p, p.keys.relin), {}))
        gA = [p.import_ct(c) for c in p.A_cts]
        gB = [p.import_ct(c) for c in p.B_cts]
        with pytest.raises(sp.SpfheError) as e:
            sp.spfhe_sparse_matmul_ct_ct(p.ctx, only_relin, p.Am, gA, p.Bm, gB, None, p.n_c)
        assert e.value.status == -4
        with pytest.raises(sp.SpfheError) as e:
            sp.spfhe_sparse_matmul_ct_ct(p.ctx, p.gkeys, p.Am, gA, p.Bm, gB, None, p.n_c + 1)
        assert e.value.status == -1
    finally:
        p.close()


def _ntt_key(p, k):
    out = np.empty_like(k)
    mi = np.arange(p.M, dtype=np.int32)
    for j in range(k.shape[0]):
        for b in range(2):
            out[j, b] = p.o.rns_ntt(k[j, b], mi)
    return out


@pytest.mark.parametrize("fused,variant", [(True, 0), (True, 3), (True, 4), (True, 5), (True, 6), (False, 0),
                                           (False, 5), (False, 6)])
def test_ct_ct_fusion_on_off_bit_exact(fused, variant):
    """ModDown and rescale epilogues inside the forward transforms or as
    separate kernels: the same bits (n = 2^12 takes the radix-16 path)."""
    case = synthetic.case_16x16(seed=0)
    p = _setup(case)
    try:
        p.spfhe.spfhe_ctx_set_fusion(p.ctx, fused)
        p.spfhe.spfhe_ctx_set_ntt_variant(p.ctx, variant)
        want, outs, stats, counts = _run_ct_ct(p)
        for h, w in zip(outs, want):
            p.assert_ct_equal(h, w)
    finally:
        p.close()
