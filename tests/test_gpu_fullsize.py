"""Parity at the benchmark's ring (N=2^16, L=24, dnum=3, K=7, rotation base
256) and launch configuration: a 128x128 product crafted to have a few
matches (the oracle needs tens of seconds per key switch at this size) is
bit-identical to the oracle, and the full 128x128 workload product decrypts
within 1e-4 of FP64 (a property that holds at any size).  At the dense
layer's ring (N=2^17, L=35, dnum=5, K=6, rotation base 16) a 64x784 x 784x128
product with three matches is bit-identical to the oracle through ct x ct,
ct x pt and the lazy-accumulation ct x pt product."""
import os

import numpy as np
import pytest

from oracle import ckks, spmspm
from paper_2604_11659_gb300 import synthetic
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu


def test_bench_ring_bit_exact_few_matches():
    ckks.threads(os.cpu_count() or 1)
    recipe = synthetic.ring_128x128()
    A = np.zeros((128, 128))
    B = np.zeros((128, 128))
    # row 3 of A meets columns 40 and 101 of B through k = 9 and k = 77;
    # B's nonzeros sit at other slots than A's, so one operand is aligned
    A[3, 9], A[3, 77], A[50, 77] = 0.5, -0.25, 0.75
    B[9, 101], B[77, 40], B[2, 7] = 0.8, -0.6, 0.3
    Acsr = spmspm.dense_to_csr(A)
    Bcsc = spmspm.dense_to_csc(B)
    p = Pair(recipe)
    try:
        o, P, sp = p.o, p.P, p.spfhe
        amounts = set()
        for r in spmspm.final_rotation_amounts(Acsr[:2], Bcsc[:2], 128, 128, P.slots):
            amounts.update(ckks.rotation_plan(r, P.slots, P.rot_base))
        keys = o.keygen(31, rot_amounts=sorted(amounts))
        gkeys = p.import_keys(keys)
        rng = np.random.default_rng(32)
        A_cts = [o.encrypt(o.encode(z, P.L, P.scale), keys, rng) for z in spmspm.pack_values(Acsr[2], P.slots)]
        B_cts = [o.encrypt(o.encode(z, P.L, P.scale), keys, rng) for z in spmspm.pack_values(Bcsc[2], P.slots)]
        mask = spmspm.make_mask(o, 0, P.L - 1)
        counts = spmspm.OpCounts()
        want = spmspm.spmspm_ct_ct(o, keys, Acsr[:2], A_cts, Bcsc[:2], B_cts, 128, 128, mask_pt=mask, counts=counts)
        assert counts.matches == 3 and counts.ks_final > 0 and counts.ks_align > 0
        outs, st = sp.spfhe_sparse_matmul_ct_ct(p.ctx, gkeys, sp.sparse_meta(Acsr[0], Acsr[1], 128, 128),
                                                [p.import_ct(c) for c in A_cts],
                                                sp.sparse_meta(Bcsc[0], Bcsc[1], 128, 128),
                                                [p.import_ct(c) for c in B_cts], p.import_pt(mask), 1)
        p.track("ct", outs[0])
        p.assert_ct_equal(outs[0], want[0])
        assert st["ks_final"] == counts.ks_final and st["ks_align"] == counts.ks_align
        C = spmspm.decrypt_result(o, keys, want, 128, 128)
        assert np.max(np.abs(C - A @ B)) < 1e-4
    finally:
        p.close()


def test_bench_workload_decrypts_within_tolerance():
    """The 128x128, 90 %-sparse product of the benchmark with the library's
    own keys, encryption and masks: max |decrypt(C) - A B| < 1e-4, for Alg. 2
    as printed and for the lazy-accumulation variant, whose relinearisation
    and final-rotation key switches equal the plan's group counts."""
    import torch
    import bench
    case = synthetic.case_128x128(seed=1)
    g = bench.GpuMatmul(case, 256, torch.cuda.current_stream().cuda_stream)
    try:
        outs, st = g.step()
        want_matches = int(sum(np.count_nonzero(case.A[:, k]) * np.count_nonzero(case.B[k, :]) for k in range(128)))
        assert st["matches"] == want_matches
        err = g.check(outs)
        g.free(outs)
        assert err < 1e-4
        outs, st = g.step(grouped=True)
        Acsr, Bcsc = spmspm.dense_to_csr(case.A), spmspm.dense_to_csc(case.B)
        relin, final = spmspm.grouped_key_switches(Acsr[:2], Bcsc[:2], 128, 128, 1 << 15, 256)
        assert st["matches"] == want_matches and st["ks_relin"] == relin and st["ks_final"] == final
        err = g.check(outs)
        g.free(outs)
        assert err < 1e-4
    finally:
        g.sp.spfhe_keys_free(g.keys)
        for h in g.A_cts + g.B_cts:
            g.sp.spfhe_ct_free(h)
        g.sp.spfhe_ctx_destroy(g.ctx)


def test_bench_ring_launch_configurations_bit_identical():
    """At the benchmark's ring with the library's own keys, a 128x128 product
    with a few hundred matches (464: seven 64-match batches and a ragged last
    one) yields bit-identical result ciphertexts whatever the match batch (64,
    the default; 7; 1, one match per launch sequence), the NTT kernel variant
    (6, the default; 5; 0) and the epilogue fusion.  Every launch computes the
    same integers by construction; this checks it at full size in the
    benchmark's launch configuration, where the oracle is too slow to follow
    every match (its exactness at this ring is the few-match test above).  The
    result decrypts within 1e-4 of A B."""
    import torch
    import bench
    rng = np.random.default_rng(7)
    A = synthetic.bernoulli_sparse(rng, 128, 128, 0.985)
    B = synthetic.bernoulli_sparse(rng, 128, 128, 0.985)
    A = synthetic.rescale_rows_to_unit_output(A, B)
    case = synthetic.MatmulCase("launch-configs", A, B, synthetic.ring_128x128())
    g = bench.GpuMatmul(case, 256, torch.cuda.current_stream().cuda_stream, ntt_chunk=0, ntt_variant=6)
    sp = g.sp

    def run():
        outs, st = g.step()
        bits = [sp.spfhe_ct_export(g.ctx, h, g.n) for h in outs]
        return outs, bits, st

    try:
        outs, ref, st = run()
        assert st["matches"] > 3 * 64 and st["matches"] % 64 != 0
        assert g.check(outs) < 1e-4
        g.free(outs)
        settings = [("match batch 7", lambda on: sp.spfhe_ctx_set_match_batch(g.ctx, 7 if on else 0)),
                    ("match batch 1", lambda on: sp.spfhe_ctx_set_match_batch(g.ctx, 1 if on else 0)),
                    ("NTT variant 5", lambda on: sp.spfhe_ctx_set_ntt_variant(g.ctx, 5 if on else 6)),
                    ("NTT variant 0", lambda on: sp.spfhe_ctx_set_ntt_variant(g.ctx, 0 if on else 6)),
                    ("fusion off", lambda on: sp.spfhe_ctx_set_fusion(g.ctx, not on))]
        for name, apply in settings:
            apply(True)
            try:
                outs, bits, st2 = run()
                g.free(outs)
            finally:
                apply(False)
            assert st2["matches"] == st["matches"], name
            assert all(np.array_equal(a, b) for a, b in zip(bits, ref)), name
    finally:
        sp.spfhe_keys_free(g.keys)
        for h in g.A_cts + g.B_cts:
            sp.spfhe_ct_free(h)
        sp.spfhe_ctx_destroy(g.ctx)


def _dense_layer_few_matches():
    """64x784 activations times 784x128 weights at the dense layer's ring with
    three matches: (0, 0) aligns A by 2 slots and needs no final rotation,
    (0, 1) sits at equal slots, (32, 3) aligns B by 1 slot and its final
    rotation is the single base-16 digit 15 * 16^3 (t - min_pos = 4096)."""
    A = np.zeros((64, 784))
    W = np.zeros((784, 128))
    A[0, 3], A[0, 9], A[0, 700], A[32, 50] = 0.6, 0.5, 0.25, 0.75
    W[700, 0], W[9, 1], W[4, 2], W[6, 2], W[50, 3] = -0.06, 0.08, 0.03, 0.04, -0.05
    return A, W


def test_dense_layer_ring_bit_exact_few_matches():
    """The dense layer's ring and launch configuration (N=2^17, L=35, dnum=5,
    K=6, rotation base 16): ct x ct (Alg. 2), ct x pt (Alg. 2 with weight
    plaintexts) and the lazy-accumulation ct x pt product the benchmark times
    are each bit-identical to the oracle on a product with three matches, and
    decrypt within 1e-4 of FP64."""
    ckks.threads(os.cpu_count() or 1)
    recipe = synthetic.ring_dense_layer()
    A, W = _dense_layer_few_matches()
    rows, cols = A.shape[0], W.shape[1]
    Acsr = spmspm.dense_to_csr(A)
    Bcsc = spmspm.dense_to_csc(W)
    p = Pair(recipe, rot_base=16)
    try:
        o, P, sp = p.o, p.P, p.spfhe
        assert (P.n, P.L, P.K) == (1 << 17, 35, 6)
        amounts = set(spmspm.final_rotation_amounts(Acsr[:2], Bcsc[:2], rows, cols, P.slots))
        # ct x pt rotates each product from A's slot to its target slot
        for m in spmspm.alg1_matches(Acsr[0], Acsr[1], Bcsc[0], Bcsc[1], rows, cols):
            amounts.add((m.a_pos % P.slots - (m.i * cols + m.j)) % P.slots)
        steps = set()
        for r in amounts:
            steps.update(ckks.rotation_plan(r, P.slots, P.rot_base))
        assert steps == {1, 2, 15 << 12}
        keys = o.keygen(41, rot_amounts=sorted(steps))
        gkeys = p.import_keys(keys)
        rng = np.random.default_rng(42)
        A_cts = [o.encrypt(o.encode(z, P.L, P.scale), keys, rng) for z in spmspm.pack_values(Acsr[2], P.slots)]
        B_cts = [o.encrypt(o.encode(z, P.L, P.scale), keys, rng) for z in spmspm.pack_values(Bcsc[2], P.slots)]
        gA = [p.import_ct(c) for c in A_cts]
        gB = [p.import_ct(c) for c in B_cts]
        Am = sp.sparse_meta(Acsr[0], Acsr[1], rows, A.shape[1])
        Bm = sp.sparse_meta(Bcsc[0], Bcsc[1], W.shape[0], cols)
        ref = A @ W

        # ct x ct, Alg. 2 as printed
        mask = spmspm.make_mask(o, 0, P.L - 1)
        counts = spmspm.OpCounts()
        want = spmspm.spmspm_ct_ct(o, keys, Acsr[:2], A_cts, Bcsc[:2], B_cts, rows, cols, mask_pt=mask,
                                   counts=counts)
        assert (counts.matches, counts.ks_align, counts.ks_final) == (3, 2, 1)
        outs, st = sp.spfhe_sparse_matmul_ct_ct(p.ctx, gkeys, Am, gA, Bm, gB, p.import_pt(mask), 1)
        p.track("ct", outs[0])
        p.assert_ct_equal(outs[0], want[0])
        assert st["ks_final"] == counts.ks_final and st["ks_align"] == counts.ks_align
        assert np.max(np.abs(spmspm.decrypt_result(o, keys, want, rows, cols) - ref)) < 1e-4

        # ct x pt: weight plaintexts encoded by the oracle, imported
        Bd = Bcsc[2]
        base = [o.encode_onehot(float(v), 0, P.L, spmspm.weight_scale(o)) for v in Bd]
        gpts = [p.import_pt(b) for b in base]
        counts = spmspm.OpCounts()
        want = spmspm.spmspm_ct_pt(o, keys, Acsr[:2], A_cts, Bcsc[:2], Bd, rows, cols, b_pts=base, counts=counts)
        outs, st = sp.spfhe_sparse_matmul_ct_pt(p.ctx, gkeys, Am, gA, Bm, None, gpts, 1)
        p.track("ct", outs[0])
        p.assert_ct_equal(outs[0], want[0])
        assert st["ks_final"] == counts.ks_final
        assert np.max(np.abs(spmspm.decrypt_result(o, keys, want, rows, cols) - ref)) < 1e-4

        # the lazy-accumulation ct x pt product (the benchmark's dense-layer path)
        counts = spmspm.OpCounts()
        want = spmspm.spmspm_ct_pt_grouped(o, keys, Acsr[:2], A_cts, Bcsc[:2], Bd, rows, cols, b_pts=base,
                                           merge_digits=True, counts=counts)
        outs, st = sp.spfhe_sparse_matmul_ct_pt_grouped(p.ctx, gkeys, Am, gA, Bm, None, gpts, 1, merge_digits=True)
        p.track("ct", outs[0])
        p.assert_ct_equal(outs[0], want[0])
        for k in ("matches", "ks_final", "rescales"):
            assert st[k] == getattr(counts, k), k
        assert np.max(np.abs(spmspm.decrypt_result(o, keys, want, rows, cols) - ref)) < 1e-4
    finally:
        p.close()
