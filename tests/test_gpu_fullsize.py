"""Parity at the benchmark's ring (N=2^16, L=24, dnum=3, K=7, rotation base
256) and launch configuration: a 128x128 product crafted to have a few
matches (the oracle needs tens of seconds per key switch at this size) is
bit-identical to the oracle, and the full 128x128 workload product decrypts
within 1e-4 of FP64 (a property that holds at any size)."""
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
