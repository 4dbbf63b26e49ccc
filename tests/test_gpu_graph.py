"""Products captured once as a CUDA graph and launched repeatedly: every
launch reproduces the oracle's result ciphertexts bit-exactly (Alg. 2 and
the lazy-accumulation variant), result handles belong to the graph, and the
operands are read at every launch."""
import numpy as np
import pytest

from oracle import spmspm
from paper_2604_11659_gb300 import synthetic
from tests.test_gpu_spmspm import _setup

pytestmark = pytest.mark.gpu


def _req(p, gA, gB, mask):
    return p.spfhe.matmul_req(p.gkeys, p.Am, gA, p.Bm, gB, mask)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("name", ["multi_chunk_8x8", "16x16"])
def test_graph_launches_bit_exact(name, variant):
    case = (synthetic.tiny_case(4, 8, 0.35, log_n=6, rot_base=4) if name == "multi_chunk_8x8"
            else synthetic.case_16x16(seed=0))
    p = _setup(case, rot_base=case.ring.rot_base)
    sp, o, P = p.spfhe, p.o, p.P
    g = None
    try:
        ell = P.L
        if variant == 0:
            mask = spmspm.make_mask(o, 0, ell - 1)
            want = spmspm.spmspm_ct_ct(o, p.keys, p.Acsr[:2], p.A_cts, p.Bcsc[:2], p.B_cts, p.rows, p.cols,
                                       mask_pt=mask)
        else:
            mask = spmspm.make_mask_grouped(o, 0, ell)
            want = spmspm.spmspm_ct_ct_grouped(o, p.keys, p.Acsr[:2], p.A_cts, p.Bcsc[:2], p.B_cts, p.rows,
                                               p.cols, mask_pt=mask)
        gA = [p.import_ct(c) for c in p.A_cts]
        gB = [p.import_ct(c) for c in p.B_cts]
        gmask = p.import_pt(mask)
        g = sp.spfhe_matmul_graph_create(p.ctx, _req(p, gA, gB, gmask), variant)
        for _ in range(2):
            sp.spfhe_matmul_graph_launch(g)
            sp.spfhe_sync(p.ctx)
            outs, st = sp.spfhe_matmul_graph_results(g, p.n_c)
            for h, w in zip(outs, want):
                p.assert_ct_equal(h, w)
                sp.spfhe_ct_free(h)   # frees the handle only
        assert st["matches"] > 0
    finally:
        if g is not None:
            sp.spfhe_matmul_graph_free(g)
        p.close()


def test_graph_reads_operands_at_every_launch():
    """Swapping the operands' contents between launches (A and B exchanged
    on a square product with equal sparsity patterns) changes the result to
    the product of the new contents."""
    case = synthetic.tiny_case(9, 8, 0.0, log_n=6, rot_base=4)   # dense: both patterns full
    case.B = case.B.copy()
    p = _setup(case, rot_base=4)
    sp, o, P = p.spfhe, p.o, p.P
    g = None
    try:
        mask = spmspm.make_mask(o, 0, P.L - 1)
        gA = [p.import_ct(c) for c in p.A_cts]
        gB = [p.import_ct(c) for c in p.B_cts]
        g = sp.spfhe_matmul_graph_create(p.ctx, _req(p, gA, gB, p.import_pt(mask)), 0)
        sp.spfhe_matmul_graph_launch(g)
        sp.spfhe_sync(p.ctx)
        # overwrite A's chunks with zeros: the next launch must give zero
        for h in gA:
            lv, sc = sp.spfhe_ct_info(h)
            zero = np.zeros((2, lv, p.n), dtype=np.uint64)
            sp.spfhe_ct_overwrite(p.ctx, h, zero)
        sp.spfhe_matmul_graph_launch(g)
        sp.spfhe_sync(p.ctx)
        outs, _ = sp.spfhe_matmul_graph_results(g, p.n_c)
        for h in outs:
            assert not p.export_ct(h).any()
            sp.spfhe_ct_free(h)
    finally:
        if g is not None:
            sp.spfhe_matmul_graph_free(g)
        p.close()


def test_graph_bad_variant():
    case = synthetic.tiny_case(0, 4, 0.5, log_n=6)
    p = _setup(case)
    sp = p.spfhe
    try:
        gA = [p.import_ct(c) for c in p.A_cts]
        gB = [p.import_ct(c) for c in p.B_cts]
        with pytest.raises(sp.SpfheError) as e:
            sp.spfhe_matmul_graph_create(p.ctx, _req(p, gA, gB, None), 7)
        assert e.value.status == -1
    finally:
        p.close()
