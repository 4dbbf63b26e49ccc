"""GPU parity on degenerate and boundary shapes (1x1x1, dot and outer
products, results of exactly S and S + 1 slots, all-zero rows and columns, a
single far match, an operand one nonzero over a chunk): Alg. 2, the
lazy-accumulation variant and the ct x pt product, each bit-exact with the
oracle on identical keys, noise, operands, masks and weight plaintexts, with
equal op counts."""
import pytest

from oracle import spmspm
from paper_2604_11659_gb300 import synthetic
from tests.test_gpu_grouped import _run_grouped
from tests.test_gpu_spmspm import _run_ct_ct, _setup

pytestmark = pytest.mark.gpu

EDGE = synthetic.edge_cases()


@pytest.mark.parametrize("variant", ["alg2", "grouped", "ct_pt"])
@pytest.mark.parametrize("name", list(EDGE))
def test_edge_shapes_bit_exact(name, variant):
    case = EDGE[name]
    p = _setup(case, rot_base=case.ring.rot_base)
    try:
        if variant == "alg2":
            want, outs, stats, counts = _run_ct_ct(p)
        elif variant == "grouped":
            want, outs, stats, counts = _run_grouped(p, True)
        else:
            o, P, sp = p.o, p.P, p.spfhe
            Bd = p.Bcsc[2]
            base = [o.encode_onehot(float(v), 0, P.L, spmspm.weight_scale(o)) for v in Bd]
            counts = spmspm.OpCounts()
            want = spmspm.spmspm_ct_pt(o, p.keys, p.Acsr[:2], p.A_cts, p.Bcsc[:2], Bd, p.rows, p.cols,
                                       b_pts=base, counts=counts)
            gA = [p.import_ct(c) for c in p.A_cts]
            gpts = [p.import_pt(b) for b in base]
            outs, stats = sp.spfhe_sparse_matmul_ct_pt(p.ctx, p.gkeys, p.Am, gA, p.Bm, None, gpts, p.n_c)
            for h in outs:
                p.track("ct", h)
        assert len(outs) == len(want) == p.n_c
        for h, w in zip(outs, want):
            p.assert_ct_equal(h, w)
        for k in ("matches", "ks_relin", "ks_align", "ks_final", "rescales"):
            assert stats[k] == getattr(counts, k), k
    finally:
        p.close()
