"""Many products in one call (spfhe_sparse_matmul_batch) and the serving loop
(spfhe_server_*): every result bit-identical to the oracle and to the same
request run alone, with requests of different shapes and levels mixed in one
batch, and a failing request (missing rotation keys) that leaves the others
untouched."""
import time

import numpy as np
import pytest

from oracle import ckks, spmspm
from paper_2604_11659_gb300 import synthetic
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu


class Req:
    pass


@pytest.fixture(scope="module")
def setup():
    recipe = synthetic.ring_tiny(log_n=7, L=6, dnum=3, rot_base=4)
    p = Pair(recipe)
    o, P, sp = p.o, p.P, p.spfhe
    p.keys = o.keygen(21, rot_amounts=ckks.rotation_key_amounts(P.slots, P.rot_base))
    p.gkeys = p.import_keys(p.keys)
    rng = np.random.default_rng(5)
    shapes = [(4, 4, 4, 0.5, P.L), (5, 3, 6, 0.3, P.L - 1), (8, 8, 8, 0.2, P.L), (6, 7, 2, 0.6, P.L - 1)]
    p.reqs = []
    for k, (rows, inner, cols, s, ell) in enumerate(shapes):
        r = Req()
        A = synthetic.bernoulli_sparse(rng, rows, inner, s)
        B = synthetic.bernoulli_sparse(rng, inner, cols, s)
        r.A = synthetic.rescale_rows_to_unit_output(A, B)
        r.B = B
        r.rows, r.cols, r.ell = rows, cols, ell
        r.Acsr = spmspm.dense_to_csr(r.A)
        r.Bcsc = spmspm.dense_to_csc(r.B)
        r.A_cts = [o.encrypt(o.encode(z, ell, P.scale), p.keys, rng) for z in spmspm.pack_values(r.Acsr[2], P.slots)]
        r.B_cts = [o.encrypt(o.encode(z, ell, P.scale), p.keys, rng) for z in spmspm.pack_values(r.Bcsc[2], P.slots)]
        r.mask = spmspm.make_mask(o, 0, ell - 1)
        r.want = spmspm.spmspm_ct_ct(o, p.keys, r.Acsr[:2], r.A_cts, r.Bcsc[:2], r.B_cts, rows, cols, mask_pt=r.mask)
        r.gA = [p.import_ct(c) for c in r.A_cts]
        r.gB = [p.import_ct(c) for c in r.B_cts]
        r.gmask = p.import_pt(r.mask)
        r.Am = sp.sparse_meta(r.Acsr[0], r.Acsr[1], rows, inner)
        r.Bm = sp.sparse_meta(r.Bcsc[0], r.Bcsc[1], inner, cols)
        r.n_c = max(1, -(-(rows * cols) // P.slots))
        alone, st = sp.spfhe_sparse_matmul_ct_ct(p.ctx, p.gkeys, r.Am, r.gA, r.Bm, r.gB, r.gmask, r.n_c)
        r.alone = [p.export_ct(p.track("ct", h)) for h in alone]
        r.stats = st
        p.reqs.append(r)
    yield p
    p.close()


def _req(p, r, keys=None):
    return p.spfhe.matmul_req(keys or p.gkeys, r.Am, r.gA, r.Bm, r.gB, r.gmask)


def test_single_calls_match_oracle(setup):
    p = setup
    for r in p.reqs:
        assert len(r.alone) == len(r.want)
        for got, w in zip(r.alone, r.want):
            assert np.array_equal(got, p.ct_limbs(w))
        assert r.alone[0].shape[1] == r.ell - 2


def test_batch_equals_alone(setup):
    p = setup
    sp = p.spfhe
    outs, stats = sp.spfhe_sparse_matmul_batch(p.ctx, [_req(p, r) for r in p.reqs], [r.n_c for r in p.reqs])
    for r, hs, st in zip(p.reqs, outs, stats):
        got = [p.export_ct(p.track("ct", h)) for h in hs]
        for g, a in zip(got, r.alone):
            assert np.array_equal(g, a)
        for k in ("matches", "ks_relin", "ks_align", "ks_final", "rescales"):
            assert st[k] == r.stats[k]


def test_server_mix_equals_alone_and_isolates_errors(setup):
    p = setup
    sp = p.spfhe
    relin_only = p.track("keys", sp.spfhe_keys_import(p.ctx, p.keys.s, _ntt_key(p, p.keys.relin), {}))
    srv = sp.spfhe_server_create(p.ctx, 1 << 30)
    got, lats = [], []
    try:
        tickets = []
        for i, r in enumerate(p.reqs):
            tickets.append(sp.spfhe_server_submit(srv, _req(p, r)))
            if i == 1:
                bad = sp.spfhe_server_submit(srv, _req(p, p.reqs[2], keys=relin_only))
                time.sleep(0.01)
        for r, t in zip(p.reqs, tickets):
            hs, st, lat = sp.spfhe_server_wait(srv, t, r.n_c)
            got.append(hs)
            lats.append(lat)
            assert st["matches"] == r.stats["matches"]
        with pytest.raises(sp.SpfheError) as e:
            sp.spfhe_server_wait(srv, bad, p.reqs[2].n_c)
        assert e.value.status == -4
    finally:
        sp.spfhe_server_destroy(srv)
    # the context is the caller's again: read the results
    for r, hs, lat in zip(p.reqs, got, lats):
        assert lat > 0
        for h, a in zip(hs, r.alone):
            assert np.array_equal(p.export_ct(p.track("ct", h)), a)


def _ntt_key(p, k):
    out = np.empty_like(k)
    mi = np.arange(p.M, dtype=np.int32)
    for j in range(k.shape[0]):
        for b in range(2):
            out[j, b] = p.o.rns_ntt(k[j, b], mi)
    return out


def test_graph_batch_equals_alone(setup):
    """Every request of the batch captured into one CUDA graph (one task
    engine over all of them, mixed levels): two launches, each request's
    chunks equal to its single call's, counters equal."""
    p = setup
    sp = p.spfhe
    g = sp.spfhe_matmul_graph_create_batch(p.ctx, [_req(p, r) for r in p.reqs], 0)
    try:
        for _ in range(2):
            sp.spfhe_matmul_graph_launch(g)
            sp.spfhe_sync(p.ctx)
            outs, stats = sp.spfhe_matmul_graph_results_batch(g, [r.n_c for r in p.reqs])
            for r, hs, st in zip(p.reqs, outs, stats):
                for h, a in zip(hs, r.alone):
                    assert np.array_equal(p.export_ct(h), a)
                    sp.spfhe_ct_free(h)   # the handle only
                for k in ("matches", "ks_relin", "ks_align", "ks_final", "rescales"):
                    assert st[k] == r.stats[k]
    finally:
        sp.spfhe_matmul_graph_free(g)


def test_graph_batch_grouped_equals_alone(setup):
    """The grouped variant over the same requests in one graph (products one
    after another, the library's own masks): each equal to its single grouped
    call."""
    p = setup
    sp = p.spfhe
    alone = []
    for r in p.reqs:
        hs, st = sp.spfhe_sparse_matmul_ct_ct_grouped(p.ctx, p.gkeys, r.Am, r.gA, r.Bm, r.gB, None, r.n_c)
        alone.append(([p.export_ct(p.track("ct", h)) for h in hs], st))
    reqs = [sp.matmul_req(p.gkeys, r.Am, r.gA, r.Bm, r.gB, None) for r in p.reqs]
    g = sp.spfhe_matmul_graph_create_batch(p.ctx, reqs, 1)
    try:
        sp.spfhe_matmul_graph_launch(g)
        sp.spfhe_sync(p.ctx)
        outs, stats = sp.spfhe_matmul_graph_results_batch(g, [r.n_c for r in p.reqs])
        for (want, st0), hs, st in zip(alone, outs, stats):
            for h, a in zip(hs, want):
                assert np.array_equal(p.export_ct(h), a)
                sp.spfhe_ct_free(h)
            for k in ("matches", "ks_relin", "ks_align", "ks_final", "rescales"):
                assert st[k] == st0[k]
    finally:
        sp.spfhe_matmul_graph_free(g)


def test_graph_batch_errors(setup):
    """A request without rotation keys fails the capture with EKEY and leaves
    the context usable; an empty request list is EINVAL."""
    p = setup
    sp = p.spfhe
    relin_only = p.track("keys", sp.spfhe_keys_import(p.ctx, p.keys.s, _ntt_key(p, p.keys.relin), {}))
    reqs = [_req(p, p.reqs[0]), _req(p, p.reqs[2], keys=relin_only)]
    with pytest.raises(sp.SpfheError) as e:
        sp.spfhe_matmul_graph_create_batch(p.ctx, reqs, 0)
    assert e.value.status == -4
    with pytest.raises(sp.SpfheError) as e:
        sp.spfhe_matmul_graph_create_batch(p.ctx, [], 0)
    assert e.value.status == -1
    r = p.reqs[1]
    hs, _ = sp.spfhe_sparse_matmul_ct_ct(p.ctx, p.gkeys, r.Am, r.gA, r.Bm, r.gB, r.gmask, r.n_c)
    for h, a in zip(hs, r.alone):
        assert np.array_equal(p.export_ct(p.track("ct", h)), a)


def test_server_isolates_a_failed_wave(setup):
    """A host-side injected failure in the waves of one request (no GPU fault:
    the engine raises SPFHE_ECUDA before launching that wave) fails only that
    request: the others, mixed into the same waves, are run again alone and
    return exactly the bits of their single calls; the server keeps serving
    requests submitted afterwards."""
    p = setup
    sp = p.spfhe
    srv = sp.spfhe_server_create(p.ctx, 1 << 30)
    try:
        sp.spfhe_server_inject_fault(srv, 2)   # the second request submitted
        tickets = [sp.spfhe_server_submit(srv, _req(p, r)) for r in p.reqs]
        assert tickets[1] == 2
        for i, (r, t) in enumerate(zip(p.reqs, tickets)):
            if i == 1:
                with pytest.raises(sp.SpfheError) as e:
                    sp.spfhe_server_wait(srv, t, r.n_c)
                assert e.value.status == -6 and "injected" in str(e.value)
                continue
            hs, st, lat = sp.spfhe_server_wait(srv, t, r.n_c)
            assert st["matches"] == r.stats["matches"]
            for h, a in zip(hs, r.alone):
                assert np.array_equal(p.export_ct(p.track("ct", h)), a)
        ws, in_use, retried = sp.spfhe_server_info(srv)
        assert retried >= 1 and in_use == 0 and ws > 0
        # a later request runs normally
        r = p.reqs[1]
        t = sp.spfhe_server_submit(srv, _req(p, r))
        hs, st, _ = sp.spfhe_server_wait(srv, t, r.n_c)
        for h, a in zip(hs, r.alone):
            assert np.array_equal(p.export_ct(p.track("ct", h)), a)
        with pytest.raises(sp.SpfheError):
            sp.spfhe_server_inject_fault(srv, t)   # already finished: unknown
    finally:
        sp.spfhe_server_destroy(srv)


def test_server_admission_budget_serialises(setup):
    """A budget below the shared batch buffers plus two requests admits one
    request at a time (each still admitted when nothing else runs); results
    stay bit-identical to the single calls."""
    p = setup
    sp = p.spfhe
    srv = sp.spfhe_server_create(p.ctx, 1)
    try:
        tickets = [sp.spfhe_server_submit(srv, _req(p, r)) for r in p.reqs]
        for r, t in zip(p.reqs, tickets):
            hs, st, _ = sp.spfhe_server_wait(srv, t, r.n_c)
            for h, a in zip(hs, r.alone):
                assert np.array_equal(p.export_ct(p.track("ct", h)), a)
        ws, in_use, retried = sp.spfhe_server_info(srv)
        assert in_use == 0 and retried == 0 and ws > 0
    finally:
        sp.spfhe_server_destroy(srv)
