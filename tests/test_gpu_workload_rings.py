"""Parity at the rings of the batch and serving workloads, in the radix-16
launch configuration the benchmark runs (N = 2^16):

* batch ring (L = 20, dnum = 4, K = 4, rotation base 16): three few-match
  products of the batch recipe's shapes (d = 32, 64 with 2:4-structured rows,
  256 with a result over two ciphertext chunks) through one
  spfhe_sparse_matmul_batch call and through the batch captured as one CUDA
  graph;
* serving ring (L = 31, dnum = 4, K = 7, rotation base 16): four requests at
  operand levels 11, 16, 21 and 31 (remaining levels 10-30), each with its own
  key set, d from 64 to 512 (a result of eight chunks), through one batch call
  (four key sets in one call) and through the continuous-batching server.

Every result chunk is compared limb by limb with the oracle's Alg. 1 + Alg. 2
product on the same keys, noise and operands (the oracle needs about a second
per key switch at these sizes, so the products are crafted to have a few
matches each), and each product decrypts within 1e-4 of FP64.
"""
import os

import numpy as np
import pytest

from oracle import ckks, spmspm
from paper_2604_11659_gb300 import synthetic
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu


class Prod:
    pass


def _amounts(prods, S, base):
    amts = set()
    for r in prods:
        for a in spmspm.final_rotation_amounts(r.Acsr[:2], r.Bcsc[:2], r.rows, r.cols, S):
            amts.update(ckks.rotation_plan(a, S, base))
    return sorted(amts)


def _prepare(p, keysets, prods, seed):
    """Oracle operands, masks and expected chunks; the same imported into the
    library; the product alone through the library."""
    o, P, sp = p.o, p.P, p.spfhe
    rng = np.random.default_rng(seed)
    for r in prods:
        keys, gkeys = keysets[r.key_set]
        r.A_cts = [o.encrypt(o.encode(z, r.ell, P.scale), keys, rng) for z in spmspm.pack_values(r.Acsr[2], P.slots)]
        r.B_cts = [o.encrypt(o.encode(z, r.ell, P.scale), keys, rng) for z in spmspm.pack_values(r.Bcsc[2], P.slots)]
        r.mask = spmspm.make_mask(o, 0, r.ell - 1)
        counts = spmspm.OpCounts()
        r.want = spmspm.spmspm_ct_ct(o, keys, r.Acsr[:2], r.A_cts, r.Bcsc[:2], r.B_cts, r.rows, r.cols,
                                     mask_pt=r.mask, counts=counts)
        r.counts = counts
        r.gkeys = gkeys
        r.gA = [p.import_ct(c) for c in r.A_cts]
        r.gB = [p.import_ct(c) for c in r.B_cts]
        r.gmask = p.import_pt(r.mask)
        r.Am = sp.sparse_meta(r.Acsr[0], r.Acsr[1], r.rows, r.A.shape[1])
        r.Bm = sp.sparse_meta(r.Bcsc[0], r.Bcsc[1], r.B.shape[0], r.cols)
        r.n_c = max(1, -(-(r.rows * r.cols) // P.slots))
        assert len(r.want) == r.n_c
        C = spmspm.decrypt_result(o, keys, r.want, r.rows, r.cols)
        assert np.max(np.abs(C - r.A @ r.B)) < 1e-4


def _req(sp, r):
    return sp.matmul_req(r.gkeys, r.Am, r.gA, r.Bm, r.gB, r.gmask)


def _check(p, r, handles, stats=None):
    assert len(handles) == r.n_c
    for h, w in zip(handles, r.want):
        p.assert_ct_equal(p.track("ct", h), w)
    if stats is not None:
        assert stats["matches"] == r.counts.matches
        assert stats["ks_relin"] == r.counts.ks_relin
        assert stats["ks_align"] == r.counts.ks_align
        assert stats["ks_final"] == r.counts.ks_final


def _prod(A, B, ell, key_set=0):
    r = Prod()
    r.A, r.B, r.ell, r.key_set = A, B, ell, key_set
    r.rows, r.cols = A.shape[0], B.shape[1]
    r.Acsr, r.Bcsc = spmspm.dense_to_csr(A), spmspm.dense_to_csc(B)
    return r


# ---------------------------------------------------------------------------
# batch ring
# ---------------------------------------------------------------------------
def _batch_products(L):
    out = []
    A = np.zeros((32, 32))
    B = np.zeros((32, 32))
    A[1, 4], A[1, 9], A[20, 30] = 0.5, -0.3, 0.25
    B[4, 7], B[9, 2], B[30, 31] = 0.7, 0.2, -0.4
    out.append(_prod(A, B, L))
    # 2:4 rows (at most two nonzeros in every group of four), two matches
    # into one result slot
    A = np.zeros((64, 64))
    B = np.zeros((64, 64))
    A[0, 0], A[0, 1], A[9, 42], A[9, 43] = 0.6, -0.5, 0.3, 0.2
    B[0, 5], B[1, 5], B[42, 60], B[2, 7] = 0.3, 0.4, -0.7, 0.9
    out.append(_prod(A, B, L))
    # d = 256: a result of 65 536 slots (two chunks); (200, 250) lands in the second
    A = np.zeros((256, 256))
    B = np.zeros((256, 256))
    A[3, 100], A[200, 5] = 0.6, 0.4
    B[100, 10], B[5, 250] = 0.5, -0.9
    out.append(_prod(A, B, L))
    return out


@pytest.fixture(scope="module")
def batch_ring():
    ckks.threads(os.cpu_count() or 1)
    p = Pair(synthetic.ring_batch64(), rot_base=16)
    try:
        prods = _batch_products(p.P.L)
        keys = p.o.keygen(61, rot_amounts=_amounts(prods, p.P.slots, 16))
        _prepare(p, [(keys, p.import_keys(keys))], prods, 62)
        p.prods = prods
        yield p
    finally:
        p.close()


def test_batch_ring_parameters(batch_ring):
    P = batch_ring.P
    assert (P.n, P.L, P.dnum, P.K) == (1 << 16, 20, 4, 4)


def test_batch_ring_single_calls_bit_exact(batch_ring):
    p = batch_ring
    sp = p.spfhe
    for r in p.prods:
        hs, st = sp.spfhe_sparse_matmul_ct_ct(p.ctx, r.gkeys, r.Am, r.gA, r.Bm, r.gB, r.gmask, r.n_c)
        _check(p, r, hs, st)
    assert p.prods[2].n_c == 2


def test_batch_ring_batch_call_bit_exact(batch_ring):
    p = batch_ring
    sp = p.spfhe
    outs, stats = sp.spfhe_sparse_matmul_batch(p.ctx, [_req(sp, r) for r in p.prods], [r.n_c for r in p.prods])
    for r, hs, st in zip(p.prods, outs, stats):
        _check(p, r, hs, st)


def test_batch_ring_graph_bit_exact(batch_ring):
    p = batch_ring
    sp = p.spfhe
    g = sp.spfhe_matmul_graph_create_batch(p.ctx, [_req(sp, r) for r in p.prods], 0)
    try:
        for _ in range(2):
            sp.spfhe_matmul_graph_launch(g)
            sp.spfhe_sync(p.ctx)
            outs, stats = sp.spfhe_matmul_graph_results_batch(g, [r.n_c for r in p.prods])
            for r, hs, st in zip(p.prods, outs, stats):
                for h, w in zip(hs, r.want):
                    p.assert_ct_equal(h, w)
                    sp.spfhe_ct_free(h)   # the handle only: the chunks belong to the graph
                assert st["matches"] == r.counts.matches
    finally:
        sp.spfhe_matmul_graph_free(g)


# ---------------------------------------------------------------------------
# serving ring
# ---------------------------------------------------------------------------
def _serving_requests():
    out = []
    A = np.zeros((64, 64))
    B = np.zeros((64, 64))
    A[2, 7], A[40, 7] = 0.5, -0.25
    B[7, 3], B[7, 60] = 0.8, 0.4
    out.append(_prod(A, B, 11, 0))
    A = np.zeros((128, 128))
    B = np.zeros((128, 128))
    A[5, 17], A[5, 90] = 0.7, 0.3
    B[17, 100], B[90, 2] = -0.6, 0.5
    out.append(_prod(A, B, 21, 1))
    A = np.zeros((64, 64))
    B = np.zeros((64, 64))
    A[63, 0] = 0.9
    B[0, 63] = -0.8
    out.append(_prod(A, B, 31, 2))
    # d = 512: 262 144 result slots, eight chunks; matches in the first and the last
    A = np.zeros((512, 512))
    B = np.zeros((512, 512))
    A[1, 300], A[511, 12] = 0.4, 0.6
    B[300, 9], B[12, 500] = 0.5, -0.7
    out.append(_prod(A, B, 16, 3))
    return out


@pytest.fixture(scope="module")
def serving_ring():
    ckks.threads(os.cpu_count() or 1)
    p = Pair(synthetic.ring_serving(), rot_base=16)
    try:
        reqs = _serving_requests()
        keysets = []
        for k in range(4):
            mine = [r for r in reqs if r.key_set == k]
            keys = p.o.keygen(70 + k, rot_amounts=_amounts(mine, p.P.slots, 16))
            keysets.append((keys, p.import_keys(keys)))
        _prepare(p, keysets, reqs, 75)
        p.reqs = reqs
        yield p
    finally:
        p.close()


def test_serving_ring_parameters(serving_ring):
    P = serving_ring.P
    assert (P.n, P.L, P.dnum, P.K) == (1 << 16, 31, 4, 7)
    assert sorted(r.ell for r in serving_ring.reqs) == [11, 16, 21, 31]
    assert serving_ring.reqs[3].n_c == 8


def test_serving_ring_batch_call_four_key_sets(serving_ring):
    """Four requests at four levels with four key sets in one batch call."""
    p = serving_ring
    sp = p.spfhe
    outs, stats = sp.spfhe_sparse_matmul_batch(p.ctx, [_req(sp, r) for r in p.reqs], [r.n_c for r in p.reqs])
    for r, hs, st in zip(p.reqs, outs, stats):
        _check(p, r, hs, st)


def test_serving_ring_server_mix(serving_ring):
    """The four requests submitted together to the continuous-batching server
    (and two of them again afterwards): every result equal to the oracle's."""
    p = serving_ring
    sp = p.spfhe
    srv = sp.spfhe_server_create(p.ctx, 64 << 30)
    try:
        order = [3, 0, 2, 1, 0, 3]
        tickets = [sp.spfhe_server_submit(srv, _req(sp, p.reqs[i])) for i in order]
        for i, t in zip(order, tickets):
            r = p.reqs[i]
            hs, st, lat = sp.spfhe_server_wait(srv, t, r.n_c)
            assert lat > 0
            _check(p, r, hs, st)
    finally:
        sp.spfhe_server_destroy(srv)
