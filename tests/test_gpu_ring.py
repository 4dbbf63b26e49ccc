"""GPU parity of the ring layer against the oracle, bit-exact on identical
keys, noise and inputs: parameters, NTT, encryption/decryption, tensor +
relinearisation, rescale, rotations through the plan, plaintext products.
Also the library's own key generation (functional and statistical checks:
its randomness is not shared with the oracle)."""
import numpy as np
import pytest

from oracle import ckks
from paper_2604_11659_gb300 import synthetic
from tests.gpu_util import Pair, need_gpu

pytestmark = pytest.mark.gpu

RECIPES = {
    "tiny": synthetic.ring_tiny(log_n=6, L=4, dnum=1, rot_base=2),
    "tiny_dnum3": synthetic.ring_tiny(log_n=7, L=6, dnum=3, rot_base=4),
    "n4096": synthetic.ring_small_16x16(),
}


@pytest.fixture(scope="module", params=list(RECIPES))
def pair(request):
    p = Pair(RECIPES[request.param])
    p.keys = p.o.keygen(5, rot_amounts=ckks.rotation_key_amounts(p.P.slots, p.P.rot_base))
    p.gkeys = p.import_keys(p.keys)
    yield p
    p.close()


def test_moduli_match_oracle(pair):
    mods, psis = pair.spfhe.spfhe_ctx_moduli(pair.ctx, pair.M)
    assert [int(x) for x in mods] == pair.P.mods
    assert [int(x) for x in psis] == pair.P.psis


@pytest.mark.parametrize("log_n,q_bits,split", [(2, [60, 40, 40], 0), (4, [60, 40, 40], 0), (10, [60, 45, 45], 0),
                                                (12, [60, 40, 40, 40], 0), (16, [60, 45, 45], 0),
                                                (16, [60, 45, 59, 57], 7), (16, [60, 45, 45], 9),
                                                (17, [60, 50, 50], 0), (17, [60, 50, 50], 9),
                                                (16, [60, 58, 56, 45], 0), (17, [60, 57, 58], 9)])
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6])
def test_ntt_forward_inverse_bit_exact(log_n, q_bits, split, variant):
    """Both butterfly paths (reduction-free below 2^58, or 2^57 for variant 5,
    bounded at and above), every pass split and kernel variant, against the
    oracle's transform; limb 1 holds q - 1 everywhere (the largest inputs)."""
    sp = need_gpu()
    import torch
    if variant and log_n < 12:
        pytest.skip("kernel variants apply to the two-pass radix-16 transform")
    recipe = synthetic.RingRecipe(log_n=log_n, q_bits=q_bits, dnum=1, scale_bits=40)
    p = Pair(recipe)
    try:
        sp.spfhe_ctx_set_ntt_split(p.ctx, split)
        sp.spfhe_ctx_set_ntt_variant(p.ctx, variant)
        n, M = p.n, p.M
        rng = np.random.default_rng(log_n)
        x = np.stack([rng.integers(0, m, n, dtype=np.uint64) for m in p.P.mods])
        x[0, :3] = [0, p.P.mods[0] - 1, 1]
        x[1, :] = p.P.mods[1] - 1
        mi = np.arange(M, dtype=np.int32)
        want = p.o.rns_ntt(x, mi)
        t = torch.from_numpy(x.view(np.int64)).cuda()
        sp.spfhe_ntt(p.ctx, t.data_ptr(), mi, inverse=False)
        sp.spfhe_sync(p.ctx)
        got = t.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want)
        sp.spfhe_ntt(p.ctx, t.data_ptr(), mi, inverse=True)
        sp.spfhe_sync(p.ctx)
        assert np.array_equal(t.cpu().numpy().view(np.uint64), x)
    finally:
        p.close()


@pytest.mark.parametrize("log_n,split", [(16, 0), (16, 7), (17, 0)])
@pytest.mark.parametrize("variant", [5, 6])
def test_ntt_many_limbs_bit_exact(log_n, split, variant):
    """256 limbs in one launch (4096 to 8192 CTAs per pass, several waves of
    resident CTAs, limbs of different moduli side by side, both butterfly
    paths); limb l holds input row l mod 4 under modulus l mod 4, so every
    limb is checked against one of the oracle's four transforms."""
    sp = need_gpu()
    import torch
    recipe = synthetic.RingRecipe(log_n=log_n, q_bits=[60, 45, 59, 57], dnum=1, scale_bits=40)
    p = Pair(recipe)
    try:
        sp.spfhe_ctx_set_ntt_split(p.ctx, split)
        sp.spfhe_ctx_set_ntt_variant(p.ctx, variant)
        n, M = p.n, p.M
        rng = np.random.default_rng(100 + log_n)
        x = np.stack([rng.integers(0, m, n, dtype=np.uint64) for m in p.P.mods])
        x[2, :] = p.P.mods[2] - 1
        want = p.o.rns_ntt(x, np.arange(M, dtype=np.int32))
        nl = 256
        mi = (np.arange(nl) % M).astype(np.int32)
        xs = x[mi]
        t = torch.from_numpy(xs.view(np.int64)).cuda()
        sp.spfhe_ntt(p.ctx, t.data_ptr(), mi, inverse=False)
        sp.spfhe_sync(p.ctx)
        got = t.cpu().numpy().view(np.uint64)
        bad = [l for l in range(nl) if not np.array_equal(got[l], want[mi[l]])]
        assert not bad, "limbs differ from the oracle: %s" % bad[:8]
        sp.spfhe_ntt(p.ctx, t.data_ptr(), mi, inverse=True)
        sp.spfhe_sync(p.ctx)
        assert np.array_equal(t.cpu().numpy().view(np.uint64), xs)
    finally:
        p.close()


def test_decrypt_bit_exact(pair):
    o, P = pair.o, pair.P
    rng = np.random.default_rng(1)
    z = rng.uniform(-1, 1, P.slots)
    ct = o.encrypt(o.encode(z, P.L, P.scale), pair.keys, rng)
    h = pair.import_ct(ct)
    pt = pair.track("pt", pair.spfhe.spfhe_decrypt(pair.ctx, pair.gkeys, h))
    got = pair.spfhe.spfhe_pt_export(pair.ctx, pt, pair.n)
    assert np.array_equal(got, o.rns_ntt(o.decrypt(ct, pair.keys).m))
    dec = pair.spfhe.spfhe_decode(pair.ctx, pt, P.slots).real
    assert np.max(np.abs(dec - z)) < 1e-6


def test_mult_relin_rescale_bit_exact(pair):
    o, P = pair.o, pair.P
    rng = np.random.default_rng(2)
    a = o.encrypt(o.encode(rng.uniform(-1, 1, P.slots), P.L, P.scale), pair.keys, rng)
    b = o.encrypt(o.encode(rng.uniform(-1, 1, P.slots), P.L, P.scale), pair.keys, rng)
    want = o.mult_relin(a, b, pair.keys)
    h = pair.track("ct", pair.spfhe.spfhe_mult_relin(pair.ctx, pair.gkeys, pair.import_ct(a), pair.import_ct(b)))
    pair.assert_ct_equal(h, want)
    pair.spfhe.spfhe_rescale(pair.ctx, h)
    pair.assert_ct_equal(h, o.rescale(want))


def test_keyswitch_at_every_level(pair):
    """Relinearisation at each level ell < L (digit groups truncate)."""
    o, P = pair.o, pair.P
    rng = np.random.default_rng(3)
    for ell in range(P.L, 0, -1):
        a = o.encrypt(o.encode(rng.uniform(-1, 1, P.slots), ell, P.scale), pair.keys, rng)
        want = o.mult_relin(a, a, pair.keys)
        ha = pair.import_ct(a)
        h = pair.track("ct", pair.spfhe.spfhe_mult_relin(pair.ctx, pair.gkeys, ha, ha))
        pair.assert_ct_equal(h, want)


@pytest.mark.parametrize("chunk", [1, 3, 7, 64])
def test_ntt_chunks_do_not_change_bits(pair, chunk):
    """Cutting the transform batches into launch pairs of `chunk` limbs
    (splitting items and limb maps) leaves every key switch bit-exact."""
    o, P = pair.o, pair.P
    rng = np.random.default_rng(11)
    a = o.encrypt(o.encode(rng.uniform(-1, 1, P.slots), P.L, P.scale), pair.keys, rng)
    want = o.mult_relin(a, a, pair.keys)
    want_rot = o.rotate(a, 3, pair.keys)
    sp = pair.spfhe
    sp.spfhe_ctx_set_ntt_chunk(pair.ctx, chunk)
    try:
        ha = pair.import_ct(a)
        pair.assert_ct_equal(pair.track("ct", sp.spfhe_mult_relin(pair.ctx, pair.gkeys, ha, ha)), want)
        pair.assert_ct_equal(pair.track("ct", sp.spfhe_rotate(pair.ctx, pair.gkeys, ha, 3)), want_rot)
    finally:
        sp.spfhe_ctx_set_ntt_chunk(pair.ctx, 0)


def test_ntt_chunk_tuner_picks_a_candidate(pair):
    sp = pair.spfhe
    cands = [0, 5, 64]
    best, ms = sp.spfhe_tune_ntt_chunk(pair.ctx, pair.P.L - 1, 4, cands)
    try:
        assert best in cands and len(ms) == 3 and all(t > 0 for t in ms)
        assert ms[cands.index(best)] == min(ms)
    finally:
        sp.spfhe_ctx_set_ntt_chunk(pair.ctx, 0)


@pytest.mark.parametrize("r", [1, 3, 5, 17, -1, -7, 1000, 31])
def test_rotate_plan_bit_exact(pair, r):
    o, P = pair.o, pair.P
    rng = np.random.default_rng(100 + r)
    z = rng.uniform(-1, 1, P.slots)
    ct = o.encrypt(o.encode(z, P.L - 1, P.scale), pair.keys, rng)
    want = o.rotate(ct, r, pair.keys)
    h = pair.track("ct", pair.spfhe.spfhe_rotate(pair.ctx, pair.gkeys, pair.import_ct(ct), r))
    pair.assert_ct_equal(h, want)


def test_mul_plain_and_add_bit_exact(pair):
    o, P = pair.o, pair.P
    rng = np.random.default_rng(4)
    ct = o.encrypt(o.encode(rng.uniform(-1, 1, P.slots), P.L, P.scale), pair.keys, rng)
    pt = o.encode_onehot(0.5, 3, P.L, float(P.q[-1]))
    h = pair.track("ct", pair.spfhe.spfhe_mul_plain(pair.ctx, pair.import_ct(ct), pair.import_pt(pt)))
    pair.assert_ct_equal(h, o.mul_plain(ct, pt))
    s = pair.track("ct", pair.spfhe.spfhe_add(pair.ctx, pair.import_ct(ct), pair.import_ct(ct)))
    pair.assert_ct_equal(s, o.add(ct, ct))


def test_encode_matches_oracle_within_one(pair):
    o, P = pair.o, pair.P
    z = np.random.default_rng(6).uniform(-1, 1, P.slots)
    pt = pair.track("pt", pair.spfhe.spfhe_encode(pair.ctx, z, P.L, P.scale))
    got = pair.spfhe.spfhe_pt_export(pair.ctx, pt, pair.n)
    want = o.rns_ntt(o.encode(z, P.L, P.scale).m)
    # compare in the coefficient domain: the encoders may differ by one unit
    # where a value lands on a rounding tie
    gc = o.rns_intt(got)[0].astype(object)
    wc = o.rns_intt(want)[0].astype(object)
    q0 = P.q[0]
    d = [((int(a) - int(b) + q0 // 2) % q0) - q0 // 2 for a, b in zip(gc, wc)]
    assert max(abs(x) for x in d) <= 1


def test_library_keygen_functional_and_noise(pair):
    sp, P, o = pair.spfhe, pair.P, pair.o
    keys = pair.track("keys", sp.spfhe_keygen(pair.ctx, 1234))
    rng = np.random.default_rng(7)
    z = rng.uniform(-1, 1, P.slots)
    w = rng.uniform(-1, 1, P.slots)
    ca = pair.track("ct", sp.spfhe_encrypt(pair.ctx, keys, pair.track("pt", sp.spfhe_encode(pair.ctx, z, P.L, P.scale)), 1))
    cb = pair.track("ct", sp.spfhe_encrypt(pair.ctx, keys, pair.track("pt", sp.spfhe_encode(pair.ctx, w, P.L, P.scale)), 2))
    dec = sp.spfhe_decode(pair.ctx, pair.track("pt", sp.spfhe_decrypt(pair.ctx, keys, ca)), P.slots).real
    assert np.max(np.abs(dec - z)) < 1e-6
    m = pair.track("ct", sp.spfhe_mult_relin(pair.ctx, keys, ca, cb))
    sp.spfhe_rescale(pair.ctx, m)
    dec = sp.spfhe_decode(pair.ctx, pair.track("pt", sp.spfhe_decrypt(pair.ctx, keys, m)), P.slots).real
    assert np.max(np.abs(dec - z * w)) < 1e-5
    r = pair.track("ct", sp.spfhe_rotate(pair.ctx, keys, ca, 5))
    dec = sp.spfhe_decode(pair.ctx, pair.track("pt", sp.spfhe_decrypt(pair.ctx, keys, r)), P.slots).real
    assert np.max(np.abs(dec - np.roll(z, -5))) < 1e-5
    # fresh-encryption noise of an encryption of zero: |e| <= 19, std near 3.2
    zero = pair.track("pt", sp.spfhe_encode(pair.ctx, np.zeros(1), P.L, P.scale))
    cz = pair.track("ct", sp.spfhe_encrypt(pair.ctx, keys, zero, 99))
    e = o.rns_intt(sp.spfhe_pt_export(pair.ctx, pair.track("pt", sp.spfhe_decrypt(pair.ctx, keys, cz)), pair.n))[0]
    q0 = P.q[0]
    ec = np.where(e > q0 // 2, -((np.uint64(q0) - e).astype(np.int64)), e.astype(np.int64))
    assert np.max(np.abs(ec)) <= 19
    if pair.n >= 4096:
        assert 2.6 < np.std(ec) < 3.8


def test_alu_peak_microbenchmarks():
    """The measured ALU speed of light: positive rates in a plausible range,
    and a lazy butterfly (nine 32-bit multiplies) slower than one 32-bit
    multiply-add."""
    sp = need_gpu()
    from paper_2604_11659_gb300 import params as gparams
    ctx = sp.spfhe_ctx_create(gparams.ctx_params(synthetic.ring_tiny(log_n=6, L=4, dnum=1, rot_base=2)))
    try:
        bfly, bfly_split, imad, wide = sp.spfhe_prof_alu_peak(ctx)
        assert 1e10 < bfly < 1e14 and 1e10 < bfly_split < 1e14 and 1e11 < imad < 1e15 and 1e11 < wide < 1e15
        assert max(bfly, bfly_split) < imad / 4
    finally:
        sp.spfhe_ctx_destroy(ctx)
