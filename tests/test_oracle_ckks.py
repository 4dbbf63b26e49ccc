"""Pins for the oracle's CKKS layer: encoding against the O(n S) definition,
the closed-form one-hot encoding, rotation semantics, key switching noise,
relinearisation against a direct s^2 decryption, and rescale."""
import numpy as np
import pytest

from oracle import ckks
from paper_2604_11659_gb300 import synthetic
from tests.oracle_util import oracle_params


@pytest.fixture(scope="module")
def small():
    P = oracle_params(synthetic.ring_tiny(log_n=6, L=4, dnum=1, rot_base=2))
    o = ckks.Oracle(P)
    keys = o.keygen(11, rot_amounts=ckks.rotation_key_amounts(P.slots, P.rot_base))
    return P, o, keys


def test_encode_fft_matches_definition():
    for log_n in (3, 5, 7):
        n = 1 << log_n
        rng = np.random.default_rng(log_n)
        z = rng.uniform(-1, 1, n // 2) + 1j * rng.uniform(-1, 1, n // 2)
        a = ckks.encode_coeffs(z, n, 2.0 ** 30)
        b = ckks.encode_coeffs_direct(z, n, 2.0 ** 30)
        assert np.max(np.abs(a - b)) <= 1
        assert np.mean(a == b) > 0.99


def test_decode_inverts_encode():
    n = 1 << 8
    z = np.random.default_rng(0).uniform(-1, 1, n // 2)
    m = ckks.encode_coeffs(z, n, 2.0 ** 40)
    q0 = ckks.gen_primes(8, 60, 1)[0]
    res = ckks.to_rns(m, [q0])[0]
    out = ckks.decode_coeffs(res, q0, 2.0 ** 40)
    assert np.max(np.abs(out - z)) < 1e-9


def test_slots_are_evaluations_at_5_powers():
    """decode(m) is m(zeta^(5^i)) / scale, evaluated directly for n = 16."""
    n = 16
    q0 = ckks.gen_primes(4, 60, 1)[0]
    m = np.array([3, -1, 4, 1, -5, 9, 2, -6, 5, 3, -5, 8, 9, -7, 9, 3])
    z = ckks.decode_coeffs(ckks.to_rns(m, [q0])[0], q0, 1.0)
    for i in range(n // 2):
        x = np.exp(1j * np.pi * pow(5, i, 2 * n) / n)
        assert abs(z[i] - sum(int(c) * x ** j for j, c in enumerate(m))) < 1e-9


@pytest.mark.parametrize("slot", [0, 1, 5, 17, 31])
def test_onehot_closed_form_equals_encoding(slot):
    n, S = 64, 32
    z = np.zeros(S)
    z[slot] = 0.7
    a = ckks.onehot_coeffs(0.7, slot, n, 2.0 ** 40)
    b = ckks.encode_coeffs_direct(z, n, 2.0 ** 40)
    assert np.max(np.abs(a - b)) <= 1
    # slot-p one-hot is exactly the automorphism X -> X^(5^-p) of slot 0's
    q = ckks.gen_primes(6, 60, 1)[0]
    g = pow(pow(5, slot, 2 * n), -1, 2 * n)
    base = ckks.to_rns(ckks.onehot_coeffs(0.7, 0, n, 2.0 ** 40), [q])[0]
    assert np.array_equal(ckks.automorphism(base, g, q), ckks.to_rns(a, [q])[0])


def test_encrypt_decrypt(small):
    P, o, keys = small
    rng = np.random.default_rng(5)
    z = rng.uniform(-1, 1, P.slots)
    ct = o.encrypt(o.encode(z, P.L, P.scale), keys, rng)
    assert np.max(np.abs(o.decode(o.decrypt(ct, keys)).real - z)) < 1e-9


@pytest.mark.parametrize("r", [1, 2, 3, 7, 13, 31, -1, -5])
def test_rotation_is_left_slot_shift(small, r):
    P, o, keys = small
    rng = np.random.default_rng(100 + r)
    z = rng.uniform(-1, 1, P.slots)
    ct = o.encrypt(o.encode(z, P.L, P.scale), keys, rng)
    out = o.decode(o.decrypt(o.rotate(ct, r, keys), keys)).real
    assert np.max(np.abs(out - np.roll(z, -r))) < 1e-6


def test_rotation_plan_digits():
    assert ckks.rotation_plan(0, 2048, 16) == []
    assert ckks.rotation_plan(1, 2048, 16) == [1]
    assert ckks.rotation_plan(0x5A3, 2048, 16) == [3, 0xA0, 0x500]
    assert ckks.rotation_plan(-1, 2048, 16) == [15, 15 * 16, 7 * 256]
    assert sum(ckks.rotation_plan(1234, 32768, 256)) == 1234
    amts = ckks.rotation_key_amounts(2048, 16)
    assert len(amts) == 15 + 15 + 7
    for r in range(0, 2048, 37):
        assert all(a in amts for a in ckks.rotation_plan(r, 2048, 16))


def test_keyswitch_noise_bound_multi_digit():
    """Key switching with dnum=3 at every level: decrypt(KS(c)) - c*s' has
    infinity norm within alpha*sqrt(n)*6*sigma*(D/P)*dnum + K*n (loose bound)."""
    P = oracle_params(synthetic.ring_tiny(log_n=6, L=6, dnum=3))
    o = ckks.Oracle(P)
    keys = o.keygen(3)
    rng = np.random.default_rng(9)
    s_rns = o.small_to_rns(keys.s)
    s2 = o.rns_polymul(s_rns, s_rns, np.arange(P.L + P.K, dtype=np.int32))
    for ell in (6, 5, 3, 1):
        c = np.stack([rng.integers(0, q, P.n, dtype=np.uint64) for q in P.q[:ell]])
        k0, k1 = o.keyswitch(c, keys.relin)
        mi = np.arange(ell, dtype=np.int32)
        got = [(int(a) + int(b)) % q for a, b, q in
               zip(k0[0], o.rns_polymul(k1, s_rns[:ell], mi)[0], [P.q[0]] * P.n)]
        want = o.rns_polymul(c, s2[:ell], mi)[0]
        q0 = P.q[0]
        err = [((g - int(w) + q0 // 2) % q0) - q0 // 2 for g, w in zip(got, want)]
        alpha = P.alpha
        D = max(np.prod([float(q) for q in P.q[j:j + alpha]]) for j in range(0, ell, alpha))
        Pp = np.prod([float(p) for p in P.p])
        bound = P.dnum * alpha * P.n * 6 * 3.2 * D / Pp + P.K * P.n + 1
        assert max(abs(e) for e in err) < bound


def test_relinearisation_matches_s2_decryption(small):
    P, o, keys = small
    rng = np.random.default_rng(21)
    z1 = rng.uniform(-1, 1, P.slots)
    z2 = rng.uniform(-1, 1, P.slots)
    c1 = o.encrypt(o.encode(z1, P.L, P.scale), keys, rng)
    c2 = o.encrypt(o.encode(z2, P.L, P.scale), keys, rng)
    d0, d1, d2, sc = o.tensor(c1, c2)
    s = o.small_to_rns(keys.s, P.L)
    mi = np.arange(P.L, dtype=np.int32)
    s2 = o.rns_polymul(s, s, mi)
    q0 = P.q[0]
    direct = (d0[0] + o.rns_polymul(d1, s, mi)[0] % np.uint64(q0)) % np.uint64(q0)
    direct = (direct + o.rns_polymul(d2, s2, mi)[0]) % np.uint64(q0)
    rel = o.decrypt(o.relinearize(d0, d1, d2, sc, keys), keys).m[0]
    diff = [((int(a) - int(b) + q0 // 2) % q0) - q0 // 2 for a, b in zip(rel, direct)]
    assert max(abs(x) for x in diff) < 10 ** 5
    out = o.decode(o.decrypt(o.rescale(o.relinearize(d0, d1, d2, sc, keys)), keys)).real
    assert np.max(np.abs(out - z1 * z2)) < 1e-6


def test_mask_isolates_one_slot(small):
    P, o, keys = small
    rng = np.random.default_rng(33)
    z = rng.uniform(-1, 1, P.slots)
    ct = o.rescale(o.mult_relin(o.encrypt(o.encode(z, P.L, P.scale), keys, rng),
                                o.encrypt(o.encode(np.ones(P.slots), P.L, P.scale), keys, rng), keys))
    m = o.encode_onehot(1.0, 9, ct.level, float(P.q[ct.level - 1]))
    out = o.decode(o.decrypt(o.rescale(o.mul_plain(ct, m)), keys)).real
    want = np.zeros(P.slots)
    want[9] = z[9]
    assert np.max(np.abs(out - want)) < 1e-6


def test_hoisted_rotations_decrypt_to_shifted_slots():
    """One ModUp shared by several rotation amounts (automorphism applied to
    the extended digits): each result decrypts to the left-shifted slots,
    within the noise of one key switch, like the plain rotation."""
    recipe = synthetic.ring_tiny(log_n=7, L=6, dnum=3, rot_base=4)
    P = oracle_params(recipe)
    o = ckks.Oracle(P)
    keys = o.keygen(3, rot_amounts=ckks.rotation_key_amounts(P.slots, P.rot_base))
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, P.slots)
    ct = o.encrypt(o.encode(z, P.L, P.scale), keys, rng)
    amounts = [1, 2, 3, 4, 8, 12, 16, 48]
    outs = o.rotate_hoisted(ct, amounts, keys)
    for r, h in zip(amounts, outs):
        got = np.real(o.decode(o.decrypt(h, keys)))
        assert np.max(np.abs(got - np.roll(z, -r))) < 1e-6
        plain = np.real(o.decode(o.decrypt(o.rotate_single(ct, r, keys), keys)))
        assert np.max(np.abs(got - plain)) < 1e-6
