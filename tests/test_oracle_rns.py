"""Pins for the oracle's RNS primitives: basis conversion, rescale and the
Galois automorphism, checked with Python big integers and ring identities."""
import numpy as np
import pytest

from oracle import ckks


def _crt(residues, mods):
    """Chinese remaindering with Python ints (value in [0, prod))."""
    M = 1
    for m in mods:
        M *= m
    x = 0
    for r, m in zip(residues, mods):
        Mi = M // m
        x += int(r) * Mi * pow(Mi, -1, m)
    return x % M, M


def test_crt_round_trip_signed():
    mods = ckks.gen_primes(5, 40, 3)
    vals = [0, 1, -1, 12345678901234, -98765432109876, (1 << 100) + 7]
    for v in vals:
        res = [v % m for m in mods]
        x, M = _crt(res, mods)
        cen = x if x <= M // 2 else x - M
        assert cen == v


def test_bconv_is_x_plus_small_multiple_of_D():
    n = 16
    src = ckks.gen_primes(4, 45, 3)
    dst = ckks.gen_primes(4, 60, 2)
    rng = np.random.default_rng(3)
    x = np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in src])
    out = ckks.bconv(x, src, dst)
    D = src[0] * src[1] * src[2]
    for c in range(n):
        X, _ = _crt([x[i, c] for i in range(3)], src)
        us = set()
        for t, p in enumerate(dst):
            diff = (int(out[t, c]) - X) % p
            # diff = u*D mod p for a single 0 <= u < 3 shared by every target
            us.add(next(u for u in range(3) if (u * D) % p == diff))
        assert len(us) == 1


@pytest.mark.parametrize("ell", [2, 3, 5])
def test_rescale_is_rounded_division_by_top_prime(ell):
    P = ckks.make_params(4, [60] + [40] * (ell - 1), 1, 1, 2.0 ** 40)
    o = ckks.Oracle(P)
    n = P.n
    rng = np.random.default_rng(ell)
    c = np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in P.q[:ell]])
    # add a few values whose top residue sits at the centring boundary
    ct = ckks.Ct(c.copy(), c.copy(), 1.0)
    qt = P.q[ell - 1]
    ct.c0[ell - 1, 0] = qt // 2
    ct.c0[ell - 1, 1] = qt // 2 + 1
    out = o.rescale(ct)
    for k in range(n):
        X, _ = _crt([ct.c0[i, k] for i in range(ell)], P.q[:ell])
        r = X % qt
        if r > qt // 2:
            r -= qt
        Y = (X - r) // qt
        assert (X - r) % qt == 0
        for i in range(ell - 1):
            assert int(out.c0[i, k]) == Y % P.q[i]


def test_automorphism_monomials_and_homomorphism():
    log_n, n = 5, 32
    q = ckks.gen_primes(log_n, 50, 1)[0]
    psi = ckks.find_psi(q, log_n)
    for g in (5, 25, 2 * n - 1, 7):
        for j in range(n):
            e = np.zeros(n, np.uint64)
            e[j] = 3
            out = ckks.automorphism(e, g, q)
            t = (j * g) % (2 * n)
            want = np.zeros(n, np.uint64)
            if t < n:
                want[t] = 3
            else:
                want[t - n] = q - 3
            assert np.array_equal(out, want)
    rng = np.random.default_rng(0)
    a = rng.integers(0, q, n, dtype=np.uint64)
    b = rng.integers(0, q, n, dtype=np.uint64)
    for g in (5, 125 % (2 * n), 2 * n - 1):
        lhs = ckks.automorphism(ckks.polymul(a, b, log_n, q, psi), g, q)
        rhs = ckks.polymul(ckks.automorphism(a, g, q), ckks.automorphism(b, g, q), log_n, q, psi)
        assert np.array_equal(lhs, rhs)
    g, h = 5, 25
    assert np.array_equal(ckks.automorphism(ckks.automorphism(a, g, q), h, q),
                          ckks.automorphism(a, (g * h) % (2 * n), q))
    assert np.array_equal(ckks.automorphism(a, 1, q), a)


def test_centred_bconv_is_the_centred_representative():
    """or_bconv_centred returns [x]_D in [-D/2, D/2) reduced mod each target
    (checked with Python integers)."""
    import ctypes
    n = 64
    src = ckks.gen_primes(5, 60, 4)
    dst = ckks.gen_primes(5, 45, 3)
    rng = np.random.default_rng(11)
    x = np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in src])
    D = 1
    for q in src:
        D *= q
    # include values at the two ends of the centred range
    for c, X in ((0, D // 2 - 1), (1, D // 2), (2, D - 1), (3, 0)):
        for i, q in enumerate(src):
            x[i, c] = X % q
    out = np.zeros((len(dst), n), np.uint64)
    L = ckks.lib()
    L.or_bconv_centred.argtypes = [ckks.u64p, ckks.u64p, ctypes.c_int, ckks.u64p, ckks.u64p, ctypes.c_int, ctypes.c_int]
    s = np.array(src, np.uint64)
    d = np.array(dst, np.uint64)
    L.or_bconv_centred(ckks._p(x), ckks._p(s), len(src), ckks._p(out), ckks._p(d), len(dst), n)
    for c in range(n):
        X, _ = _crt([x[i, c] for i in range(len(src))], src)
        cen = X if X < D // 2 else X - D
        if c in (0, 1):
            # X/D within 2^-200 of one half: either representative is valid
            assert all(int(out[t, c]) in (cen % p, (cen + D) % p, (cen - D) % p) for t, p in enumerate(dst))
            continue
        assert [int(out[t, c]) for t in range(len(dst))] == [cen % p for p in dst]


def test_moddown_rounds_to_nearest():
    """Key switching output decrypts to c*s' + e with e zero-mean: the mean of
    the error over all coefficients is far below the floor+overflow bias
    (about (K-1)/2 * sum(s)) that an uncorrected conversion leaves."""
    from tests.oracle_util import oracle_params
    from paper_2604_11659_gb300 import synthetic
    P = oracle_params(synthetic.ring_tiny(log_n=10, L=4, dnum=1))
    o = ckks.Oracle(P)
    keys = o.keygen(2)
    rng = np.random.default_rng(4)
    s_rns = o.small_to_rns(keys.s)
    s2 = o.rns_polymul(s_rns, s_rns, np.arange(P.L + P.K, dtype=np.int32))
    errs = []
    for _ in range(4):
        c = np.stack([rng.integers(0, q, P.n, dtype=np.uint64) for q in P.q])
        k0, k1 = o.keyswitch(c, keys.relin)
        mi = np.arange(P.L, dtype=np.int32)
        got = (k0[0] + o.rns_polymul(k1, s_rns[: P.L], mi)[0]) % np.uint64(P.q[0])
        want = o.rns_polymul(c, s2[: P.L], mi)[0]
        q0 = P.q[0]
        errs.extend(((int(a) - int(b) + q0 // 2) % q0) - q0 // 2 for a, b in zip(got, want))
    errs = np.array(errs, dtype=np.float64)
    # zero-mean rounding: |mean| well inside a few standard errors
    assert abs(errs.mean()) < 5 * errs.std() / np.sqrt(errs.size)
