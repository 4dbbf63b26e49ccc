"""Pins for the oracle's number theory and negacyclic NTT.

Each check compares the oracle with something other than itself: sympy's
primality test, evaluation of a(X) at the n roots of X^n + 1 by Horner's rule
in Python integers, and a negacyclic product computed from numpy's
convolution of integer arrays.
"""
import numpy as np
import pytest
import sympy

from oracle import ckks


def _brv(x, bits):
    return int(format(x, "0%db" % bits)[::-1], 2) if bits else 0


@pytest.mark.parametrize("log_n,bits", [(4, 40), (6, 45), (12, 60), (16, 50), (17, 60)])
def test_primes_are_the_first_ntt_friendly_below_2b(log_n, bits):
    two_n = 2 << log_n
    ps = ckks.gen_primes(log_n, bits, 3)
    assert len(set(ps)) == 3
    prev = 1 << bits
    for p in ps:
        assert sympy.isprime(p)
        assert p % two_n == 1 and p < (1 << bits)
        # no NTT-friendly prime skipped between the previous one and this one
        c = prev + 1 - two_n if prev == (1 << bits) else prev - two_n
        while c > p:
            assert not sympy.isprime(c)
            c -= two_n
        prev = p


def test_make_params_order_and_distinct():
    P = ckks.make_params(12, [60, 40, 40, 40], 3, 1, 2.0 ** 40)
    assert len(set(P.mods)) == 7
    assert P.q[0].bit_length() == 60 and all(q.bit_length() == 40 for q in P.q[1:])
    assert all(p.bit_length() == 60 for p in P.p)
    assert P.q[1] > P.q[2] > P.q[3]
    assert P.q[0] > P.p[0] > P.p[1] > P.p[2]


@pytest.mark.parametrize("log_n", [1, 3, 6, 12, 16])
def test_psi_is_primitive_2n_root_and_first_candidate(log_n):
    n = 1 << log_n
    q = ckks.gen_primes(log_n, 50, 1)[0]
    psi = ckks.find_psi(q, log_n)
    assert pow(psi, n, q) == q - 1 and pow(psi, 2 * n, q) == 1
    for x in range(2, 100):
        cand = pow(x, (q - 1) // (2 * n), q)
        if pow(cand, n, q) == q - 1:
            assert cand == psi
            break


def _eval_at_roots(a, log_n, q, psi):
    """a(x_k) for x_k = psi^(2 brv(k) + 1), Horner's rule in Python ints."""
    n = 1 << log_n
    out = []
    for k in range(n):
        x = pow(psi, 2 * _brv(k, log_n) + 1, q)
        acc = 0
        for c in reversed([int(v) for v in a]):
            acc = (acc * x + c) % q
        out.append(acc)
    return np.array(out, dtype=np.uint64)


@pytest.mark.parametrize("log_n", [1, 2, 3, 5, 7])
def test_ntt_is_evaluation_at_roots_of_xn_plus_1(log_n):
    n = 1 << log_n
    q = ckks.gen_primes(log_n, 60, 1)[0]
    psi = ckks.find_psi(q, log_n)
    roots = {pow(psi, 2 * _brv(k, log_n) + 1, q) for k in range(n)}
    assert len(roots) == n and all(pow(x, n, q) == q - 1 for x in roots)
    rng = np.random.default_rng(log_n)
    for a in (rng.integers(0, q, n, dtype=np.uint64), np.full(n, q - 1, np.uint64),
              np.zeros(n, np.uint64), np.eye(1, n, n - 1, dtype=np.uint64)[0]):
        ref = _eval_at_roots(a, log_n, q, psi)
        assert np.array_equal(ckks.ntt_direct(a, log_n, q, psi), ref)
        assert np.array_equal(ckks.ntt_fwd(a, log_n, q, psi), ref)


@pytest.mark.parametrize("log_n,bits", [(4, 40), (8, 60), (10, 45), (12, 60)])
def test_intt_inverts_ntt(log_n, bits):
    n = 1 << log_n
    q = ckks.gen_primes(log_n, bits, 1)[0]
    psi = ckks.find_psi(q, log_n)
    a = np.random.default_rng(1).integers(0, q, n, dtype=np.uint64)
    assert np.array_equal(ckks.ntt_inv(ckks.ntt_fwd(a, log_n, q, psi), log_n, q, psi), a)


def _negacyclic_numpy(a, b, q):
    """Integer convolution (numpy object arrays) folded by X^n = -1."""
    n = len(a)
    full = np.convolve(np.array([int(x) for x in a], dtype=object),
                       np.array([int(x) for x in b], dtype=object))
    res = [0] * n
    for k, v in enumerate(full):
        if k < n:
            res[k] += v
        else:
            res[k - n] -= v
    return np.array([x % q for x in res], dtype=np.uint64)


@pytest.mark.parametrize("log_n,bits", [(3, 40), (6, 60), (8, 50)])
def test_polymul_equals_negacyclic_convolution(log_n, bits):
    n = 1 << log_n
    q = ckks.gen_primes(log_n, bits, 1)[0]
    psi = ckks.find_psi(q, log_n)
    rng = np.random.default_rng(log_n + bits)
    a = rng.integers(0, q, n, dtype=np.uint64)
    b = rng.integers(0, q, n, dtype=np.uint64)
    ref = _negacyclic_numpy(a, b, q)
    assert np.array_equal(ckks.negacyclic_schoolbook(a, b, q), ref)
    assert np.array_equal(ckks.polymul(a, b, log_n, q, psi), ref)


def test_polymul_by_x_is_negacyclic_shift():
    log_n, n = 5, 32
    q = ckks.gen_primes(log_n, 40, 1)[0]
    psi = ckks.find_psi(q, log_n)
    a = np.arange(1, n + 1, dtype=np.uint64)
    x = np.zeros(n, np.uint64)
    x[1] = 1
    out = ckks.polymul(a, x, log_n, q, psi)
    assert out[0] == q - a[-1] and np.array_equal(out[1:], a[:-1])
