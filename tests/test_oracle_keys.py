"""Pins for the oracle's key material and encryption: the switching-key
formula of hybrid key switching, secret-key encryption, and the three
samplers.

Switching key from s' to s, digit j, over every modulus m of q_0..q_{L-1},
p_0..p_{K-1}:  k_j = (-a_j s + e_j + g_j s', a_j) with g_j = P mod q_i on
the limbs q_i of digit j and 0 on every other modulus (P = prod p_k).  Here
k0 + k1 s - g_j s' is computed with integer negacyclic convolutions in Python
and must be, on every modulus, the centred residue of ONE small integer
polynomial e_j (|e| <= 6 sigma).  s' is s^2 for the relinearisation key and
sigma_g(s) = s(X^g), g = 5^r mod 2n, for the rotation key of r, both formed
here from the integer secret."""
import numpy as np
import pytest

from oracle import ckks
from paper_2604_11659_gb300 import synthetic
from tests.oracle_util import oracle_params

SIGMA = 3.2


def _negacyclic(a, b):
    n = len(a)
    c = [0] * n
    for i, ai in enumerate(a):
        if ai:
            for j, bj in enumerate(b):
                if i + j < n:
                    c[i + j] += ai * bj
                else:
                    c[i + j - n] -= ai * bj
    return c


def _galois(s, g):
    n = len(s)
    out = [0] * n
    for k, c in enumerate(s):
        e = (k * g) % (2 * n)
        if e < n:
            out[e] += c
        else:
            out[e - n] -= c
    return out


def _centred(x, m):
    x %= m
    return x - m if x > m // 2 else x


@pytest.fixture(scope="module")
def tiny():
    P = oracle_params(synthetic.ring_tiny(log_n=5, L=4, dnum=2, rot_base=2))
    o = ckks.Oracle(P)
    keys = o.keygen(17, rot_amounts=[3])
    return P, o, keys


def _check_key(P, s, key, s_new):
    Pprod = 1
    for pk in P.p:
        Pprod *= pk
    mods = P.mods
    assert key.shape == (P.dnum, 2, P.L + P.K, P.n)
    for j in range(P.dnum):
        digit = range(j * P.alpha, min((j + 1) * P.alpha, P.L))
        errs = []
        for i, m in enumerate(mods):
            k0 = [int(v) for v in key[j, 0, i]]
            k1 = [int(v) for v in key[j, 1, i]]
            assert max(k0) < m and max(k1) < m
            k1s = _negacyclic(k1, s)
            g = Pprod % m if i in digit else 0
            errs.append([_centred(k0[t] + k1s[t] - g * s_new[t], m) for t in range(P.n)])
        # one integer error polynomial, the same on every modulus, and small
        for e in errs[1:]:
            assert e == errs[0], j
        assert max(abs(v) for v in errs[0]) <= int(6 * SIGMA)
        assert any(errs[0])


@pytest.mark.parametrize("which", ["relin", "rot3"])
def test_switching_key_formula(tiny, which):
    P, o, keys = tiny
    s = [int(v) for v in keys.s]
    if which == "relin":
        _check_key(P, s, keys.relin, _negacyclic(s, s))
    else:
        _check_key(P, s, keys.rot[3], _galois(s, pow(5, 3, 2 * P.n)))


def _plant(P, key, s_new, kind):
    """A copy of the relinearisation key with one plausible mistake."""
    bad = key.copy()
    Pprod = 1
    for pk in P.p:
        Pprod *= pk
    for j in range(P.dnum):
        digit = range(j * P.alpha, min((j + 1) * P.alpha, P.L))
        for i, m in enumerate(P.mods):
            if kind == "gadget without P" and i in digit:
                delta = (1 - Pprod) % m
            elif kind == "gadget on every limb" and i not in digit and i < P.L:
                delta = Pprod % m
            else:
                continue
            bad[j, 0, i] = np.array([(int(k) + delta * v) % m for k, v in zip(bad[j, 0, i], s_new)], dtype=np.uint64)
    return bad


@pytest.mark.parametrize("kind", ["gadget without P", "gadget on every limb", "inverse rotation"])
def test_planted_key_mistakes_fail_the_pin(tiny, kind):
    P, o, keys = tiny
    s = [int(v) for v in keys.s]
    if kind == "inverse rotation":
        # the key of sigma_g checked as if it were the key of sigma_g^-1
        g_inv = pow(pow(5, 3, 2 * P.n), -1, 2 * P.n)
        with pytest.raises(AssertionError):
            _check_key(P, s, keys.rot[3], _galois(s, g_inv))
        return
    s2 = _negacyclic(s, s)
    with pytest.raises(AssertionError):
        _check_key(P, s, _plant(P, keys.relin, s2, kind), s2)


def test_samplers():
    P = oracle_params(synthetic.ring_tiny(log_n=12, L=3, dnum=1, rot_base=2))
    o = ckks.Oracle(P)
    rng = np.random.default_rng(5)
    n = P.n
    s = o.sample_secret(rng)
    vals, counts = np.unique(s, return_counts=True)
    assert vals.tolist() == [-1, 0, 1]
    # each value with probability 1/3: within five standard deviations
    sd = np.sqrt(n * (1 / 3) * (2 / 3))
    assert np.all(np.abs(counts - n / 3) < 5 * sd)
    e = np.concatenate([o.sample_error(rng) for _ in range(8)])
    assert e.dtype == np.int64 and np.max(np.abs(e)) <= int(6 * SIGMA)
    # rounded Gaussian: mean 0, variance sigma^2 + 1/12
    N = e.size
    assert abs(np.mean(e)) < 5 * SIGMA / np.sqrt(N)
    assert abs(np.var(e) - (SIGMA ** 2 + 1 / 12)) < 0.05 * SIGMA ** 2
    u = o.sample_uniform(rng, P.mods)
    for i, m in enumerate(P.mods):
        assert int(u[i].max()) < m
        assert abs(float(np.mean(u[i].astype(np.float64))) / m - 0.5) < 5 * np.sqrt(1 / 12 / n)


def test_encryption_formula(tiny):
    """Secret-key encryption (c0, c1) = (-a s + e + m, a): c0 + c1 s - m is
    one small integer error polynomial on every modulus of the level."""
    P, o, keys = tiny
    s = [int(v) for v in keys.s]
    rng = np.random.default_rng(8)
    pt = o.encode(rng.uniform(-1, 1, P.slots), P.L, P.scale)
    ct = o.encrypt(pt, keys, rng)
    errs = []
    for i, m in enumerate(P.mods[: P.L]):
        c1s = _negacyclic([int(v) for v in ct.c1[i]], s)
        errs.append([_centred(int(ct.c0[i][t]) + c1s[t] - int(pt.m[i][t]), m) for t in range(P.n)])
    for e in errs[1:]:
        assert e == errs[0]
    assert 0 < max(abs(v) for v in errs[0]) <= int(6 * SIGMA)
