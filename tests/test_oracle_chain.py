"""Pin for the oracle's Alg. 1 + Alg. 2 chain, one intermediate at a time.

On a tiny ring (n = 2^5, S = 16 slots, d = 3) every intermediate of every
match -- the aligned operands, the tensor product (three components, decrypted
with s and s^2), the relinearised product, both rescales, the masked product,
the final rotation and the running sum -- is decrypted here with a full CRT
over all active limbs in Python integers and decoded by the direct slot sum
m(zeta^(5^i)) / scale.  Each must hold the slot vector the paper's steps
describe:
  * alignment (Alg. 1): the operand whose nonzero sits at the larger slot is
    rotated left by the slot difference;
  * EvalMult / Relinearize (Alg. 2): slot-wise product, scale Delta^2;
  * Rescale: same slots, scale divided by the dropped prime;
  * makeMask + EvalMult: only slot min_pos survives;
  * EvalRotate(min_pos - (i*size + j)): the value lands in slot i*size + j;
  * EvalAdd: the result holds C = A B.
The traced chain ends bit-identical to spmspm_ct_ct, so this pins the
oracle's own sequence, and the q_0-only decode (reading G9) agrees with the
full-CRT decode at every step whose message fits in q_0 (all but the
Delta^2-scaled products before the first rescale)."""
import numpy as np
import pytest

from oracle import ckks, spmspm
from paper_2604_11659_gb300 import synthetic
from tests.oracle_util import oracle_params

TOL = 1e-6


def _crt(limbs, mods):
    """Centred integer of each coefficient from its residues (Python ints)."""
    Q = 1
    for q in mods:
        Q *= q
    out = []
    for j in range(limbs.shape[1]):
        x = 0
        for i, q in enumerate(mods):
            Qi = Q // q
            x += int(limbs[i, j]) * Qi * pow(Qi, -1, q)
        x %= Q
        if x > Q // 2:
            x -= Q
        out.append(x)
    return out, Q


def _negacyclic(a, b):
    n = len(a)
    c = [0] * n
    for i, ai in enumerate(a):
        if ai == 0:
            continue
        for j, bj in enumerate(b):
            k = i + j
            if k < n:
                c[k] += ai * bj
            else:
                c[k - n] -= ai * bj
    return c


def _decrypt_full(comps, s, mods):
    """sum_k c_k s^k over Z, reduced centred mod Q_ell (the product of the
    active limbs); comps are RNS polynomials (limbs, n)."""
    polys = [_crt(np.asarray(c), mods)[0] for c in comps]
    Q = 1
    for q in mods:
        Q *= q
    s_int = [int(v) for v in s]
    acc = list(polys[0])
    s_pow = s_int
    for k in range(1, len(polys)):
        term = _negacyclic(polys[k], s_pow)
        acc = [x + y for x, y in zip(acc, term)]
        if k + 1 < len(polys):
            s_pow = _negacyclic(s_pow, s_int)
    out = []
    for x in acc:
        x %= Q
        if x > Q // 2:
            x -= Q
        out.append(x)
    return out


def _slots(m, scale):
    n = len(m)
    zeta = np.exp(1j * np.pi / n)
    return np.array([sum(float(c) * zeta ** (pow(5, i, 2 * n) * j % (2 * n)) for j, c in enumerate(m))
                     for i in range(n // 2)]) / scale


def _check(o, keys, comps, scale, want, what):
    ell = np.asarray(comps[0]).shape[0]
    mods = o.mods[:ell]
    m = _decrypt_full(comps, keys.s, mods)
    got = _slots(m, scale)
    assert np.max(np.abs(got - want)) < TOL, what
    # the q_0-only decode holds while |m| < q_0 / 2 (not at scale Delta^2)
    if len(comps) == 2 and scale * (np.max(np.abs(want)) + 1.0) < mods[0] / 4:
        fast = np.real(o.decode(o.decrypt(ckks.Ct(np.asarray(comps[0]), np.asarray(comps[1]), scale), keys)))
        assert np.max(np.abs(fast - np.real(got))) < 1e-9, what + " (q_0-only decode)"


def _left(v, r):
    return np.roll(v, -r)


def _trace_chain(seed, o=None, make_mask=spmspm.make_mask):
    """Walks every match of a 3x3 product through the oracle's steps and
    checks each intermediate; raises AssertionError at the first mismatch."""
    if o is None:
        o = ckks.Oracle(oracle_params(synthetic.ring_tiny(log_n=5, L=4, dnum=1, rot_base=2)))
    P = o.P
    S, d = P.slots, 3
    rng = np.random.default_rng(seed)
    A = synthetic.bernoulli_sparse(rng, d, d, 0.4)
    B = synthetic.bernoulli_sparse(rng, d, d, 0.4)
    A = synthetic.rescale_rows_to_unit_output(A, B)
    Aip, Aix, Ad = spmspm.dense_to_csr(A)
    Bip, Bix, Bd = spmspm.dense_to_csc(B)
    keys = o.keygen(seed, rot_amounts=ckks.rotation_key_amounts(S, P.rot_base))
    erng = np.random.default_rng(seed + 100)
    za, zb = spmspm.pack_values(Ad, S)[0], spmspm.pack_values(Bd, S)[0]
    ctA = o.encrypt(o.encode(za, P.L, P.scale), keys, erng)
    ctB = o.encrypt(o.encode(zb, P.L, P.scale), keys, erng)
    _check(o, keys, (ctA.c0, ctA.c1), ctA.scale, za, "fresh A")
    _check(o, keys, (ctB.c0, ctB.c1), ctB.scale, zb, "fresh B")

    matches = spmspm.alg1_matches(Aip, Aix, Bip, Bix, d, d)
    assert len(matches) >= 3
    result = o.zero_ct(P.L - 2, spmspm.result_scale(o))
    want_sum = np.zeros(S)
    aligned_any = False
    for mt in matches:
        sa, sb = mt.a_pos, mt.b_pos
        vA, vB, wa, wb = ctA, ctB, za, zb
        if sa < sb:
            vB, wb = o.rotate(ctB, sb - sa, keys), _left(zb, sb - sa)
            _check(o, keys, (vB.c0, vB.c1), vB.scale, wb, "aligned B")
        elif sb < sa:
            vA, wa = o.rotate(ctA, sa - sb, keys), _left(za, sa - sb)
            _check(o, keys, (vA.c0, vA.c1), vA.scale, wa, "aligned A")
        aligned_any |= sa != sb
        min_slot = min(sa, sb)
        assert wa[min_slot] == A[mt.i, mt.k] and wb[min_slot] == B[mt.k, mt.j]
        d0, d1, d2, sc = o.tensor(vA, vB)
        assert sc == P.scale * P.scale
        _check(o, keys, (d0, d1, d2), sc, wa * wb, "tensor (decrypted with s, s^2)")
        dot = o.relinearize(d0, d1, d2, sc, keys)
        _check(o, keys, (dot.c0, dot.c1), dot.scale, wa * wb, "relinearised")
        dot = o.rescale(dot)
        assert dot.scale == sc / o.mods[P.L - 1]
        _check(o, keys, (dot.c0, dot.c1), dot.scale, wa * wb, "first rescale")
        dot = o.mul_plain(dot, make_mask(o, min_slot, dot.level))
        one = np.zeros(S)
        one[min_slot] = wa[min_slot] * wb[min_slot]
        _check(o, keys, (dot.c0, dot.c1), dot.scale, one, "masked")
        dot = o.rescale(dot)
        assert dot.level == P.L - 2
        _check(o, keys, (dot.c0, dot.c1), dot.scale, one, "second rescale")
        t = mt.i * d + mt.j
        dot = o.rotate(dot, (min_slot - t) % S, keys)
        placed = _left(one, (min_slot - t) % S)
        assert placed[t] == A[mt.i, mt.k] * B[mt.k, mt.j] and np.count_nonzero(placed) <= 1
        _check(o, keys, (dot.c0, dot.c1), dot.scale, placed, "final rotation")
        result = o.add(result, dot)
        want_sum = want_sum + placed
        _check(o, keys, (result.c0, result.c1), result.scale, want_sum, "accumulated")
    assert aligned_any
    C = (A @ B).reshape(-1)
    assert np.max(np.abs(want_sum[: d * d] - C)) < 1e-12
    # the traced chain is the oracle's own
    ref = spmspm.spmspm_ct_ct(o, keys, (Aip, Aix), [ctA], (Bip, Bix), [ctB], d, d)[0]
    assert np.array_equal(ref.c0, result.c0) and np.array_equal(ref.c1, result.c1)


@pytest.mark.parametrize("seed", [3, 12])
def test_alg2_chain_intermediates_by_full_crt(seed):
    _trace_chain(seed)


def _mutant(kind):
    o = ckks.Oracle(oracle_params(synthetic.ring_tiny(log_n=5, L=4, dnum=1, rot_base=2)))
    S = o.P.slots
    make_mask = spmspm.make_mask
    if kind == "rotation to the right":
        rot = o.rotate
        o.rotate = lambda ct, r, keys: rot(ct, (-r) % S, keys)
    elif kind == "rescale keeps the scale":
        rs = o.rescale
        o.rescale = lambda ct: ckks.Ct(rs(ct).c0, rs(ct).c1, ct.scale)
    elif kind == "tensor without a cross term":
        ts = o.tensor
        o.tensor = lambda x, y: (lambda t: (t[0], o.rns_polymul(x.c0, y.c1, o._mi(x.level)), t[2], t[3]))(ts(x, y))
    elif kind == "mask one slot off":
        make_mask = lambda orc, slot, level: spmspm.make_mask(orc, (slot + 1) % S, level)
    elif kind == "relinearisation key of the wrong secret power":
        rl = o.relinearize
        o.relinearize = lambda d0, d1, d2, sc, keys: rl(d0, d2, d1, sc, keys)
    return o, make_mask


@pytest.mark.parametrize("kind", ["rotation to the right", "rescale keeps the scale", "tensor without a cross term",
                                  "mask one slot off", "relinearisation key of the wrong secret power"])
def test_planted_mistakes_fail_the_chain_pin(kind):
    """Each plausible mistake, planted in the oracle, is caught."""
    o, make_mask = _mutant(kind)
    with pytest.raises(AssertionError):
        _trace_chain(3, o=o, make_mask=make_mask)
