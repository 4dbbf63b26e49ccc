"""Plain CPU oracle for the encrypted sparse x sparse matmul (CKKS SpMSpM).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline leg; never by the product package.  It shares no code
with the CUDA library.

What it computes, in the paper's order:
  * Alg. 1 (Sec. 3): CSR(A) x CSC(B) merge over every (i, j); on a match the
    operand whose nonzero sits at the larger slot is rotated left by the slot
    difference, nothing is rotated when the slots agree (Sec. 3.2.2).
  * Alg. 2 (Sec. 3.3): EvalMult -> Relinearize -> Rescale -> makeMask ->
    EvalMult(mask) -> Relinearize (a no-op on a 2-component product) ->
    Rescale -> EvalRotate(min_pos - (i*size + j)) -> EvalAdd into the result.
  * a plain RNS-CKKS (Sec. 2.1 names the scheme; the paper fixes no
    parameters) underneath: encode/decode by the canonical embedding,
    secret-key encryption, hybrid key switching, rescale, Galois rotations.
  * the FP64 product A @ B, the "baseline correct solution" of Sec. 4.2.

Ring elements are numpy uint64 arrays of shape (limbs, n) in the
COEFFICIENT domain.  Random draws (secret, masks a, errors e) come from a
numpy Generator seeded by the caller; they are inputs, and are exported with
the keys so that another implementation can be fed the same values.

Readings of points the paper leaves open:
  R1 special primes K raised to ceil(bits(largest digit)/60) (hybrid key
     switching needs P >= the digit modulus; dnum kept as configured);
  R2 primes q = 1 mod 2n searched downward from 2^b; psi the first
     x^((q-1)/2n), x = 2, 3, ..., with psi^n = -1;
  R3 packing: CSR data[p] (A) and CSC data[p] (B) in slot p mod S of chunk
     p // S, result C[i, j] in slot t mod S of chunk t // S, t = i*ncols + j;
  R4 EvalRotate(v, r) is a left rotation (slot r moves to slot 0), realised
     as the automorphism X -> X^(5^r mod 2n) followed by key switching;
  R5 rotation amounts are applied through a plan: r mod S written in base
     b = rot_base, one key switch per nonzero digit d*b^t, ascending t;
  R6 the mask of Alg. 2 is encoded at scale q_{L-2} (the prime the second
     rescale removes) so every product ends at scale Delta^2/q_{L-1};
  R7 Relinearize after the mask product is a no-op;
  R8 encode: m_j = round_half_away((2*Delta/n) Re sum_i z_i zeta^(-5^i j));
     one-hot encodings are evaluated in closed form with the angle reduced
     exactly: Re zeta^(-5^p j) = (-1)^floor(t/n) cos(pi (t mod n)/n),
     t = 5^p j mod 2n;
  R9 ct x pt variant: B's value is encoded straight into slot a_slot at scale
     q_{L-1} (alignment of B becomes re-encoding; the mask merges into the
     weight plaintext), then rescale, final rotation, add: depth 1;
  R10 Alg. 1's loop bounds "0 to N" are read as i < rows, j < cols;
  R11 the empty product (no match) is the all-zero ciphertext at level L-2.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

u64p = ctypes.POINTER(ctypes.c_uint64)
MAXMODS = 96


class _OrParams(ctypes.Structure):
    _fields_ = [
        ("log_n", ctypes.c_int),
        ("L", ctypes.c_int),
        ("K", ctypes.c_int),
        ("dnum", ctypes.c_int),
        ("mods", ctypes.c_uint64 * MAXMODS),
        ("psis", ctypes.c_uint64 * MAXMODS),
    ]


_lib = None


def lib():
    """Load (building if needed) the C part of the oracle."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u64 = ctypes.c_uint64
        L.or_powmod.restype = u64
        L.or_powmod.argtypes = [u64, u64, u64]
        L.or_invmod.restype = u64
        L.or_invmod.argtypes = [u64, u64]
        L.or_is_prime.restype = ctypes.c_int
        L.or_is_prime.argtypes = [u64]
        L.or_gen_primes.restype = ctypes.c_int
        L.or_gen_primes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p, ctypes.c_int, u64p]
        L.or_find_psi.restype = u64
        L.or_find_psi.argtypes = [u64, ctypes.c_int]
        for name in ("or_ntt_fwd", "or_ntt_inv"):
            getattr(L, name).argtypes = [u64p, ctypes.c_int, u64, u64]
            getattr(L, name).restype = None
        L.or_ntt_direct.argtypes = [u64p, u64p, ctypes.c_int, u64, u64]
        L.or_negacyclic_schoolbook.argtypes = [u64p, u64p, u64p, ctypes.c_int, u64]
        L.or_polymul.argtypes = [u64p, u64p, u64p, ctypes.c_int, u64, u64]
        L.or_automorphism.argtypes = [u64p, u64p, ctypes.c_int, u64, u64]
        L.or_bconv.argtypes = [u64p, u64p, ctypes.c_int, u64p, u64p, ctypes.c_int, ctypes.c_int]
        pp = ctypes.POINTER(_OrParams)
        L.or_keyswitch.argtypes = [pp, u64p, ctypes.c_int, u64p, u64p, u64p]
        L.or_modup.argtypes = [pp, u64p, ctypes.c_int, u64p]
        L.or_ks_ext.argtypes = [pp, u64p, ctypes.c_int, u64p, u64, u64p, u64p]
        L.or_rescale.argtypes = [pp, u64p, ctypes.c_int]
        ip = ctypes.POINTER(ctypes.c_int)
        L.or_rns_polymul.argtypes = [pp, u64p, u64p, u64p, ctypes.c_int, ip]
        L.or_rns_ntt_fwd.argtypes = [pp, u64p, ctypes.c_int, ip]
        L.or_rns_ntt_inv.argtypes = [pp, u64p, ctypes.c_int, ip]
        L.or_threads.argtypes = [ctypes.c_int]
        L.or_threads.restype = ctypes.c_int
        L.or_mulmod_vec.argtypes = [u64p, u64p, u64p, ctypes.c_size_t, u64]
        L.or_mulmod_scalar.argtypes = [u64p, u64, u64p, ctypes.c_size_t, u64]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"], (a.dtype, a.flags)
    return a.ctypes.data_as(u64p)


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# ---------------------------------------------------------------------------
# small wrappers over the C primitives
# ---------------------------------------------------------------------------
def threads(n: int = 0) -> int:
    """Set (n > 0) and return the number of OpenMP threads of the limb loops."""
    return int(lib().or_threads(n))


def is_prime(x: int) -> bool:
    return bool(lib().or_is_prime(x))


def gen_primes(log_n: int, bits: int, count: int, exclude=()) -> list[int]:
    ex = np.array(list(exclude) or [0], dtype=np.uint64)
    out = np.zeros(max(count, 1), dtype=np.uint64)
    got = lib().or_gen_primes(log_n, bits, count, _p(ex), len(exclude), _p(out))
    if got != count:
        raise ValueError("not enough %d-bit primes = 1 mod 2^%d" % (bits, log_n + 1))
    return [int(v) for v in out[:count]]


def find_psi(q: int, log_n: int) -> int:
    return int(lib().or_find_psi(q, log_n))


def ntt_fwd(a: np.ndarray, log_n: int, q: int, psi: int) -> np.ndarray:
    x = np.ascontiguousarray(a, dtype=np.uint64).copy()
    lib().or_ntt_fwd(_p(x), log_n, q, psi)
    return x


def ntt_inv(a: np.ndarray, log_n: int, q: int, psi: int) -> np.ndarray:
    x = np.ascontiguousarray(a, dtype=np.uint64).copy()
    lib().or_ntt_inv(_p(x), log_n, q, psi)
    return x


def ntt_direct(a: np.ndarray, log_n: int, q: int, psi: int) -> np.ndarray:
    x = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.zeros_like(x)
    lib().or_ntt_direct(_p(x), _p(out), log_n, q, psi)
    return out


def negacyclic_schoolbook(a, b, q: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    out = np.zeros_like(a)
    lib().or_negacyclic_schoolbook(_p(a), _p(b), _p(out), a.size, q)
    return out


def polymul(a, b, log_n: int, q: int, psi: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    out = np.zeros_like(a)
    lib().or_polymul(_p(a), _p(b), _p(out), log_n, q, psi)
    return out


def automorphism(a, g: int, q: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.zeros_like(a)
    lib().or_automorphism(_p(a), _p(out), a.size, g, q)
    return out


def bconv(x: np.ndarray, src: list[int], dst: list[int]) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.uint64)
    n = x.shape[-1]
    s = np.array(src, dtype=np.uint64)
    d = np.array(dst, dtype=np.uint64)
    out = np.zeros((len(dst), n), dtype=np.uint64)
    lib().or_bconv(_p(x), _p(s), len(src), _p(out), _p(d), len(dst), n)
    return out


def mulmod(a: np.ndarray, b, q: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.zeros_like(a)
    if np.isscalar(b) or isinstance(b, int):
        lib().or_mulmod_scalar(_p(a), int(b) % q, _p(out), a.size, q)
    else:
        b = np.ascontiguousarray(b, dtype=np.uint64)
        lib().or_mulmod_vec(_p(a), _p(b), _p(out), a.size, q)
    return out


def addmod(a, b, q: int) -> np.ndarray:
    # residues < 2^62, so the sum never wraps a uint64
    return (a + b) % np.uint64(q)


def submod(a, b, q: int) -> np.ndarray:
    return (a + (np.uint64(q) - b)) % np.uint64(q)


def negmod(a, q: int) -> np.ndarray:
    return (np.uint64(q) - a) % np.uint64(q)


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------
@dataclass
class Params:
    log_n: int
    q: list            # q_0 .. q_{L-1}
    p: list            # p_0 .. p_{K-1}
    dnum: int
    scale: float
    rot_base: int
    psis: list = field(default_factory=list)   # per modulus, q's then p's

    @property
    def n(self):
        return 1 << self.log_n

    @property
    def slots(self):
        return self.n // 2

    @property
    def L(self):
        return len(self.q)

    @property
    def K(self):
        return len(self.p)

    @property
    def alpha(self):
        return -(-self.L // self.dnum)

    @property
    def mods(self):
        return list(self.q) + list(self.p)

    def c_struct(self) -> _OrParams:
        s = _OrParams()
        s.log_n, s.L, s.K, s.dnum = self.log_n, self.L, self.K, self.dnum
        for i, m in enumerate(self.mods):
            s.mods[i] = m
            s.psis[i] = self.psis[i]
        return s


def special_prime_count(q_bits: list, dnum: int, p_bits: int = 60, k_stated: int = 0) -> int:
    """Reading R1: the smallest K with K*p_bits >= bits of the largest digit
    (digits = consecutive groups of ceil(L/dnum) limbs), never below the
    configured K."""
    L = len(q_bits)
    alpha = -(-L // dnum)
    widest = max(sum(q_bits[j:j + alpha]) for j in range(0, L, alpha))
    return max(k_stated, -(-widest // p_bits))


def make_params(log_n: int, q_bits: list, K: int, dnum: int, scale: float,
                rot_base: int = 2, p_bits: int = 60) -> Params:
    """Primes per reading R2: q_0 first, then the scaling primes (one
    downward search per distinct bit size, in order), then K special primes,
    all distinct."""
    chosen: list[int] = []
    q = []
    for b in q_bits:
        (v,) = gen_primes(log_n, b, 1, exclude=chosen)
        q.append(v)
        chosen.append(v)
    p = []
    for _ in range(K):
        (v,) = gen_primes(log_n, p_bits, 1, exclude=chosen)
        p.append(v)
        chosen.append(v)
    prm = Params(log_n=log_n, q=q, p=p, dnum=dnum, scale=float(scale), rot_base=rot_base)
    prm.psis = [find_psi(m, log_n) for m in prm.mods]
    return prm


# ---------------------------------------------------------------------------
# encoding (canonical embedding, slot i <-> zeta^(5^i), zeta = e^(i pi/n))
# ---------------------------------------------------------------------------
def _round_half_away(x: np.ndarray) -> np.ndarray:
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def slot_exponents(n: int) -> np.ndarray:
    """5^i mod 2n for i in [0, n/2)."""
    S = n // 2
    e = np.empty(S, dtype=np.int64)
    g = 1
    for i in range(S):
        e[i] = g
        g = (g * 5) % (2 * n)
    return e


def encode_coeffs(z, n: int, scale: float) -> np.ndarray:
    """Integer coefficients m_j = round_half_away((2 scale/n) Re sum_i z_i zeta^(-5^i j))
    of the encoding of the slot vector z (len <= n/2, zero padded), computed
    with one length-n FFT: sum over all odd exponents (2k+1) of v_k
    zeta^(-(2k+1) j) with v at 5^i equal to z_i and at -5^i equal to conj(z_i)."""
    S = n // 2
    zz = np.zeros(S, dtype=np.complex128)
    z = np.asarray(z, dtype=np.complex128)
    zz[: z.size] = z
    ex = slot_exponents(n)
    v = np.zeros(n, dtype=np.complex128)
    v[(ex - 1) // 2] = zz
    v[(2 * n - ex - 1) // 2] = np.conj(zz)
    j = np.arange(n)
    zeta_mj = np.exp(-1j * np.pi * j / n)
    m = (scale / n) * np.real(zeta_mj * np.fft.fft(v))
    return _round_half_away(m).astype(np.int64)


def encode_coeffs_direct(z, n: int, scale: float) -> np.ndarray:
    """O(n * S) evaluation of the same definition (pin for encode_coeffs)."""
    S = n // 2
    zz = np.zeros(S, dtype=np.complex128)
    z = np.asarray(z, dtype=np.complex128)
    zz[: z.size] = z
    ex = slot_exponents(n)
    j = np.arange(n)
    acc = np.zeros(n)
    for i in range(S):
        t = (ex[i] * j) % (2 * n)
        acc += np.real(zz[i] * np.exp(-1j * np.pi * t / n))
    return _round_half_away((2 * scale / n) * acc).astype(np.int64)


def onehot_coeffs(value: float, slot: int, n: int, scale: float) -> np.ndarray:
    """Encoding of value * e_slot (reading R8): closed form of encode_coeffs for
    a one-hot slot vector, angle reduced exactly in integers."""
    g = pow(5, slot, 2 * n)
    j = np.arange(n, dtype=np.int64)
    t = (g * j) % (2 * n)
    u = t % n
    sgn = np.where(t >= n, -1.0, 1.0)
    mag = _round_half_away(value * (2.0 * scale / n) * np.cos(np.pi * u / n))
    return (sgn * mag).astype(np.int64)


def to_rns(m: np.ndarray, mods: list) -> np.ndarray:
    """Signed integer coefficients -> residues, one limb per modulus."""
    m = np.asarray(m, dtype=np.int64)
    out = np.empty((len(mods), m.size), dtype=np.uint64)
    for i, q in enumerate(mods):
        out[i] = np.mod(m, np.int64(q)).astype(np.uint64)
    return out


def decode_coeffs(m0: np.ndarray, q0: int, scale: float, n_slots: int | None = None) -> np.ndarray:
    """Decode from limb q_0 (centred residues), reading G9 of the plan:
    z_i = m(zeta^(5^i)) / scale."""
    n = m0.size
    big = m0 > np.uint64(q0 // 2)
    # centred residue as a double (exact for |c| < 2^53)
    c = np.where(big, -((np.uint64(q0) - m0).astype(np.float64)), m0.astype(np.float64))
    j = np.arange(n)
    w = c * np.exp(1j * np.pi * j / n)
    V = n * np.fft.ifft(w)                     # V[k] = sum_j c_j zeta^((2k+1) j)
    ex = slot_exponents(n)
    z = V[(ex - 1) // 2] / scale
    if n_slots is not None:
        z = z[:n_slots]
    return z


# ---------------------------------------------------------------------------
# ciphertexts, keys
# ---------------------------------------------------------------------------
@dataclass
class Ct:
    c0: np.ndarray      # (ell, n) uint64, coefficient domain
    c1: np.ndarray
    scale: float

    @property
    def level(self):
        return self.c0.shape[0]

    def copy(self):
        return Ct(self.c0.copy(), self.c1.copy(), self.scale)


@dataclass
class Pt:
    m: np.ndarray       # (ell, n) uint64 residues, coefficient domain
    scale: float

    @property
    def level(self):
        return self.m.shape[0]


@dataclass
class Keys:
    s: np.ndarray                       # ternary secret, int64 (n,)
    relin: np.ndarray                   # [dnum][2][L+K][n] uint64
    rot: dict                           # amount -> [dnum][2][L+K][n]


class Oracle:
    """RNS-CKKS on the CPU, coefficient domain, over one parameter set."""

    def __init__(self, params: Params, nthreads: int | None = None):
        self.P = params
        self._cs = params.c_struct()
        self.n = params.n
        self.mods = params.mods
        if nthreads is not None:
            threads(nthreads)

    # -- helpers -----------------------------------------------------------
    def _mi(self, ell: int) -> np.ndarray:
        return np.arange(ell, dtype=np.int32)

    def rns_polymul(self, a: np.ndarray, b: np.ndarray, mod_idx) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        mi = np.ascontiguousarray(mod_idx, dtype=np.int32)
        out = np.zeros_like(a)
        lib().or_rns_polymul(ctypes.byref(self._cs), _p(a), _p(b), _p(out), len(mi), _ip(mi))
        return out

    def rns_ntt(self, a: np.ndarray, mod_idx=None) -> np.ndarray:
        """Coefficient -> evaluation representation (forward NTT per limb,
        bit-reversed order of evaluation points)."""
        x = np.ascontiguousarray(a, dtype=np.uint64).copy()
        mi = np.arange(x.shape[0], dtype=np.int32) if mod_idx is None else np.ascontiguousarray(mod_idx, dtype=np.int32)
        lib().or_rns_ntt_fwd(ctypes.byref(self._cs), _p(x), len(mi), _ip(mi))
        return x

    def rns_intt(self, a: np.ndarray, mod_idx=None) -> np.ndarray:
        x = np.ascontiguousarray(a, dtype=np.uint64).copy()
        mi = np.arange(x.shape[0], dtype=np.int32) if mod_idx is None else np.ascontiguousarray(mod_idx, dtype=np.int32)
        lib().or_rns_ntt_inv(ctypes.byref(self._cs), _p(x), len(mi), _ip(mi))
        return x

    def small_to_rns(self, v: np.ndarray, nmods: int | None = None, mod_idx=None) -> np.ndarray:
        mods = self.mods if mod_idx is None else [self.mods[i] for i in mod_idx]
        if nmods is not None:
            mods = mods[:nmods]
        return to_rns(v, mods)

    # -- encoding ----------------------------------------------------------
    def encode(self, z, level: int, scale: float) -> Pt:
        m = encode_coeffs(z, self.n, scale)
        return Pt(to_rns(m, self.mods[:level]), scale)

    def encode_onehot(self, value: float, slot: int, level: int, scale: float) -> Pt:
        m = onehot_coeffs(value, slot, self.n, scale)
        return Pt(to_rns(m, self.mods[:level]), scale)

    def decode(self, pt: Pt, n_slots: int | None = None) -> np.ndarray:
        return decode_coeffs(pt.m[0], self.mods[0], pt.scale, n_slots)

    # -- keys ----------------------------------------------------------------
    def sample_secret(self, rng: np.random.Generator) -> np.ndarray:
        return rng.integers(-1, 2, size=self.n).astype(np.int64)

    def sample_error(self, rng: np.random.Generator, sigma: float = 3.2) -> np.ndarray:
        e = _round_half_away(rng.normal(0.0, sigma, size=self.n))
        return np.clip(e, -6 * sigma, 6 * sigma).astype(np.int64)

    def sample_uniform(self, rng: np.random.Generator, mods: list) -> np.ndarray:
        return np.stack([rng.integers(0, m, size=self.n, dtype=np.uint64) for m in mods])

    def gen_switch_key(self, s: np.ndarray, s_new_rns: np.ndarray, rng) -> np.ndarray:
        """Key switching key from s_new to s (reading G12 of the plan):
        k_j = (-a_j s + e_j + g_j s_new, a_j) over q_0..q_{L-1}, p_0..p_{K-1},
        with g_j = P mod q_i for q_i in digit j and 0 on every other modulus."""
        P = self.P
        L, K, n = P.L, P.K, self.n
        nm = L + K
        alpha = P.alpha
        mods = self.mods
        s_rns = self.small_to_rns(s)
        Pprod = 1
        for pk in P.p:
            Pprod *= pk
        out = np.zeros((P.dnum, 2, nm, n), dtype=np.uint64)
        all_idx = np.arange(nm, dtype=np.int32)
        for j in range(P.dnum):
            a = self.sample_uniform(rng, mods)
            e = self.small_to_rns(self.sample_error(rng))
            as_ = self.rns_polymul(a, s_rns, all_idx)
            k0 = np.empty((nm, n), dtype=np.uint64)
            for i, m in enumerate(mods):
                v = submod(e[i], as_[i], m)
                if i < L and j * alpha <= i < min((j + 1) * alpha, L):
                    gi = Pprod % m
                    v = addmod(v, mulmod(s_new_rns[i], gi, m), m)
                k0[i] = v
            out[j, 0] = k0
            out[j, 1] = a
        return out

    def keygen(self, seed: int, rot_amounts=()) -> Keys:
        rng = np.random.default_rng(seed)
        s = self.sample_secret(rng)
        s_rns = self.small_to_rns(s)
        nm = self.P.L + self.P.K
        s2 = self.rns_polymul(s_rns, s_rns, np.arange(nm, dtype=np.int32))
        relin = self.gen_switch_key(s, s2, rng)
        rot = {}
        for r in sorted(set(int(x) % self.P.slots for x in rot_amounts)):
            if r == 0:
                continue
            g = pow(5, r, 2 * self.n)
            srot = np.stack([automorphism(s_rns[i], g, m) for i, m in enumerate(self.mods)])
            rot[r] = self.gen_switch_key(s, srot, rng)
        return Keys(s=s, relin=relin, rot=rot)

    # -- encryption ------------------------------------------------------------
    def encrypt(self, pt: Pt, keys: Keys, rng: np.random.Generator) -> Ct:
        """Secret-key encryption: (c0, c1) = (-a s + e + m, a)."""
        ell = pt.level
        mods = self.mods[:ell]
        a = self.sample_uniform(rng, mods)
        e = self.small_to_rns(self.sample_error(rng), ell)
        s_rns = self.small_to_rns(keys.s, ell)
        as_ = self.rns_polymul(a, s_rns, self._mi(ell))
        c0 = np.stack([addmod(submod(e[i], as_[i], q), pt.m[i], q) for i, q in enumerate(mods)])
        return Ct(c0, a, pt.scale)

    def decrypt(self, ct: Ct, keys: Keys) -> Pt:
        ell = ct.level
        s_rns = self.small_to_rns(keys.s, ell)
        c1s = self.rns_polymul(ct.c1, s_rns, self._mi(ell))
        m = np.stack([addmod(ct.c0[i], c1s[i], q) for i, q in enumerate(self.mods[:ell])])
        return Pt(m, ct.scale)

    # -- homomorphic operations ------------------------------------------------
    def add(self, x: Ct, y: Ct) -> Ct:
        assert x.level == y.level
        if abs(x.scale - y.scale) > 1e-9 * abs(x.scale):
            raise ValueError("scale mismatch")
        mods = self.mods[: x.level]
        c0 = np.stack([addmod(x.c0[i], y.c0[i], q) for i, q in enumerate(mods)])
        c1 = np.stack([addmod(x.c1[i], y.c1[i], q) for i, q in enumerate(mods)])
        return Ct(c0, c1, x.scale)

    def zero_ct(self, level: int, scale: float) -> Ct:
        z = np.zeros((level, self.n), dtype=np.uint64)
        return Ct(z, z.copy(), scale)

    def tensor(self, x: Ct, y: Ct):
        """EvalMult without relinearisation: (x0 y0, x0 y1 + x1 y0, x1 y1)."""
        assert x.level == y.level
        ell = x.level
        mi = self._mi(ell)
        mods = self.mods[:ell]
        d0 = self.rns_polymul(x.c0, y.c0, mi)
        d1a = self.rns_polymul(x.c0, y.c1, mi)
        d1b = self.rns_polymul(x.c1, y.c0, mi)
        d1 = np.stack([addmod(d1a[i], d1b[i], q) for i, q in enumerate(mods)])
        d2 = self.rns_polymul(x.c1, y.c1, mi)
        return d0, d1, d2, x.scale * y.scale

    def keyswitch(self, c: np.ndarray, ksk: np.ndarray):
        ell = c.shape[0]
        c = np.ascontiguousarray(c, dtype=np.uint64)
        ksk = np.ascontiguousarray(ksk, dtype=np.uint64)
        o0 = np.zeros_like(c)
        o1 = np.zeros_like(c)
        lib().or_keyswitch(ctypes.byref(self._cs), _p(c), ell, _p(ksk), _p(o0), _p(o1))
        return o0, o1

    def relinearize(self, d0, d1, d2, scale, keys: Keys) -> Ct:
        k0, k1 = self.keyswitch(d2, keys.relin)
        ell = d0.shape[0]
        mods = self.mods[:ell]
        c0 = np.stack([addmod(d0[i], k0[i], q) for i, q in enumerate(mods)])
        c1 = np.stack([addmod(d1[i], k1[i], q) for i, q in enumerate(mods)])
        return Ct(c0, c1, scale)

    def mult_relin(self, x: Ct, y: Ct, keys: Keys) -> Ct:
        d0, d1, d2, sc = self.tensor(x, y)
        return self.relinearize(d0, d1, d2, sc, keys)

    def rescale(self, ct: Ct) -> Ct:
        ell = ct.level
        qt = self.mods[ell - 1]
        c0 = np.ascontiguousarray(ct.c0.copy())
        c1 = np.ascontiguousarray(ct.c1.copy())
        lib().or_rescale(ctypes.byref(self._cs), _p(c0), ell)
        lib().or_rescale(ctypes.byref(self._cs), _p(c1), ell)
        return Ct(c0[: ell - 1].copy(), c1[: ell - 1].copy(), ct.scale / qt)

    def mul_plain(self, ct: Ct, pt: Pt) -> Ct:
        assert ct.level == pt.level
        mi = self._mi(ct.level)
        return Ct(self.rns_polymul(ct.c0, pt.m, mi), self.rns_polymul(ct.c1, pt.m, mi), ct.scale * pt.scale)

    def rotate_single(self, ct: Ct, r: int, keys: Keys) -> Ct:
        """One key switch: sigma_g on both components, g = 5^r mod 2n, then
        switch sigma_g(s) -> s."""
        r %= self.P.slots
        if r == 0:
            return ct.copy()
        if r not in keys.rot:
            raise KeyError("no rotation key for %d" % r)
        g = pow(5, r, 2 * self.n)
        mods = self.mods[: ct.level]
        a0 = np.stack([automorphism(ct.c0[i], g, q) for i, q in enumerate(mods)])
        a1 = np.stack([automorphism(ct.c1[i], g, q) for i, q in enumerate(mods)])
        k0, k1 = self.keyswitch(a1, keys.rot[r])
        c0 = np.stack([addmod(a0[i], k0[i], q) for i, q in enumerate(mods)])
        return Ct(c0, k1, ct.scale)

    def modup(self, c: np.ndarray) -> np.ndarray:
        """ModUp of every digit of c (coefficient domain): [beta][ell+K][n]."""
        c = np.ascontiguousarray(c, dtype=np.uint64)
        ell = c.shape[0]
        beta = -(-ell // self.P.alpha)
        ext = np.zeros((beta, ell + self.P.K, self.n), dtype=np.uint64)
        lib().or_modup(ctypes.byref(self._cs), _p(c), ell, _p(ext))
        return ext

    def rotate_hoisted(self, ct: Ct, amounts: list, keys: Keys) -> list:
        """Rotations of one ciphertext by several amounts (each with a key of
        its own) sharing one ModUp of c1: the automorphism is applied to the
        extended digits, then inner product and ModDown per amount."""
        ext = self.modup(ct.c1)
        ell = ct.level
        mods = self.mods[:ell]
        out = []
        for r in amounts:
            r %= self.P.slots
            if r == 0:
                out.append(ct.copy())
                continue
            if r not in keys.rot:
                raise KeyError("no rotation key for %d" % r)
            g = pow(5, r, 2 * self.n)
            k0 = np.zeros((ell, self.n), dtype=np.uint64)
            k1 = np.zeros((ell, self.n), dtype=np.uint64)
            ksk = np.ascontiguousarray(keys.rot[r], dtype=np.uint64)
            lib().or_ks_ext(ctypes.byref(self._cs), _p(ext), ell, _p(ksk), g, _p(k0), _p(k1))
            a0 = np.stack([automorphism(ct.c0[i], g, q) for i, q in enumerate(mods)])
            c0 = np.stack([addmod(a0[i], k0[i], q) for i, q in enumerate(mods)])
            out.append(Ct(c0, k1, ct.scale))
        return out

    def rotation_plan(self, r: int) -> list:
        return rotation_plan(r, self.P.slots, self.P.rot_base)

    def rotate(self, ct: Ct, r: int, keys: Keys) -> Ct:
        """EvalRotate (reading R4/R5): left rotation by r through the plan."""
        out = ct
        for amt in self.rotation_plan(r):
            out = self.rotate_single(out, amt, keys)
        return out if out is not ct else ct.copy()


def rotation_plan(r: int, slots: int, base: int) -> list:
    """Reading R5: r mod S in base `base`, one step d*base^t per nonzero digit,
    ascending t."""
    r %= slots
    steps = []
    w = 1
    while r:
        d = r % base
        if d:
            steps.append(d * w)
        r //= base
        w *= base
    return steps


def rotation_key_amounts(slots: int, base: int) -> list:
    """Every amount d*base^t (< slots) a plan can ask for."""
    out = []
    w = 1
    while w < slots:
        for d in range(1, base):
            if d * w < slots:
                out.append(d * w)
        w *= base
    return out
