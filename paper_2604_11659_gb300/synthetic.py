"""Seeded synthetic workloads (matrices and parameter recipes).

This module holds no CKKS arithmetic: it only draws the plaintext matrices
that both the CUDA path and the CPU oracle consume, and names the parameter
recipes (ring degree, prime sizes, dnum, scale) of each workload.  The paper
evaluates on random matrices of sizes 8 and 16 with sparsity 0-100 % (Sec. 4);
the larger workloads below follow the same recipe at the sizes the GPU path is
measured on.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class RingRecipe:
    log_n: int
    q_bits: list          # q_0 .. q_{L-1}
    dnum: int
    scale_bits: int
    k_stated: int = 0     # special primes named by the workload (0 = unstated)
    p_bits: int = 60
    rot_base: int = 2

    @property
    def L(self):
        return len(self.q_bits)

    @property
    def scale(self) -> float:
        return float(2 ** self.scale_bits)



# Workload recipes -----------------------------------------------------------
def ring_small_16x16() -> RingRecipe:
    """N=2^12, q_0 60-bit + 3 x 40-bit scaling primes, dnum=1, scale 2^40."""
    return RingRecipe(log_n=12, q_bits=[60, 40, 40, 40], dnum=1, scale_bits=40, k_stated=1, rot_base=16)


def ring_128x128() -> RingRecipe:
    """N=2^16, L=24 (q_0 60-bit + 23 x 45-bit), dnum=3, scale 2^45."""
    return RingRecipe(log_n=16, q_bits=[60] + [45] * 23, dnum=3, scale_bits=45, k_stated=3, rot_base=256)


def ring_batch64() -> RingRecipe:
    """N=2^16, L=20, dnum=4 (scaling primes 45-bit, scale 2^45)."""
    return RingRecipe(log_n=16, q_bits=[60] + [45] * 19, dnum=4, scale_bits=45, k_stated=0, rot_base=256)


def ring_dense_layer() -> RingRecipe:
    """N=2^17, L=35 (q_0 60-bit + 34 x 50-bit), dnum=5, scale 2^50."""
    return RingRecipe(log_n=17, q_bits=[60] + [50] * 34, dnum=5, scale_bits=50, k_stated=4, rot_base=256)


def ring_tiny(log_n: int = 6, L: int = 4, dnum: int = 1, rot_base: int = 2) -> RingRecipe:
    """Small rings for fast tests (same prime sizes as the 16x16 workload)."""
    return RingRecipe(log_n=log_n, q_bits=[60] + [40] * (L - 1), dnum=dnum, scale_bits=40, rot_base=rot_base)


# Matrices -----------------------------------------------------------------
def bernoulli_sparse(rng: np.random.Generator, rows: int, cols: int, sparsity: float,
                     lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Entries uniform in [lo, hi], each zeroed i.i.d. with prob. `sparsity`."""
    M = rng.uniform(lo, hi, size=(rows, cols))
    keep = rng.random((rows, cols)) >= sparsity
    return np.where(keep, M, 0.0)


def structured_2_4(rng: np.random.Generator, rows: int, cols: int, sparsity: float) -> np.ndarray:
    """At most 2 nonzeros in every group of 4 consecutive row entries: pick 2
    positions per group, keep each with probability 2(1 - sparsity)
    (density 1 - sparsity for sparsity >= 0.5)."""
    assert cols % 4 == 0
    M = np.zeros((rows, cols))
    p_keep = min(1.0, 2.0 * (1.0 - sparsity))
    for i in range(rows):
        for g in range(0, cols, 4):
            pos = rng.choice(4, size=2, replace=False)
            for p in pos:
                if rng.random() < p_keep:
                    M[i, g + p] = rng.uniform(-1.0, 1.0)
    return M


def rescale_rows_to_unit_output(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Divide row i of A by max_j |(A B)_ij| when that exceeds 1, so every
    |output| <= 1."""
    C = A @ B
    A = A.copy()
    for i in range(A.shape[0]):
        m = np.max(np.abs(C[i])) if C.shape[1] else 0.0
        if m > 1.0:
            A[i] /= m
    return A


def relu_activations(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """50 % exact zeros, the rest uniform in [0, 1]."""
    M = rng.uniform(0.0, 1.0, size=(rows, cols))
    return np.where(rng.random((rows, cols)) < 0.5, 0.0, M)


def pruned_weights(rng: np.random.Generator, rows: int, cols: int, sigma: float = 0.05,
                   sparsity: float = 0.9) -> np.ndarray:
    """N(0, sigma^2) weights magnitude-pruned to `sparsity` (keep the largest)."""
    W = rng.normal(0.0, sigma, size=(rows, cols))
    k = int(round((1.0 - sparsity) * W.size))
    if k <= 0:
        return np.zeros_like(W)
    thr = np.sort(np.abs(W).ravel())[::-1][k - 1]
    return np.where(np.abs(W) >= thr, W, 0.0)


@dataclass
class MatmulCase:
    name: str
    A: np.ndarray
    B: np.ndarray
    ring: RingRecipe
    B_plain: bool = False     # True: B stays a plaintext operand (ct x pt)
    meta: dict = field(default_factory=dict)


def case_16x16(seed: int = 0, sparsity: float = 0.75) -> MatmulCase:
    """16x16 operands uniform in [-1, 1], `sparsity` zeroed i.i.d., rows of A
    rescaled so every |output| <= 1."""
    rng = np.random.default_rng(seed)
    A = bernoulli_sparse(rng, 16, 16, sparsity)
    B = bernoulli_sparse(rng, 16, 16, sparsity)
    A = rescale_rows_to_unit_output(A, B)
    return MatmulCase("16x16_s%d" % round(100 * sparsity), A, B, ring_small_16x16())


def case_128x128(seed: int = 1, sparsity: float = 0.9) -> MatmulCase:
    """128x128 operands uniform in [-1, 1], 90 % i.i.d. sparsity each."""
    rng = np.random.default_rng(seed)
    A = bernoulli_sparse(rng, 128, 128, sparsity)
    B = bernoulli_sparse(rng, 128, 128, sparsity)
    return MatmulCase("128x128_s%d" % round(100 * sparsity), A, B, ring_128x128())


def case_dense_layer(seed: int = 3, plain_weights: bool = False) -> MatmulCase:
    """64x784 ReLU-like activations times 784x128 pruned N(0, 0.05^2) weights."""
    rng = np.random.default_rng(seed)
    A = relu_activations(rng, 64, 784)
    W = pruned_weights(rng, 784, 128)
    return MatmulCase("dense_layer_64x784x128", A, W, ring_dense_layer(), B_plain=plain_weights)


def ring_serving() -> RingRecipe:
    """N=2^16, L=31 (q_0 60-bit + 30 x 45-bit), dnum=4, scale 2^45."""
    return RingRecipe(log_n=16, q_bits=[60] + [45] * 30, dnum=4, scale_bits=45, k_stated=0, rot_base=16)


def batch64_cases(seed: int = 2, count: int = 64, dims=(32, 64, 128, 256), sparsity=(0.70, 0.95)) -> list:
    """`count` independent square products: d drawn from `dims` (the batch
    workload uses {32, 64, 128, 256}), sparsity uniform in `sparsity` (the
    batch workload: [0.70, 0.95]), half i.i.d. Bernoulli, half 2:4
    structured."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        d = int(rng.choice(list(dims)))
        s = float(rng.uniform(sparsity[0], sparsity[1]))
        if b % 2 == 0:
            A = bernoulli_sparse(rng, d, d, s)
            B = bernoulli_sparse(rng, d, d, s)
        else:
            A = structured_2_4(rng, d, d, s)
            B = structured_2_4(rng, d, d, s)
        out.append(MatmulCase("batch%d_d%d" % (b, d), A, B, ring_batch64(), meta={"d": d, "sparsity": s}))
    return out


def tiny_case(seed: int, d: int, sparsity: float, log_n: int = 6, L: int = 4, dnum: int = 1,
              rot_base: int = 2, rows: int | None = None, inner: int | None = None,
              cols: int | None = None) -> MatmulCase:
    """Small rectangular product for fast tests."""
    rng = np.random.default_rng(seed)
    rows = rows or d
    inner = inner or d
    cols = cols or d
    A = bernoulli_sparse(rng, rows, inner, sparsity)
    B = bernoulli_sparse(rng, inner, cols, sparsity)
    A = rescale_rows_to_unit_output(A, B)
    return MatmulCase("tiny_%dx%dx%d" % (rows, inner, cols), A, B,
                      ring_tiny(log_n, L, dnum, rot_base))


def edge_cases(seed: int = 40, log_n: int = 6, rot_base: int = 4) -> dict:
    """Degenerate and boundary shapes on a tiny ring (S = 2^(log_n-1) slots):
    a 1x1x1 product, a dot product (1 x 9 x 1), an outer product (inner
    dimension 1), a result of exactly S slots, one of S + 1 (a one-slot
    second chunk), an all-zero row of A with an all-zero column of B, a single
    match far from slot 0, and an operand of S + 1 nonzeros (a one-slot
    second operand chunk)."""
    rng = np.random.default_rng(seed)
    ring = ring_tiny(log_n, 4, 1, rot_base)
    S = 1 << (log_n - 1)
    out = {}

    def add(name, A, B):
        out[name] = MatmulCase(name, rescale_rows_to_unit_output(A, B), B, ring)

    add("scalar_1x1x1", np.array([[0.7]]), np.array([[-0.9]]))
    add("dot_1x9x1", rng.uniform(-1, 1, (1, 9)), rng.uniform(-1, 1, (9, 1)))
    add("outer_6x1x5", rng.uniform(-1, 1, (6, 1)), rng.uniform(-1, 1, (1, 5)))
    add("result_S", bernoulli_sparse(rng, 4, 3, 0.3), bernoulli_sparse(rng, 3, S // 4, 0.3))
    add("result_S_plus_1", bernoulli_sparse(rng, 3, 4, 0.3), bernoulli_sparse(rng, 4, (S + 3) // 3, 0.3))
    A = bernoulli_sparse(rng, 5, 5, 0.3)
    B = bernoulli_sparse(rng, 5, 5, 0.3)
    A[2] = 0.0
    B[:, 3] = 0.0
    add("zero_row_and_col_5x5", A, B)
    A = np.zeros((8, 8))
    B = np.zeros((8, 8))
    A[7, 5] = 0.8
    B[5, 6] = -0.6
    add("single_match_8x8", A, B)
    d = 6
    A = rng.uniform(-1, 1, (d, d))
    A.flat[rng.choice(d * d, d * d - (S + 1), replace=False)] = 0.0
    add("operand_S_plus_1_nnz", A, bernoulli_sparse(rng, d, d, 0.5))
    return out


@dataclass
class ServeRequest:
    case: MatmulCase
    level: int          # operand level (limbs) of the request's ciphertexts
    key_set: int
    arrival_s: float


def serving_stream(seed: int = 4, count: int = 2000, dims=(64, 128, 256, 512), rate_per_s: float = 1.0,
                   key_sets: int = 4, levels=(10, 30)) -> list:
    """Poisson arrivals (exponential gaps, `rate_per_s`) of square products:
    d from `dims`, sparsity uniform in [0.50, 0.95] (i.i.d.), remaining levels
    uniform in `levels` (operand level = remaining + 1 limbs), key set uniform
    over `key_sets`."""
    rng = np.random.default_rng(seed)
    ring = ring_serving()
    t = 0.0
    out = []
    for r in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        d = int(rng.choice(list(dims)))
        s = float(rng.uniform(0.50, 0.95))
        A = bernoulli_sparse(rng, d, d, s)
        B = bernoulli_sparse(rng, d, d, s)
        A = rescale_rows_to_unit_output(A, B)
        lvl = int(rng.integers(levels[0], levels[1] + 1)) + 1
        out.append(ServeRequest(MatmulCase("req%d_d%d" % (r, d), A, B, ring, meta={"d": d, "sparsity": s}),
                                lvl, int(rng.integers(0, key_sets)), t))
    return out
