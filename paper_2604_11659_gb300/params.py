"""Library-side parameter construction from a workload recipe (no arithmetic
beyond choosing how many special primes hybrid key switching needs)."""
from __future__ import annotations

from . import spfhe


def special_primes(q_bits, dnum: int, p_bits: int = 60, k_stated: int = 0) -> int:
    """Smallest K with K * p_bits at least the bit size of the widest key
    switching digit (consecutive groups of ceil(L/dnum) primes), so that the
    special modulus P covers every digit modulus; never below the stated K."""
    L = len(q_bits)
    alpha = -(-L // dnum)
    widest = max(sum(q_bits[j:j + alpha]) for j in range(0, L, alpha))
    return max(k_stated, -(-widest // p_bits))


def ctx_params(recipe, rot_base: int | None = None) -> "spfhe.Params":
    K = special_primes(recipe.q_bits, recipe.dnum, recipe.p_bits, recipe.k_stated)
    return spfhe.make_params(recipe.log_n, recipe.q_bits, K, recipe.dnum, recipe.scale,
                             rot_base or recipe.rot_base, recipe.p_bits)
