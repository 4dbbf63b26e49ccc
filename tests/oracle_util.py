"""Test helpers: build oracle parameters from a workload recipe."""
from oracle import ckks


def oracle_params(recipe, rot_base=None):
    K = ckks.special_prime_count(recipe.q_bits, recipe.dnum, recipe.p_bits, recipe.k_stated)
    return ckks.make_params(recipe.log_n, recipe.q_bits, K, recipe.dnum, recipe.scale,
                            rot_base=rot_base or recipe.rot_base, p_bits=recipe.p_bits)
