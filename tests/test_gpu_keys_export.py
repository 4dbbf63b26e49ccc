"""Key checkpoint (spfhe_keys_export) on the GPU: exporting a key set gives
back exactly what spfhe_keys_import was given, and a key set made by the
library's own keygen, exported and imported into a second context with the
same parameters, encrypts, decrypts, relinearises and rotates bit-identically
to the original."""
import ctypes

import numpy as np
import pytest

from oracle import ckks
from paper_2604_11659_gb300 import params as gparams
from paper_2604_11659_gb300 import synthetic
from tests.gpu_util import Pair, need_gpu
from tests.oracle_util import oracle_params

pytestmark = pytest.mark.gpu

RECIPES = {
    "tiny_dnum1": synthetic.ring_tiny(log_n=6, L=4, dnum=1, rot_base=2),
    "tiny_dnum3": synthetic.ring_tiny(log_n=7, L=6, dnum=3, rot_base=4),
}


def _key_shape(P):
    return (P.dnum, 2, P.L + P.K, P.n)


@pytest.mark.parametrize("name", list(RECIPES))
def test_export_returns_what_was_imported(name):
    p = Pair(RECIPES[name])
    try:
        o, P, sp = p.o, p.P, p.spfhe
        keys = o.keygen(21, rot_amounts=ckks.rotation_key_amounts(P.slots, P.rot_base))
        gk = p.import_keys(keys)
        secret, relin, rot = sp.spfhe_keys_export(p.ctx, gk, P.n, _key_shape(P))
        assert np.array_equal(secret, np.asarray(keys.s, dtype=np.int64))
        mi = np.arange(p.M, dtype=np.int32)

        def ntt_key(k):
            return np.stack([np.stack([o.rns_ntt(k[j, b], mi) for b in range(2)]) for j in range(k.shape[0])])

        assert np.array_equal(relin, ntt_key(keys.relin))
        assert sorted(rot) == sorted(keys.rot)
        for a, k in keys.rot.items():
            assert np.array_equal(rot[a], ntt_key(k)), a
    finally:
        p.close()


def test_library_keys_survive_export_and_import():
    sp = need_gpu()
    recipe = RECIPES["tiny_dnum3"]
    ctx1 = sp.spfhe_ctx_create(gparams.ctx_params(recipe))
    ctx2 = sp.spfhe_ctx_create(gparams.ctx_params(recipe))
    n, L = 1 << recipe.log_n, recipe.L
    handles = []
    try:
        k1 = sp.spfhe_keygen(ctx1, 99)
        handles.append((sp.spfhe_keys_free, k1))
        shape = _key_shape(oracle_params(recipe))
        secret, relin, rot = sp.spfhe_keys_export(ctx1, k1, n, shape)
        assert set(np.unique(secret)) <= {-1, 0, 1} and np.count_nonzero(secret) > n // 4
        assert rot and all(0 < a < n // 2 for a in rot)
        k2 = sp.spfhe_keys_import(ctx2, secret, relin, rot)
        handles.append((sp.spfhe_keys_free, k2))
        # the round trip is exact
        s2, r2, rot2 = sp.spfhe_keys_export(ctx2, k2, n, shape)
        assert np.array_equal(s2, secret) and np.array_equal(r2, relin)
        assert sorted(rot2) == sorted(rot) and all(np.array_equal(rot2[a], rot[a]) for a in rot)

        rng = np.random.default_rng(5)
        z = rng.uniform(-1, 1, n // 2)
        outs = []
        for ctx, keys in ((ctx1, k1), (ctx2, k2)):
            pt = sp.spfhe_encode(ctx, z, L, recipe.scale)
            ct = sp.spfhe_encrypt(ctx, keys, pt, 7)
            sq = sp.spfhe_mult_relin(ctx, keys, ct, ct)
            rt = sp.spfhe_rotate(ctx, keys, ct, 3)
            dec = sp.spfhe_decrypt(ctx, keys, ct)
            handles += [(sp.spfhe_pt_free, pt), (sp.spfhe_ct_free, ct), (sp.spfhe_ct_free, sq),
                        (sp.spfhe_ct_free, rt), (sp.spfhe_pt_free, dec)]
            outs.append((sp.spfhe_ct_export(ctx, ct, n), sp.spfhe_ct_export(ctx, sq, n),
                         sp.spfhe_ct_export(ctx, rt, n), sp.spfhe_pt_export(ctx, dec, n)))
            vals = sp.spfhe_decode(ctx, dec, n // 2).real
            assert np.max(np.abs(vals - z)) < 1e-6
        for a, b in zip(*outs):
            assert np.array_equal(a, b)
    finally:
        for free, h in reversed(handles):
            free(h)
        sp.spfhe_ctx_destroy(ctx2)
        sp.spfhe_ctx_destroy(ctx1)


def test_export_errors():
    p = Pair(RECIPES["tiny_dnum1"])
    other = None
    try:
        sp = p.spfhe
        keys = p.o.keygen(3, rot_amounts=[1, 2])
        gk = p.import_keys(keys)
        lib = sp.lib()
        count = ctypes.c_size_t(0)
        assert lib.spfhe_keys_export(p.ctx, gk, None, None, ctypes.byref(count), None, None) == 0
        assert count.value == 2
        # room for one rotation key, the set holds two
        small = ctypes.c_size_t(1)
        amts = np.zeros(1, dtype=np.int32)
        st = lib.spfhe_keys_export(p.ctx, gk, None, None, ctypes.byref(small), sp._i32(amts), None)
        assert st == -1
        # keys of another context
        other = sp.spfhe_ctx_create(gparams.ctx_params(RECIPES["tiny_dnum1"]))
        st = lib.spfhe_keys_export(other, gk, None, None, ctypes.byref(count), None, None)
        assert st == -1
        # amounts only (no key limbs)
        amts = np.zeros(2, dtype=np.int32)
        count = ctypes.c_size_t(2)
        assert lib.spfhe_keys_export(p.ctx, gk, None, None, ctypes.byref(count), sp._i32(amts), None) == 0
        assert sorted(amts.tolist()) == [1, 2] and amts.tolist() == sorted(amts.tolist())
    finally:
        if other is not None:
            sp.spfhe_ctx_destroy(other)
        p.close()
