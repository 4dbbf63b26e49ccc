"""Helpers shared by the GPU parity tests: build matching oracle / library
contexts from one workload recipe and move oracle-made keys, ciphertexts and
plaintexts into the library (evaluation representation) and back."""
import numpy as np
import pytest

from oracle import ckks
from paper_2604_11659_gb300 import params as gparams
from tests.oracle_util import oracle_params


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_11659_gb300 import spfhe
    return spfhe


class Pair:
    """An oracle and a library context over the same recipe."""

    def __init__(self, recipe, rot_base=None):
        self.spfhe = need_gpu()
        self.recipe = recipe
        self.P = oracle_params(recipe, rot_base=rot_base)
        self.o = ckks.Oracle(self.P)
        self.gp = gparams.ctx_params(recipe, rot_base=rot_base)
        self.ctx = self.spfhe.spfhe_ctx_create(self.gp)
        self.n = self.P.n
        self.M = self.P.L + self.P.K
        self._handles = []

    def close(self):
        sp = self.spfhe
        for kind, h in reversed(self._handles):
            {"ct": sp.spfhe_ct_free, "pt": sp.spfhe_pt_free, "keys": sp.spfhe_keys_free}[kind](h)
        self._handles = []
        sp.spfhe_ctx_destroy(self.ctx)

    def track(self, kind, h):
        self._handles.append((kind, h))
        return h

    # -- oracle -> library ------------------------------------------------------
    def ntt_rows(self, rows: np.ndarray, mod_idx=None) -> np.ndarray:
        return self.o.rns_ntt(rows, mod_idx)

    def import_keys(self, keys: ckks.Keys):
        def ntt_key(k):
            out = np.empty_like(k)
            mi = np.arange(self.M, dtype=np.int32)
            for j in range(k.shape[0]):
                for b in range(2):
                    out[j, b] = self.o.rns_ntt(k[j, b], mi)
            return out
        relin = ntt_key(keys.relin)
        rot = {a: ntt_key(k) for a, k in keys.rot.items()}
        return self.track("keys", self.spfhe.spfhe_keys_import(self.ctx, keys.s, relin, rot))

    def ct_limbs(self, ct: ckks.Ct) -> np.ndarray:
        return np.stack([self.o.rns_ntt(ct.c0), self.o.rns_ntt(ct.c1)])

    def import_ct(self, ct: ckks.Ct):
        return self.track("ct", self.spfhe.spfhe_ct_import(self.ctx, self.ct_limbs(ct), ct.level, ct.scale))

    def import_pt(self, pt: ckks.Pt):
        return self.track("pt", self.spfhe.spfhe_pt_import(self.ctx, self.o.rns_ntt(pt.m), pt.scale, False))

    # -- library -> numpy -------------------------------------------------------
    def export_ct(self, h) -> np.ndarray:
        return self.spfhe.spfhe_ct_export(self.ctx, h, self.n)

    def assert_ct_equal(self, h, ct: ckks.Ct):
        got = self.export_ct(h)
        want = self.ct_limbs(ct)
        assert got.shape == want.shape, (got.shape, want.shape)
        bad = np.argwhere(got != want)
        assert bad.size == 0, "first mismatches at %s" % bad[:5].tolist()
        lv, sc = self.spfhe.spfhe_ct_info(h)
        assert lv == ct.level and abs(sc - ct.scale) <= 1e-9 * abs(ct.scale)
