"""ctypes binding of libspfhe (include/spfhe.h).

Each `spfhe_*` function here has the name and arguments of the C entry point
and only marshals arguments (numpy arrays, ints) and turns a non-zero status
into SpfheError.  All ring arithmetic runs in the library's sm_103a kernels;
there is no Python or CPU fallback: loading fails loudly if libspfhe.so was
not built (run paper_2604_11659_gb300.build.build()).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspfhe.so")

c_u64p = ctypes.POINTER(ctypes.c_uint64)
c_i64p = ctypes.POINTER(ctypes.c_int64)
c_i32p = ctypes.POINTER(ctypes.c_int32)
c_dblp = ctypes.POINTER(ctypes.c_double)
handle = ctypes.c_void_p

STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ELEVEL", -4: "EKEY", -5: "ESCALE", -6: "ECUDA",
          -7: "ETIMEOUT", -8: "EPARAM"}


class SpfheError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (%d): %s" % (STATUS.get(status, "?"), status, msg))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_uint32), ("L", ctypes.c_uint32), ("q_bits", ctypes.POINTER(ctypes.c_uint32)),
                ("K", ctypes.c_uint32), ("p_bits", ctypes.c_uint32), ("dnum", ctypes.c_uint32),
                ("scale", ctypes.c_double), ("rot_base", ctypes.c_uint32)]


class SparseMeta(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32), ("nnz", ctypes.c_int32),
                ("indptr", c_i32p), ("indices", c_i32p)]


class Stats(ctypes.Structure):
    _fields_ = [("matches", ctypes.c_uint64), ("ks_relin", ctypes.c_uint64), ("ks_align", ctypes.c_uint64),
                ("ks_final", ctypes.c_uint64), ("rescales", ctypes.c_uint64), ("launches", ctypes.c_uint64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lib = None

# (name, restype, argtypes) of every exported entry point
_SIGS = [
    ("spfhe_last_error", ctypes.c_char_p, []),
    ("spfhe_ctx_create", ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_void_p, ctypes.POINTER(handle)]),
    ("spfhe_ctx_destroy", ctypes.c_int, [handle]),
    ("spfhe_ctx_moduli", ctypes.c_int, [handle, c_u64p, c_u64p]),
    ("spfhe_sync", ctypes.c_int, [handle]),
    ("spfhe_launch_count", ctypes.c_uint64, [handle]),
    ("spfhe_ctx_set_match_batch", ctypes.c_int, [handle, ctypes.c_uint32]),
    ("spfhe_ctx_set_ntt_chunk", ctypes.c_int, [handle, ctypes.c_uint32]),
    ("spfhe_ctx_set_ntt_split", ctypes.c_int, [handle, ctypes.c_uint32]),
    ("spfhe_ctx_set_align_budget", ctypes.c_int, [handle, ctypes.c_uint64]),
    ("spfhe_ctx_set_ntt_variant", ctypes.c_int, [handle, ctypes.c_uint32]),
    ("spfhe_ctx_set_fusion", ctypes.c_int, [handle, ctypes.c_int]),
    ("spfhe_tune_ntt_chunk", ctypes.c_int, [handle, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32,
                                            ctypes.POINTER(ctypes.c_uint32), c_dblp]),
    ("spfhe_prof_enable", ctypes.c_int, [handle, ctypes.c_int]),
    ("spfhe_prof_read", ctypes.c_int, [handle, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), c_dblp, c_dblp, c_dblp]),
    ("spfhe_prof_classes", ctypes.c_int, []),
    ("spfhe_prof_keyswitch", ctypes.c_int, [handle, ctypes.POINTER(ctypes.c_uint64), c_dblp]),
    ("spfhe_prof_transform_limbs", ctypes.c_int, [handle, ctypes.c_int, c_dblp, c_dblp, c_dblp]),
    ("spfhe_prof_alu_rates", ctypes.c_int, [handle, c_dblp, ctypes.c_size_t]),
    ("spfhe_prof_class_name", ctypes.c_char_p, [ctypes.c_int]),
    ("spfhe_prof_alu_peak", ctypes.c_int, [handle, c_dblp, c_dblp, c_dblp, c_dblp]),
    ("spfhe_keygen", ctypes.c_int, [handle, ctypes.c_uint64, ctypes.POINTER(handle)]),
    ("spfhe_keys_import", ctypes.c_int, [handle, c_i64p, c_u64p, ctypes.c_size_t, c_i32p,
                                         ctypes.POINTER(c_u64p), ctypes.POINTER(handle)]),
    ("spfhe_keys_export", ctypes.c_int, [handle, handle, c_i64p, c_u64p, ctypes.POINTER(ctypes.c_size_t), c_i32p,
                                         ctypes.POINTER(c_u64p)]),
    ("spfhe_keys_free", None, [handle]),
    ("spfhe_encode", ctypes.c_int, [handle, c_dblp, c_dblp, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_double,
                                    ctypes.POINTER(handle)]),
    ("spfhe_pt_import", ctypes.c_int, [handle, c_u64p, ctypes.c_uint32, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(handle)]),
    ("spfhe_pt_export", ctypes.c_int, [handle, handle, c_u64p]),
    ("spfhe_pt_info", ctypes.c_int, [handle, ctypes.POINTER(ctypes.c_uint32), c_dblp]),
    ("spfhe_pt_free", None, [handle]),
    ("spfhe_decode", ctypes.c_int, [handle, handle, c_dblp, c_dblp, ctypes.c_size_t]),
    ("spfhe_encrypt", ctypes.c_int, [handle, handle, handle, ctypes.c_uint64, ctypes.POINTER(handle)]),
    ("spfhe_decrypt", ctypes.c_int, [handle, handle, handle, ctypes.POINTER(handle)]),
    ("spfhe_ct_import", ctypes.c_int, [handle, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_double,
                                       ctypes.POINTER(handle)]),
    ("spfhe_ct_export", ctypes.c_int, [handle, handle, ctypes.c_void_p]),
    ("spfhe_ct_info", ctypes.c_int, [handle, ctypes.POINTER(ctypes.c_uint32), c_dblp]),
    ("spfhe_ct_free", None, [handle]),
    ("spfhe_mult_relin", ctypes.c_int, [handle, handle, handle, handle, ctypes.POINTER(handle)]),
    ("spfhe_rescale", ctypes.c_int, [handle, handle]),
    ("spfhe_rotate", ctypes.c_int, [handle, handle, handle, ctypes.c_int32, ctypes.POINTER(handle)]),
    ("spfhe_mul_plain", ctypes.c_int, [handle, handle, handle, ctypes.POINTER(handle)]),
    ("spfhe_add", ctypes.c_int, [handle, handle, handle, ctypes.POINTER(handle)]),
    ("spfhe_ntt", ctypes.c_int, [handle, ctypes.c_void_p, ctypes.c_uint32, c_i32p, ctypes.c_int]),
    ("spfhe_rescale_noalloc", ctypes.c_int, [handle, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]),
    ("spfhe_plan_matches", ctypes.c_int, [ctypes.POINTER(SparseMeta), ctypes.POINTER(SparseMeta), c_i32p,
                                          ctypes.POINTER(ctypes.c_uint64)]),
    ("spfhe_sparse_matmul_ct_ct", ctypes.c_int, [handle, handle, ctypes.POINTER(SparseMeta), ctypes.POINTER(handle),
                                                 ctypes.c_size_t, ctypes.POINTER(SparseMeta),
                                                 ctypes.POINTER(handle), ctypes.c_size_t, handle,
                                                 ctypes.POINTER(handle), ctypes.c_size_t, ctypes.POINTER(Stats)]),
    ("spfhe_sparse_matmul_ct_pt", ctypes.c_int, [handle, handle, ctypes.POINTER(SparseMeta), ctypes.POINTER(handle),
                                                 ctypes.c_size_t, ctypes.POINTER(SparseMeta), c_dblp,
                                                 ctypes.POINTER(handle), ctypes.POINTER(handle), ctypes.c_size_t,
                                                 ctypes.POINTER(Stats)]),
    ("spfhe_matmul_graph_launch", ctypes.c_int, [handle]),
    ("spfhe_ct_overwrite", ctypes.c_int, [handle, handle, ctypes.c_void_p]),
    ("spfhe_matmul_graph_free", None, [handle]),
    ("spfhe_sparse_matmul_ct_pt_grouped", ctypes.c_int,
     [handle, handle, ctypes.POINTER(SparseMeta), ctypes.POINTER(handle), ctypes.c_size_t, ctypes.POINTER(SparseMeta),
      c_dblp, ctypes.POINTER(handle), ctypes.c_int, ctypes.POINTER(handle), ctypes.c_size_t, ctypes.POINTER(Stats)]),
    ("spfhe_naive_matmul_ct_ct", ctypes.c_int,
     [handle, handle, ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
      ctypes.POINTER(handle), ctypes.c_size_t, ctypes.POINTER(handle), ctypes.c_size_t, handle,
      ctypes.POINTER(handle), ctypes.c_size_t, ctypes.POINTER(Stats)]),
    ("spfhe_sparse_matmul_ct_ct_grouped", ctypes.c_int,
     [handle, handle, ctypes.POINTER(SparseMeta), ctypes.POINTER(handle), ctypes.c_size_t, ctypes.POINTER(SparseMeta),
      ctypes.POINTER(handle), ctypes.c_size_t, handle, ctypes.c_int, ctypes.POINTER(handle), ctypes.c_size_t,
      ctypes.POINTER(Stats)]),
]

class MatmulReq(ctypes.Structure):
    _fields_ = [("keys", handle), ("A_csr", ctypes.POINTER(SparseMeta)), ("A_chunks", ctypes.POINTER(handle)),
                ("n_a", ctypes.c_size_t), ("B_csc", ctypes.POINTER(SparseMeta)), ("B_chunks", ctypes.POINTER(handle)),
                ("n_b", ctypes.c_size_t), ("mask0", handle)]


_SIGS += [
    ("spfhe_matmul_graph_create", ctypes.c_int, [handle, ctypes.POINTER(MatmulReq), ctypes.c_int,
                                                 ctypes.POINTER(handle)]),
    ("spfhe_matmul_graph_results", ctypes.c_int, [handle, ctypes.POINTER(handle), ctypes.c_size_t,
                                                  ctypes.POINTER(Stats)]),
    ("spfhe_matmul_graph_create_batch", ctypes.c_int, [handle, ctypes.c_size_t, ctypes.POINTER(MatmulReq),
                                                       ctypes.c_int, ctypes.POINTER(handle)]),
    ("spfhe_sparse_matmul_batch", ctypes.c_int, [handle, ctypes.c_size_t, ctypes.POINTER(MatmulReq),
                                                 ctypes.POINTER(handle), ctypes.c_size_t, ctypes.POINTER(Stats)]),
    ("spfhe_server_create", ctypes.c_int, [handle, ctypes.c_uint64, ctypes.POINTER(handle)]),
    ("spfhe_server_submit", ctypes.c_int, [handle, ctypes.POINTER(MatmulReq), ctypes.POINTER(ctypes.c_uint64)]),
    ("spfhe_server_wait", ctypes.c_int, [handle, ctypes.c_uint64, ctypes.POINTER(handle), ctypes.c_size_t,
                                         ctypes.POINTER(Stats), c_dblp]),
    ("spfhe_server_destroy", ctypes.c_int, [handle]),
    ("spfhe_server_inject_fault", ctypes.c_int, [handle, ctypes.c_uint64]),
    ("spfhe_server_info", ctypes.c_int, [handle, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.POINTER(ctypes.c_uint64)]),
    ("spfhe_tune_rotation_base", ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                                ctypes.POINTER(SparseMeta), ctypes.POINTER(SparseMeta),
                                                ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint32),
                                                ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
]

EXPORTED = [s[0] for s in _SIGS]


def lib():
    """The loaded library; raises if the CUDA extension is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libspfhe.so is not built (%s); run paper_2604_11659_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise SpfheError(status, lib().spfhe_last_error().decode(errors="replace"))


def _u64(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(c_u64p)


def _i32(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(c_i32p)


def _dbl(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(c_dblp)


def _handles(lst):
    arr = (handle * max(1, len(lst)))()
    for i, h in enumerate(lst):
        arr[i] = h
    return arr


# ---------------------------------------------------------------------------
# thin wrappers, one per entry point
# ---------------------------------------------------------------------------
def make_params(log_n: int, q_bits, K: int, dnum: int, scale: float, rot_base: int, p_bits: int = 60):
    qb = (ctypes.c_uint32 * len(q_bits))(*q_bits)
    p = Params(log_n, len(q_bits), ctypes.cast(qb, ctypes.POINTER(ctypes.c_uint32)), K, p_bits, dnum, float(scale),
               rot_base)
    p._keep = qb
    return p


def spfhe_ctx_create(params: Params, stream: int = 0):
    out = handle()
    _check(lib().spfhe_ctx_create(ctypes.byref(params), ctypes.c_void_p(stream or None), ctypes.byref(out)))
    return out


def spfhe_ctx_destroy(ctx):
    _check(lib().spfhe_ctx_destroy(ctx))


def spfhe_ctx_moduli(ctx, count: int):
    mods = np.zeros(count, np.uint64)
    psis = np.zeros(count, np.uint64)
    _check(lib().spfhe_ctx_moduli(ctx, _u64(mods), _u64(psis)))
    return mods, psis


def spfhe_sync(ctx):
    _check(lib().spfhe_sync(ctx))


def spfhe_ctx_set_match_batch(ctx, matches: int):
    _check(lib().spfhe_ctx_set_match_batch(ctx, int(matches)))


def spfhe_ctx_set_ntt_chunk(ctx, limbs: int):
    _check(lib().spfhe_ctx_set_ntt_chunk(ctx, int(limbs)))


def spfhe_ctx_set_ntt_split(ctx, pass_a_stages: int):
    _check(lib().spfhe_ctx_set_ntt_split(ctx, int(pass_a_stages)))


def spfhe_ctx_set_fusion(ctx, enable: bool):
    _check(lib().spfhe_ctx_set_fusion(ctx, 1 if enable else 0))


def spfhe_ctx_set_align_budget(ctx, nbytes: int):
    _check(lib().spfhe_ctx_set_align_budget(ctx, int(nbytes)))


def spfhe_ctx_set_ntt_variant(ctx, variant: int):
    _check(lib().spfhe_ctx_set_ntt_variant(ctx, int(variant)))


def spfhe_tune_ntt_chunk(ctx, ell: int, items: int, candidates):
    """Time each candidate chunk, set the fastest; returns (best, ms list)."""
    cand = (ctypes.c_uint32 * len(candidates))(*[int(c) for c in candidates])
    ms = (ctypes.c_double * len(candidates))()
    best = ctypes.c_uint32()
    _check(lib().spfhe_tune_ntt_chunk(ctx, int(ell), int(items), cand, len(candidates), ctypes.byref(best), ms))
    return int(best.value), [float(x) for x in ms]


def spfhe_launch_count(ctx) -> int:
    return int(lib().spfhe_launch_count(ctx))


def spfhe_prof_enable(ctx, enable: bool):
    _check(lib().spfhe_prof_enable(ctx, int(enable)))


def spfhe_prof_classes() -> int:
    return int(lib().spfhe_prof_classes())


def spfhe_prof_class_name(cls: int) -> str:
    return lib().spfhe_prof_class_name(cls).decode()


def spfhe_prof_read(ctx, cls: int) -> dict:
    la = ctypes.c_uint64()
    ms = ctypes.c_double()
    by = ctypes.c_double()
    wk = ctypes.c_double()
    _check(lib().spfhe_prof_read(ctx, cls, ctypes.byref(la), ctypes.byref(ms), ctypes.byref(by), ctypes.byref(wk)))
    return {"launches": int(la.value), "ms": ms.value, "bytes": by.value, "work": wk.value}


def spfhe_prof_transform_limbs(ctx, cls: int):
    """(first-pass limbs, second-pass limbs, fused second-pass limbs) of a
    transform class since spfhe_prof_enable."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().spfhe_prof_transform_limbs(ctx, cls, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def spfhe_prof_keyswitch(ctx):
    calls = ctypes.c_uint64()
    by = ctypes.c_double()
    _check(lib().spfhe_prof_keyswitch(ctx, ctypes.byref(calls), ctypes.byref(by)))
    return int(calls.value), by.value


def spfhe_prof_alu_peak(ctx):
    """(butterflies/s, split-product butterflies/s, mad.lo ops/s, mad.wide
    ops/s) measured on the GPU."""
    b, bs, i, w = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().spfhe_prof_alu_peak(ctx, ctypes.byref(b), ctypes.byref(bs), ctypes.byref(i), ctypes.byref(w)))
    return b.value, bs.value, i.value, w.value


def spfhe_prof_alu_rates(ctx):
    """(butterflies/s with mul_shoup3, mul_shoup3s, mul_shoup4s; mad.lo,
    mad.wide, mad.hi per second) measured on the GPU."""
    r = (ctypes.c_double * 6)()
    _check(lib().spfhe_prof_alu_rates(ctx, r, 6))
    return tuple(r)


def spfhe_prof_all(ctx) -> dict:
    out = {}
    for c in range(spfhe_prof_classes()):
        d = spfhe_prof_read(ctx, c)
        d["limbs"] = spfhe_prof_transform_limbs(ctx, c)
        out[spfhe_prof_class_name(c)] = d
    return out


def spfhe_keygen(ctx, seed: int):
    out = handle()
    _check(lib().spfhe_keygen(ctx, seed, ctypes.byref(out)))
    return out


def spfhe_keys_import(ctx, secret: np.ndarray, relin: np.ndarray, rot: dict):
    secret = np.ascontiguousarray(secret, dtype=np.int64)
    relin = np.ascontiguousarray(relin, dtype=np.uint64)
    amts = np.array(sorted(rot), dtype=np.int32)
    arrs = [np.ascontiguousarray(rot[int(a)], dtype=np.uint64) for a in amts]
    ptrs = (c_u64p * max(1, len(arrs)))(*[_u64(a) for a in arrs])
    out = handle()
    _check(lib().spfhe_keys_import(ctx, secret.ctypes.data_as(c_i64p), _u64(relin), len(arrs), _i32(amts),
                                   ptrs, ctypes.byref(out)))
    return out


def spfhe_keys_export(ctx, keys, n: int, key_shape):
    """Returns (secret, relin, {amount: key}) in the layout spfhe_keys_import
    takes; key_shape = (dnum, 2, L + K, n)."""
    count = ctypes.c_size_t(0)
    _check(lib().spfhe_keys_export(ctx, keys, None, None, ctypes.byref(count), None, None))
    secret = np.empty(n, dtype=np.int64)
    relin = np.empty(key_shape, dtype=np.uint64)
    amts = np.empty(max(1, count.value), dtype=np.int32)
    arrs = [np.empty(key_shape, dtype=np.uint64) for _ in range(count.value)]
    ptrs = (c_u64p * max(1, len(arrs)))(*[_u64(a) for a in arrs])
    _check(lib().spfhe_keys_export(ctx, keys, secret.ctypes.data_as(c_i64p), _u64(relin), ctypes.byref(count),
                                   _i32(amts), ptrs))
    return secret, relin, {int(a): k for a, k in zip(amts[: count.value], arrs)}


def spfhe_keys_free(keys):
    lib().spfhe_keys_free(keys)


def spfhe_encode(ctx, values, level: int, scale: float):
    v = np.asarray(values)
    re = np.ascontiguousarray(np.real(v), dtype=np.float64)
    im = np.ascontiguousarray(np.imag(v), dtype=np.float64) if np.iscomplexobj(v) else None
    out = handle()
    _check(lib().spfhe_encode(ctx, _dbl(re), _dbl(im), re.size, level, float(scale), ctypes.byref(out)))
    return out


def spfhe_pt_import(ctx, limbs: np.ndarray, scale: float, coeff_domain: bool):
    limbs = np.ascontiguousarray(limbs, dtype=np.uint64)
    out = handle()
    _check(lib().spfhe_pt_import(ctx, _u64(limbs), limbs.shape[0], float(scale), int(coeff_domain),
                                 ctypes.byref(out)))
    return out


def spfhe_pt_info(pt):
    lv = ctypes.c_uint32()
    sc = ctypes.c_double()
    _check(lib().spfhe_pt_info(pt, ctypes.byref(lv), ctypes.byref(sc)))
    return lv.value, sc.value


def spfhe_pt_export(ctx, pt, n: int) -> np.ndarray:
    level, _ = spfhe_pt_info(pt)
    out = np.zeros((level, n), np.uint64)
    _check(lib().spfhe_pt_export(ctx, pt, _u64(out)))
    return out


def spfhe_pt_free(pt):
    lib().spfhe_pt_free(pt)


def spfhe_decode(ctx, pt, n_vals: int) -> np.ndarray:
    re = np.zeros(n_vals)
    im = np.zeros(n_vals)
    _check(lib().spfhe_decode(ctx, pt, _dbl(re), _dbl(im), n_vals))
    return re + 1j * im


def spfhe_encrypt(ctx, keys, pt, seed: int):
    out = handle()
    _check(lib().spfhe_encrypt(ctx, keys, pt, seed, ctypes.byref(out)))
    return out


def spfhe_decrypt(ctx, keys, ct):
    out = handle()
    _check(lib().spfhe_decrypt(ctx, keys, ct, ctypes.byref(out)))
    return out


def spfhe_ct_import(ctx, limbs, level: int, scale: float):
    """limbs: numpy uint64 [2][level][n] (host) or an int device/host address."""
    out = handle()
    if isinstance(limbs, np.ndarray):
        limbs = np.ascontiguousarray(limbs, dtype=np.uint64)
        ptr = limbs.ctypes.data
    else:
        ptr = int(limbs)
    _check(lib().spfhe_ct_import(ctx, ctypes.c_void_p(ptr), level, float(scale), ctypes.byref(out)))
    if isinstance(limbs, np.ndarray):
        spfhe_sync(ctx)   # the host array may be released by the caller after return
    return out


def spfhe_ct_info(ct):
    lv = ctypes.c_uint32()
    sc = ctypes.c_double()
    _check(lib().spfhe_ct_info(ct, ctypes.byref(lv), ctypes.byref(sc)))
    return lv.value, sc.value


def spfhe_ct_export(ctx, ct, n: int, out=None) -> np.ndarray:
    level, _ = spfhe_ct_info(ct)
    if out is None:
        out = np.zeros((2, level, n), np.uint64)
    _check(lib().spfhe_ct_export(ctx, ct, ctypes.c_void_p(out.ctypes.data)))
    return out


def spfhe_ct_free(ct):
    lib().spfhe_ct_free(ct)


def spfhe_mult_relin(ctx, keys, a, b):
    out = handle()
    _check(lib().spfhe_mult_relin(ctx, keys, a, b, ctypes.byref(out)))
    return out


def spfhe_rescale(ctx, ct):
    _check(lib().spfhe_rescale(ctx, ct))


def spfhe_rotate(ctx, keys, ct, r: int):
    out = handle()
    _check(lib().spfhe_rotate(ctx, keys, ct, int(r), ctypes.byref(out)))
    return out


def spfhe_mul_plain(ctx, ct, pt):
    out = handle()
    _check(lib().spfhe_mul_plain(ctx, ct, pt, ctypes.byref(out)))
    return out


def spfhe_add(ctx, a, b):
    out = handle()
    _check(lib().spfhe_add(ctx, a, b, ctypes.byref(out)))
    return out


def spfhe_ntt(ctx, dev_ptr: int, mod_idx, inverse: bool):
    mi = np.ascontiguousarray(mod_idx, dtype=np.int32)
    _check(lib().spfhe_ntt(ctx, ctypes.c_void_p(dev_ptr), mi.size, _i32(mi), int(inverse)))


def spfhe_rescale_noalloc(ctx, in_dev_ptr: int, level: int, out_dev_ptr: int):
    _check(lib().spfhe_rescale_noalloc(ctx, ctypes.c_void_p(in_dev_ptr), level, ctypes.c_void_p(out_dev_ptr)))


def sparse_meta(indptr: np.ndarray, indices: np.ndarray, rows: int, cols: int) -> SparseMeta:
    ip = np.ascontiguousarray(indptr, dtype=np.int32)
    ix = np.ascontiguousarray(indices, dtype=np.int32)
    m = SparseMeta(rows, cols, int(ip[-1]) if ip.size else 0, _i32(ip), _i32(ix) if ix.size else None)
    m._keep = (ip, ix)
    return m


def spfhe_plan_matches(A: SparseMeta, B: SparseMeta) -> np.ndarray:
    cnt = ctypes.c_uint64(0)
    _check(lib().spfhe_plan_matches(ctypes.byref(A), ctypes.byref(B), None, ctypes.byref(cnt)))
    out = np.zeros((max(1, cnt.value), 5), np.int32)
    _check(lib().spfhe_plan_matches(ctypes.byref(A), ctypes.byref(B), _i32(out), ctypes.byref(cnt)))
    return out[: cnt.value]


def spfhe_sparse_matmul_ct_ct(ctx, keys, A: SparseMeta, A_chunks, B: SparseMeta, B_chunks, mask0, n_c: int):
    outs = (handle * n_c)()
    st = Stats()
    _check(lib().spfhe_sparse_matmul_ct_ct(ctx, keys, ctypes.byref(A), _handles(A_chunks), len(A_chunks),
                                           ctypes.byref(B), _handles(B_chunks), len(B_chunks), mask0, outs, n_c,
                                           ctypes.byref(st)))
    return [handle(outs[i]) for i in range(n_c)], st.as_dict()


def spfhe_sparse_matmul_ct_ct_grouped(ctx, keys, A: SparseMeta, A_chunks, B: SparseMeta, B_chunks, mask0, n_c: int,
                                      merge_digits: bool = True):
    outs = (handle * n_c)()
    st = Stats()
    _check(lib().spfhe_sparse_matmul_ct_ct_grouped(ctx, keys, ctypes.byref(A), _handles(A_chunks), len(A_chunks),
                                                   ctypes.byref(B), _handles(B_chunks), len(B_chunks), mask0,
                                                   1 if merge_digits else 0, outs, n_c, ctypes.byref(st)))
    return [handle(outs[i]) for i in range(n_c)], st.as_dict()


def matmul_req(keys, A: SparseMeta, A_chunks, B: SparseMeta, B_chunks, mask0=None) -> MatmulReq:
    a = _handles(A_chunks)
    b = _handles(B_chunks)
    r = MatmulReq(keys, ctypes.pointer(A), a, len(A_chunks), ctypes.pointer(B), b, len(B_chunks), mask0)
    r._keep = (A, B, a, b)
    return r


def n_result_chunks(A: SparseMeta, B: SparseMeta, slots: int) -> int:
    return max(1, -(-(A.rows * B.cols) // slots))


def spfhe_sparse_matmul_batch(ctx, reqs, n_c_per_req):
    arr = (MatmulReq * max(1, len(reqs)))(*reqs)
    total = sum(n_c_per_req)
    outs = (handle * max(1, total))()
    st = (Stats * max(1, len(reqs)))()
    _check(lib().spfhe_sparse_matmul_batch(ctx, len(reqs), arr, outs, total, st))
    res, o = [], 0
    for k in n_c_per_req:
        res.append([handle(outs[o + i]) for i in range(k)])
        o += k
    return res, [st[i].as_dict() for i in range(len(reqs))]


def spfhe_server_create(ctx, hbm_budget_bytes: int):
    out = handle()
    _check(lib().spfhe_server_create(ctx, int(hbm_budget_bytes), ctypes.byref(out)))
    return out


def spfhe_server_submit(srv, req: MatmulReq) -> int:
    t = ctypes.c_uint64()
    _check(lib().spfhe_server_submit(srv, ctypes.byref(req), ctypes.byref(t)))
    return int(t.value)


def spfhe_server_wait(srv, ticket: int, n_c: int):
    outs = (handle * n_c)()
    st = Stats()
    lat = ctypes.c_double()
    _check(lib().spfhe_server_wait(srv, ticket, outs, n_c, ctypes.byref(st), ctypes.byref(lat)))
    return [handle(outs[i]) for i in range(n_c)], st.as_dict(), lat.value


def spfhe_tune_rotation_base(log_n: int, L: int, K: int, dnum: int, A: SparseMeta, B: SparseMeta,
                             key_budget_bytes: int):
    b = ctypes.c_uint32()
    ks = ctypes.c_uint64()
    kb = ctypes.c_uint64()
    _check(lib().spfhe_tune_rotation_base(log_n, L, K, dnum, ctypes.byref(A), ctypes.byref(B), int(key_budget_bytes),
                                          ctypes.byref(b), ctypes.byref(ks), ctypes.byref(kb)))
    return int(b.value), int(ks.value), int(kb.value)


def spfhe_server_destroy(srv):
    _check(lib().spfhe_server_destroy(srv))


def spfhe_server_inject_fault(srv, ticket: int):
    _check(lib().spfhe_server_inject_fault(srv, int(ticket)))


def spfhe_server_info(srv):
    """(bytes reserved for the shared batch buffers, bytes held by admitted
    unfinished requests, requests re-run alone after a failed wave)"""
    ws, used, retried = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().spfhe_server_info(srv, ctypes.byref(ws), ctypes.byref(used), ctypes.byref(retried)))
    return int(ws.value), int(used.value), int(retried.value)


NAIVE_DENSE, NAIVE_SPARSE, NAIVE_SPARSE_LITERAL = 0, 1, 2


def spfhe_naive_matmul_ct_ct(ctx, keys, mode: int, A_nonzero: np.ndarray, B_nonzero: np.ndarray, A_chunks, B_chunks,
                             mask0, n_c: int):
    """Element-wise baseline (Naive Dense / Naive Sparse) over row-major dense
    packing; A_nonzero / B_nonzero: boolean zero patterns (rows x inner,
    inner x cols).  Returns (result handles, stats)."""
    an = np.ascontiguousarray(A_nonzero, dtype=np.uint8)
    bn = np.ascontiguousarray(B_nonzero, dtype=np.uint8)
    rows, inner = an.shape
    cols = bn.shape[1]
    outs = (handle * n_c)()
    st = Stats()
    _check(lib().spfhe_naive_matmul_ct_ct(ctx, keys, int(mode), rows, inner, cols, an.ctypes.data, bn.ctypes.data,
                                          _handles(A_chunks), len(A_chunks), _handles(B_chunks), len(B_chunks), mask0,
                                          outs, n_c, ctypes.byref(st)))
    return [handle(outs[i]) for i in range(n_c)], st.as_dict()


def spfhe_sparse_matmul_ct_pt(ctx, keys, A: SparseMeta, A_chunks, B: SparseMeta, B_values, B_pts, n_c: int):
    outs = (handle * n_c)()
    st = Stats()
    bv = None if B_values is None else np.ascontiguousarray(B_values, dtype=np.float64)
    bp = None if B_pts is None else _handles(B_pts)
    _check(lib().spfhe_sparse_matmul_ct_pt(ctx, keys, ctypes.byref(A), _handles(A_chunks), len(A_chunks),
                                           ctypes.byref(B), _dbl(bv), bp, outs, n_c, ctypes.byref(st)))
    return [handle(outs[i]) for i in range(n_c)], st.as_dict()


def spfhe_sparse_matmul_ct_pt_grouped(ctx, keys, A: SparseMeta, A_chunks, B: SparseMeta, B_values, B_pts, n_c: int,
                                      merge_digits: bool = True):
    outs = (handle * n_c)()
    st = Stats()
    bv = None if B_values is None else np.ascontiguousarray(B_values, dtype=np.float64)
    bp = None if B_pts is None else _handles(B_pts)
    _check(lib().spfhe_sparse_matmul_ct_pt_grouped(ctx, keys, ctypes.byref(A), _handles(A_chunks), len(A_chunks),
                                                   ctypes.byref(B), _dbl(bv), bp, 1 if merge_digits else 0, outs,
                                                   n_c, ctypes.byref(st)))
    return [handle(outs[i]) for i in range(n_c)], st.as_dict()


def spfhe_matmul_graph_create(ctx, req, variant: int = 0):
    out = handle()
    _check(lib().spfhe_matmul_graph_create(ctx, ctypes.byref(req), int(variant), ctypes.byref(out)))
    return out


def spfhe_matmul_graph_create_batch(ctx, reqs, variant: int = 0):
    arr = (MatmulReq * max(1, len(reqs)))(*reqs)
    out = handle()
    _check(lib().spfhe_matmul_graph_create_batch(ctx, len(reqs), arr, int(variant), ctypes.byref(out)))
    return out


def spfhe_matmul_graph_results_batch(g, n_c_per_req):
    """Every request's result handles (a list per request) and counters."""
    total = sum(n_c_per_req)
    outs = (handle * max(1, total))()
    st = (Stats * max(1, len(n_c_per_req)))()
    _check(lib().spfhe_matmul_graph_results(g, outs, total, st))
    res, o = [], 0
    for k in n_c_per_req:
        res.append([handle(outs[o + i]) for i in range(k)])
        o += k
    return res, [st[i].as_dict() for i in range(len(n_c_per_req))]


def spfhe_matmul_graph_launch(g):
    _check(lib().spfhe_matmul_graph_launch(g))


def spfhe_matmul_graph_results(g, n_c: int):
    outs = (handle * n_c)()
    st = Stats()
    _check(lib().spfhe_matmul_graph_results(g, outs, n_c, ctypes.byref(st)))
    return [handle(outs[i]) for i in range(n_c)], st.as_dict()


def spfhe_matmul_graph_free(g):
    lib().spfhe_matmul_graph_free(g)


def spfhe_ct_overwrite(ctx, ct, limbs):
    """Copy new limbs ([2][level][n] uint64, host numpy) into ct; waits for
    the copy (the host buffer may be reused on return)."""
    a = np.ascontiguousarray(limbs, dtype=np.uint64)
    _check(lib().spfhe_ct_overwrite(ctx, ct, ctypes.c_void_p(a.ctypes.data)))
    spfhe_sync(ctx)
