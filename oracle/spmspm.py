"""Oracle for Alg. 1 + Alg. 2 (CSR x CSC encrypted sparse matmul), plain CPU.

TEST INFRASTRUCTURE ONLY (tests/, __graft_entry__.smoke(), bench.py's
cpu_baseline leg).  Follows the paper step by step; see oracle/ckks.py for the
readings R1..R11 it relies on.  spmspm_ct_ct_grouped is a reordering of
Alg. 2 (lazy accumulation), not the paper's op order; it exists to check the
library's variant of the same name.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from .ckks import Ct, Keys, Oracle, Pt, _p, addmod, lib, rotation_plan


# ---------------------------------------------------------------------------
# plaintext side: formats, brute force, Alg. 1 merge
# ---------------------------------------------------------------------------
def dense_to_csr(M: np.ndarray):
    """CSR of a dense matrix: (indptr, indices, data) with rows of sorted
    column indices (Sec. 2.3, Fig. 2)."""
    M = np.asarray(M)
    indptr = [0]
    indices = []
    data = []
    for i in range(M.shape[0]):
        for k in range(M.shape[1]):
            if M[i, k] != 0:
                indices.append(k)
                data.append(float(M[i, k]))
        indptr.append(len(indices))
    return np.array(indptr, np.int32), np.array(indices, np.int32), np.array(data, np.float64)


def dense_to_csc(M: np.ndarray):
    """CSC: the CSR of the transpose (column pointers, row indices)."""
    return dense_to_csr(np.asarray(M).T)


def matmul_fp64(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """C[i, j] = sum_k A[i, k] B[k, j] in FP64 (Sec. 4.2's plaintext baseline)."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    C = np.zeros((A.shape[0], B.shape[1]))
    for i in range(A.shape[0]):
        for j in range(B.shape[1]):
            C[i, j] = np.sum(A[i, :] * B[:, j])
    return C


def frobenius(X: np.ndarray, Y: np.ndarray) -> float:
    """||X - Y||_F, the accuracy measure of Sec. 4.2."""
    return float(np.sqrt(np.sum((np.asarray(X) - np.asarray(Y)) ** 2)))


@dataclass
class Match:
    i: int
    j: int
    k: int
    a_pos: int
    b_pos: int


def alg1_matches(A_indptr, A_indices, B_indptr, B_indices, rows: int, cols: int) -> list:
    """Alg. 1's merge: for every (i, j), walk row i of A (CSR) and column j of
    B (CSC) with two pointers; a match is a_col == b_row (reading R10 for the
    loop bounds)."""
    out = []
    for i in range(rows):
        for j in range(cols):
            a_start, a_end = int(A_indptr[i]), int(A_indptr[i + 1])
            b_start, b_end = int(B_indptr[j]), int(B_indptr[j + 1])
            a_pos, b_pos = a_start, b_start
            while a_pos < a_end and b_pos < b_end:
                a_col = int(A_indices[a_pos])
                b_row = int(B_indices[b_pos])
                if a_col == b_row:
                    out.append(Match(i, j, a_col, a_pos, b_pos))
                    a_pos += 1
                    b_pos += 1
                elif a_col < b_row:
                    a_pos += 1
                else:
                    b_pos += 1
    return out


# ---------------------------------------------------------------------------
# encrypted side
# ---------------------------------------------------------------------------
def pack_values(data: np.ndarray, slots: int) -> list:
    """Reading R3: value p in slot p mod S of chunk p // S, zero padding."""
    nchunks = max(1, -(-len(data) // slots))
    out = []
    for c in range(nchunks):
        z = np.zeros(slots)
        part = data[c * slots:(c + 1) * slots]
        z[: len(part)] = part
        out.append(z)
    return out


def mask_scale(orc: Oracle, ell: int | None = None) -> float:
    """Reading R6: for operands at level ell (default L) the mask is encoded at
    the scale of q_{ell-2}, the prime the second rescale removes."""
    ell = orc.P.L if ell is None else ell
    return float(orc.mods[ell - 2])


def result_scale(orc: Oracle, ell: int | None = None, scale_a: float | None = None,
                 scale_b: float | None = None) -> float:
    """Scale of every accumulated product: scale_A * scale_B / q_{ell-1} (R6)."""
    ell = orc.P.L if ell is None else ell
    sa = orc.P.scale if scale_a is None else scale_a
    sb = orc.P.scale if scale_b is None else scale_b
    return sa * sb / orc.mods[ell - 1]


@dataclass
class OpCounts:
    matches: int = 0
    ks_relin: int = 0
    ks_align: int = 0
    ks_final: int = 0
    rescales: int = 0


def make_mask(orc: Oracle, slot: int, level: int) -> Pt:
    """makeMask(size^2, min_pos) of Alg. 2: one-hot plaintext at `slot` for a
    product at `level` (= operand level - 1), scale q_{level-1} (readings R8,
    R6)."""
    return orc.encode_onehot(1.0, slot, level, float(orc.mods[level - 1]))


def spmspm_ct_ct(orc: Oracle, keys: Keys, A_csr, A_cts: list, B_csc, B_cts: list,
                 rows: int, cols: int, mask_pt: Pt | None = None, counts: OpCounts | None = None,
                 match_limit: int | None = None) -> list:
    """Alg. 1 + Alg. 2 over encrypted operands.

    A_csr = (indptr, indices) of A (rows x inner), B_csc = (indptr, indices) of
    B (cols x inner column pointers).  A_cts / B_cts: packed chunks (R3), all
    at one level ell >= 3 (L for fresh ciphertexts).  Returns the result
    chunks (R3) at level ell-2.

    mask_pt: optional one-hot mask at slot 0 (level L-1) to use in place of
    this oracle's own encoding; the mask for slot p is then the automorphism
    X -> X^(5^-p) of it, which is exactly the encoding of e_p (R8).
    match_limit: process only the first N matches (timing samples)."""
    P = orc.P
    S = P.slots
    if counts is None:
        counts = OpCounts()
    nres = max(1, -(-(rows * cols) // S))
    ell = A_cts[0].level
    result = [orc.zero_ct(ell - 2, result_scale(orc, ell, A_cts[0].scale, B_cts[0].scale)) for _ in range(nres)]
    matches = alg1_matches(A_csr[0], A_csr[1], B_csc[0], B_csc[1], rows, cols)
    if match_limit is not None:
        matches = matches[:match_limit]
    rot_cache = {}

    def rotated(which: str, chunk: int, amount: int) -> Ct:
        # memoisation of a deterministic function: same bits as recomputing
        key = (which, chunk, amount)
        if key not in rot_cache:
            src = (A_cts if which == "A" else B_cts)[chunk]
            rot_cache[key] = orc.rotate(src, amount, keys)
            counts.ks_align += len(rotation_plan(amount, S, P.rot_base))
        return rot_cache[key]

    for mt in matches:
        counts.matches += 1
        ca, sa = divmod(mt.a_pos, S)
        cb, sb = divmod(mt.b_pos, S)
        vA, vB = A_cts[ca], B_cts[cb]
        min_slot = sa
        if sa < sb:
            vB = rotated("B", cb, sb - sa)
            min_slot = sa
        elif sb < sa:
            vA = rotated("A", ca, sa - sb)
            min_slot = sb
        # Alg. 2
        dot = orc.mult_relin(vA, vB, keys)
        counts.ks_relin += 1
        dot = orc.rescale(dot)
        if mask_pt is None:
            mask = make_mask(orc, min_slot, dot.level)
        else:
            g = pow(pow(5, min_slot, 2 * P.n), -1, 2 * P.n)
            m = np.stack([_automorph_limb(orc, mask_pt.m[i], g, q)
                          for i, q in enumerate(orc.mods[: dot.level])])
            mask = Pt(m, mask_pt.scale)
        dot = orc.mul_plain(dot, mask)
        # Relinearize after a plaintext product: nothing to switch (R7)
        dot = orc.rescale(dot)
        counts.rescales += 2
        t = mt.i * cols + mt.j
        rc, ts = divmod(t, S)
        rot_idx = (min_slot - ts) % S
        counts.ks_final += len(rotation_plan(rot_idx, S, P.rot_base))
        dot = orc.rotate(dot, rot_idx, keys)
        result[rc] = orc.add(result[rc], dot)
    return result


# ---------------------------------------------------------------------------
# lazy accumulation: a reordering of Alg. 2 (not the paper's op order)
# ---------------------------------------------------------------------------
def make_mask_grouped(orc: Oracle, slot: int, ell: int) -> Pt:
    """One-hot plaintext e_slot at the operands' level ell, scale q_{ell-2}:
    the mask of the lazy variant multiplies the unrescaled tensor product."""
    return orc.encode_onehot(1.0, slot, ell, float(orc.mods[ell - 2]))


def _rescale_polys(orc: Oracle, polys: list) -> list:
    """Rescale (drop the top prime) of each polynomial, as orc.rescale does
    for the two of a ciphertext."""
    out = []
    for d in polys:
        c = np.ascontiguousarray(d.copy())
        ell = c.shape[0]
        lib().or_rescale(ctypes.byref(orc._cs), _p(c), ell)
        out.append(c[: ell - 1].copy())
    return out


def group_key(mt: Match, S: int, cols: int) -> tuple:
    """(result chunk, final rotation amount) of a match (reading R3/R4)."""
    sa, sb = mt.a_pos % S, mt.b_pos % S
    t = mt.i * cols + mt.j
    return t // S, (min(sa, sb) - t % S) % S


def spmspm_ct_ct_grouped(orc: Oracle, keys: Keys, A_csr, A_cts: list, B_csc, B_cts: list,
                         rows: int, cols: int, mask_pt: Pt | None = None, merge_digits: bool = True,
                         counts: OpCounts | None = None) -> list:
    """Lazy accumulation of Alg. 2's products.

    The tensor product is Alg. 2's; alignment rotations are computed per
    source ciphertext digit by digit from the top with hoisted ModUps
    (alignment_rotations).  Then, instead of relinearising, rescaling,
    masking and rotating every product:
      1. each tensor product (three polynomials at the operands' level ell)
         is multiplied by its mask e_{min_slot} (at level ell, scale
         q_{ell-2}) and summed into the group of matches that share the
         result chunk and the final rotation amount r;
      2. per group: a rescale of the three polynomials (level ell-1), one
         relinearisation (a key switch of the s^2 part) at level ell-1, a
         rescale of the resulting ciphertext (level ell-2), and a rotation
         by the lowest base-b digit of r;
      3. merge_digits: the rotated groups are summed per (chunk, remaining
         amount) and every sum is rotated by its next digit, digit by digit,
         until nothing remains; otherwise each group is rotated by the whole
         of r (its rotation plan);
      4. everything left for a result chunk is added into it.
    Rotation and relinearisation are linear in the ciphertext, so the result
    decrypts to the same product as Alg. 2 (within CKKS noise); the
    ciphertext bits differ from Alg. 2's.  Result chunks: level ell-2, scale
    scale_A scale_B / q_{ell-1}.  mask_pt: the slot-0 mask at level ell
    (make_mask_grouped); the mask for slot p is its automorphism
    X -> X^(5^-p)."""
    P = orc.P
    S = P.slots
    b = P.rot_base
    if counts is None:
        counts = OpCounts()
    ell = A_cts[0].level
    nres = max(1, -(-(rows * cols) // S))
    rscale = result_scale(orc, ell, A_cts[0].scale, B_cts[0].scale)
    result = [orc.zero_ct(ell - 2, rscale) for _ in range(nres)]
    matches = alg1_matches(A_csr[0], A_csr[1], B_csc[0], B_csc[1], rows, cols)
    if mask_pt is None:
        mask_pt = make_mask_grouped(orc, 0, ell)
    mods = orc.mods[:ell]
    mi = np.arange(ell, dtype=np.int32)
    # every alignment rotation of a source, digit by digit from the top,
    # each stage hoisted (alignment_rotations)
    need = {}
    for mt in matches:
        ca, sa = divmod(mt.a_pos, S)
        cb, sb = divmod(mt.b_pos, S)
        if sa < sb:
            need.setdefault(("B", cb), set()).add(sb - sa)
        elif sb < sa:
            need.setdefault(("A", ca), set()).add(sa - sb)
    rot_cache = {}
    for (which, chunk), amts in sorted(need.items()):
        src = (A_cts if which == "A" else B_cts)[chunk]
        for amt, ct in alignment_rotations(orc, keys, src, sorted(amts), counts).items():
            rot_cache[(which, chunk, amt)] = ct

    def rotated(which: str, chunk: int, amount: int) -> Ct:
        return rot_cache[(which, chunk, amount)]

    groups = {}
    for mt in matches:
        counts.matches += 1
        ca, sa = divmod(mt.a_pos, S)
        cb, sb = divmod(mt.b_pos, S)
        vA, vB = A_cts[ca], B_cts[cb]
        min_slot = sa
        if sa < sb:
            vB = rotated("B", cb, sb - sa)
        elif sb < sa:
            vA = rotated("A", ca, sa - sb)
            min_slot = sb
        d0, d1, d2, _ = orc.tensor(vA, vB)
        g = pow(pow(5, min_slot, 2 * P.n), -1, 2 * P.n)
        m = np.stack([_automorph_limb(orc, mask_pt.m[i], g, q) for i, q in enumerate(mods)])
        prod = [orc.rns_polymul(d, m, mi) for d in (d0, d1, d2)]
        key = group_key(mt, S, cols)
        if key in groups:
            groups[key] = [np.stack([addmod(x[i], y[i], q) for i, q in enumerate(mods)])
                           for x, y in zip(groups[key], prod)]
        else:
            groups[key] = prod

    sc = A_cts[0].scale * B_cts[0].scale * mask_pt.scale / orc.mods[ell - 1]
    done = []
    for key in sorted(groups):
        # relinearise between the rescales: the rounding of the first rescale
        # on the s^2 part is then divided by q_{ell-2} like everything else
        d = _rescale_polys(orc, groups[key])
        ct = orc.relinearize(d[0], d[1], d[2], sc, keys)
        ct = orc.rescale(ct)
        counts.rescales += 2
        counts.ks_relin += 1
        done.append((key, ct))
    _rotation_tree(orc, keys, done, result, merge_digits, counts)
    return result


def alignment_rotations(orc: Oracle, keys: Keys, src: Ct, amounts: list, counts: OpCounts) -> dict:
    """src rotated by every amount (0 < amount < S), digit by digit from the
    highest base-b digit down: at each digit position the ciphertexts that
    share the higher digits are rotated by every needed digit with one hoisted
    ModUp (Oracle.rotate_hoisted).  Returns amount -> ciphertext."""
    P = orc.P
    S, b = P.slots, P.rot_base
    top = 1
    while top * b < S:
        top *= b
    cur = {0: src}
    w = top
    while w >= 1:
        nxt = {}
        for H, ct in sorted(cur.items()):
            digs = sorted({(a // w) % b for a in amounts if a - a % (w * b) == H})
            rot = [d for d in digs if d]
            outs = orc.rotate_hoisted(ct, [d * w for d in rot], keys) if rot else []
            counts.ks_align += len(rot)
            for d in digs:
                nxt[H + d * w] = ct if d == 0 else outs[rot.index(d)]
        cur = nxt
        w //= b
    return {a: cur[a] for a in amounts}


def _rotation_tree(orc: Oracle, keys: Keys, items: list, result: list, merge_digits: bool, counts: OpCounts):
    """Rotate every ((chunk, r), ct) of `items` left by r and add it into
    result[chunk].  merge_digits: rotate by the lowest base-b digit of r, sum
    per (chunk, remaining amount), then rotate each sum by its next digit,
    digit by digit; otherwise rotate each item by r through its plan."""
    P = orc.P
    S, b = P.slots, P.rot_base
    stage = {}
    for (rc, r), ct in items:
        step = r % b if merge_digits else r
        if step:
            counts.ks_final += len(rotation_plan(step, S, P.rot_base))
            ct = orc.rotate(ct, step, keys)
        nk = (rc, r - step)
        stage[nk] = orc.add(stage[nk], ct) if nk in stage else ct
    w = b
    while any(rem for (_, rem) in stage):
        nxt = {}
        for (rc, rem) in sorted(stage):
            ct = stage[(rc, rem)]
            d = (rem // w) % b
            if d:
                ct = orc.rotate_single(ct, d * w, keys)
                counts.ks_final += 1
            nk = (rc, rem - d * w)
            nxt[nk] = orc.add(nxt[nk], ct) if nk in nxt else ct
        stage = nxt
        w *= b
    for (rc, _), ct in sorted(stage.items()):
        result[rc] = orc.add(result[rc], ct)


def spmspm_ct_pt_grouped(orc: Oracle, keys: Keys, A_csr, A_cts: list, B_csc, B_data: np.ndarray,
                         rows: int, cols: int, b_pts: list | None = None, merge_digits: bool = True,
                         counts: OpCounts | None = None) -> list:
    """Lazy accumulation of the ct x pt products (reading R9): the weight
    plaintexts B[k, j] e_{a_slot} of the matches sharing the result chunk and
    the final rotation amount r = a_slot - t are summed per A chunk, each sum
    multiplies its A chunk, the products of a group are added, rescaled once
    and rotated through _rotation_tree.  Result at level L-1, scale Delta."""
    P = orc.P
    S = P.slots
    if counts is None:
        counts = OpCounts()
    nres = max(1, -(-(rows * cols) // S))
    result = [orc.zero_ct(P.L - 1, P.scale) for _ in range(nres)]
    mods = orc.mods[: P.L]
    sums = {}
    for mt in alg1_matches(A_csr[0], A_csr[1], B_csc[0], B_csc[1], rows, cols):
        counts.matches += 1
        ca, sa = divmod(mt.a_pos, S)
        if b_pts is None:
            pt = orc.encode_onehot(float(B_data[mt.b_pos]), sa, P.L, weight_scale(orc))
        else:
            g = pow(pow(5, sa, 2 * P.n), -1, 2 * P.n)
            base = b_pts[mt.b_pos]
            pt = Pt(np.stack([_automorph_limb(orc, base.m[i], g, q) for i, q in enumerate(mods)]), base.scale)
        t = mt.i * cols + mt.j
        key = (t // S, (sa - t % S) % S)
        sk = (key, ca)
        if sk in sums:
            sums[sk] = Pt(np.stack([addmod(sums[sk].m[i], pt.m[i], q) for i, q in enumerate(mods)]), pt.scale)
        else:
            sums[sk] = pt
    groups = {}
    for (key, ca) in sorted(sums):
        prod = orc.mul_plain(A_cts[ca], sums[(key, ca)])
        groups[key] = orc.add(groups[key], prod) if key in groups else prod
    done = []
    for key in sorted(groups):
        done.append((key, orc.rescale(groups[key])))
        counts.rescales += 1
    _rotation_tree(orc, keys, done, result, merge_digits, counts)
    return result


def grouped_key_switches(A_csr, B_csc, rows: int, cols: int, slots: int, base: int, merge_digits: bool = True):
    """(relinearisations, final-rotation key switches) of the lazy variant,
    counted from the plan alone."""
    groups = set()
    for mt in alg1_matches(A_csr[0], A_csr[1], B_csc[0], B_csc[1], rows, cols):
        groups.add(group_key(mt, slots, cols))
    if not merge_digits:
        return len(groups), sum(len(rotation_plan(r, slots, base)) for _, r in groups)
    ks = sum(1 for _, r in groups if r % base)
    keys = {(rc, r - r % base) for rc, r in groups}
    w = base
    while any(rem for _, rem in keys):
        ks += sum(1 for _, rem in keys if (rem // w) % base)
        keys = {(rc, rem - ((rem // w) % base) * w) for rc, rem in keys}
        w *= base
    return len(groups), ks


def _automorph_limb(orc: Oracle, a: np.ndarray, g: int, q: int) -> np.ndarray:
    from .ckks import automorphism
    return automorphism(a, g, q)


def weight_scale(orc: Oracle) -> float:
    """Reading R9: B's plaintext is encoded at the scale of q_{L-1}."""
    return float(orc.mods[orc.P.L - 1])


def spmspm_ct_pt(orc: Oracle, keys: Keys, A_csr, A_cts: list, B_csc, B_data: np.ndarray,
                 rows: int, cols: int, b_pts: list | None = None, counts: OpCounts | None = None,
                 match_limit: int | None = None) -> list:
    """Encrypted A (CSR, packed) times plaintext B (CSC) following reading R9:
    per match, pt = encode(B[k, j] * e_{a_slot}) at scale q_{L-1}, then
    ct x pt -> rescale -> EvalRotate(a_slot - t) -> EvalAdd.  Result at level
    L-1, scale Delta.

    b_pts: optional per-nonzero plaintexts of B (CSC order) encoding
    B[k, j] * e_0 at level L; the plaintext for slot p is then its
    automorphism X -> X^(5^-p) (exactly the encoding of B[k, j] e_p)."""
    P = orc.P
    S = P.slots
    if counts is None:
        counts = OpCounts()
    nres = max(1, -(-(rows * cols) // S))
    result = [orc.zero_ct(P.L - 1, P.scale) for _ in range(nres)]
    matches = alg1_matches(A_csr[0], A_csr[1], B_csc[0], B_csc[1], rows, cols)
    if match_limit is not None:
        matches = matches[:match_limit]
    for mt in matches:
        counts.matches += 1
        ca, sa = divmod(mt.a_pos, S)
        if b_pts is None:
            pt = orc.encode_onehot(float(B_data[mt.b_pos]), sa, P.L, weight_scale(orc))
        else:
            g = pow(pow(5, sa, 2 * P.n), -1, 2 * P.n)
            base = b_pts[mt.b_pos]
            pt = Pt(np.stack([_automorph_limb(orc, base.m[i], g, q) for i, q in enumerate(orc.mods[: P.L])]),
                    base.scale)
        dot = orc.mul_plain(A_cts[ca], pt)
        dot = orc.rescale(dot)
        counts.rescales += 1
        t = mt.i * cols + mt.j
        rc, ts = divmod(t, S)
        rot_idx = (sa - ts) % S
        counts.ks_final += len(rotation_plan(rot_idx, S, P.rot_base))
        dot = orc.rotate(dot, rot_idx, keys)
        result[rc] = orc.add(result[rc], dot)
    return result


def decrypt_result(orc: Oracle, keys: Keys, chunks: list, rows: int, cols: int) -> np.ndarray:
    """Decrypt + decode the result chunks into a rows x cols matrix (R3)."""
    S = orc.P.slots
    vals = []
    for ct in chunks:
        vals.append(np.real(orc.decode(orc.decrypt(ct, keys))))
    flat = np.concatenate(vals)[: rows * cols]
    return flat.reshape(rows, cols)


def final_rotation_amounts(A_csr, B_csc, rows: int, cols: int, slots: int) -> list:
    """Every rotation amount Alg. 1 + Alg. 2 will request (for key generation)."""
    amts = set()
    for mt in alg1_matches(A_csr[0], A_csr[1], B_csc[0], B_csc[1], rows, cols):
        sa, sb = mt.a_pos % slots, mt.b_pos % slots
        if sa != sb:
            amts.add(abs(sa - sb))
        amts.add((min(sa, sb) - (mt.i * cols + mt.j) % slots) % slots)
    return sorted(amts)


# ---------------------------------------------------------------------------
# the paper's element-wise baselines (Sec. 4): Naive Dense and Naive Sparse
# ---------------------------------------------------------------------------
NAIVE_DENSE, NAIVE_SPARSE, NAIVE_SPARSE_LITERAL = 0, 1, 2


def dense_pack(M: np.ndarray, slots: int) -> list:
    """Reading R16: a dense operand packed row-major, element (r, c) of an
    R x C matrix in slot (r C + c) mod S of chunk (r C + c) // S (zeros
    included)."""
    return pack_values(np.asarray(M, dtype=np.float64).reshape(-1), slots)


def naive_triples(A_nz: np.ndarray, B_nz: np.ndarray, mode: int) -> list:
    """The (i, j, k) products an element-wise method computes, in the order
    i, j, k (every element multiplied individually, Sec. 4):
      NAIVE_DENSE: all of them;
      NAIVE_SPARSE: those with A[i, k] and B[k, j] both nonzero (reading G15:
        skipping a product when either value is zero, which still gives the
        exact product);
      NAIVE_SPARSE_LITERAL: those with at least one of the two nonzero (the
        printed rule: skip only where both values are zero)."""
    rows, inner = A_nz.shape
    cols = B_nz.shape[1]
    out = []
    for i in range(rows):
        for j in range(cols):
            for k in range(inner):
                a, b = bool(A_nz[i, k]), bool(B_nz[k, j])
                if mode == NAIVE_SPARSE and not (a and b):
                    continue
                if mode == NAIVE_SPARSE_LITERAL and not (a or b):
                    continue
                out.append((i, j, k))
    return out


def naive_ct_ct(orc: Oracle, keys: Keys, A_cts: list, B_cts: list, A_nz: np.ndarray, B_nz: np.ndarray,
                mode: int, mask_pt: Pt | None = None, counts: OpCounts | None = None) -> list:
    """The element-wise baselines of Sec. 4 over densely packed encrypted
    operands (reading R16): for every product (i, j, k) that `mode` keeps,
    both ciphertexts are rotated so that A[i, k] and B[k, j] sit in slot 0
    (the naive alignment: one rotation per operand, none when the element is
    already there), multiplied and relinearised, rescaled, masked to slot 0,
    rescaled, rotated to the target slot t = i cols + j and added into the
    result chunk t // S; the chain after the alignment is Alg. 2's.
    A_nz, B_nz: the zero patterns (plaintext structure, like CSR metadata).
    Result chunks at level ell - 2, R3 layout."""
    P = orc.P
    S = P.slots
    if counts is None:
        counts = OpCounts()
    rows, inner = A_nz.shape
    cols = B_nz.shape[1]
    nres = max(1, -(-(rows * cols) // S))
    ell = A_cts[0].level
    result = [orc.zero_ct(ell - 2, result_scale(orc, ell, A_cts[0].scale, B_cts[0].scale)) for _ in range(nres)]
    mask = make_mask(orc, 0, ell - 1) if mask_pt is None else mask_pt
    for i, j, k in naive_triples(A_nz, B_nz, mode):
        counts.matches += 1
        ca, sa = divmod(i * inner + k, S)
        cb, sb = divmod(k * cols + j, S)
        vA, vB = A_cts[ca], B_cts[cb]
        if sa:
            vA = orc.rotate(vA, sa, keys)
            counts.ks_align += len(rotation_plan(sa, S, P.rot_base))
        if sb:
            vB = orc.rotate(vB, sb, keys)
            counts.ks_align += len(rotation_plan(sb, S, P.rot_base))
        dot = orc.mult_relin(vA, vB, keys)
        counts.ks_relin += 1
        dot = orc.rescale(dot)
        dot = orc.mul_plain(dot, mask)
        dot = orc.rescale(dot)
        counts.rescales += 2
        t = i * cols + j
        rc, ts = divmod(t, S)
        r = (-ts) % S
        counts.ks_final += len(rotation_plan(r, S, P.rot_base))
        dot = orc.rotate(dot, r, keys)
        result[rc] = orc.add(result[rc], dot)
    return result


def naive_rotation_amounts(rows: int, inner: int, cols: int, slots: int) -> list:
    """Every rotation amount the element-wise baselines may request."""
    amts = set()
    for p in range(rows * inner):
        amts.add(p % slots)
    for p in range(inner * cols):
        amts.add(p % slots)
    for t in range(rows * cols):
        amts.add((-(t % slots)) % slots)
    amts.discard(0)
    return sorted(amts)
