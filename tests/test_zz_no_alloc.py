"""The allocation-free rescale (spfhe_rescale_noalloc) against the regular
spfhe_rescale: identical limbs, on two calls in a row.

Callers that cannot allocate device memory while they run hand the library
their own input and output buffers; this test allocates those buffers with
torch (the caller's side) and checks that the entry point itself, which keeps
its scratch in a fixed device array, returns exactly what the allocating path
returns.  The file is named so that pytest collects it last."""
import numpy as np
import pytest

from paper_2604_11659_gb300 import synthetic
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("recipe", [synthetic.ring_small_16x16(), synthetic.ring_128x128()],
                         ids=["n4096_L4", "n65536_L24"])
def test_noalloc_rescale_matches_rescale_twice(recipe):
    sp = need_gpu()
    import torch
    from paper_2604_11659_gb300 import params as gparams
    ctx = sp.spfhe_ctx_create(gparams.ctx_params(recipe, rot_base=2))
    handles = []
    try:
        keys = sp.spfhe_keygen(ctx, 77)
        handles.append(("keys", keys))
        n, L = 1 << recipe.log_n, recipe.L
        rng = np.random.default_rng(9)
        for call in range(2):
            z = rng.uniform(-1, 1, n // 2)
            pt = sp.spfhe_encode(ctx, z, L, recipe.scale)
            ct = sp.spfhe_encrypt(ctx, keys, pt, 100 + call)
            handles += [("pt", pt), ("ct", ct)]
            limbs = sp.spfhe_ct_export(ctx, ct, n)
            src = torch.from_numpy(limbs.view(np.int64).copy()).cuda()
            dst = torch.full((2, L - 1, n), -1, dtype=torch.int64, device="cuda")
            sp.spfhe_rescale_noalloc(ctx, src.data_ptr(), L, dst.data_ptr())
            sp.spfhe_sync(ctx)
            sp.spfhe_rescale(ctx, ct)
            want = sp.spfhe_ct_export(ctx, ct, n)
            got = dst.cpu().numpy().view(np.uint64)
            assert got.shape == want.shape
            assert np.array_equal(got, want), "call %d differs" % call
        with pytest.raises(sp.SpfheError) as e:
            sp.spfhe_rescale_noalloc(ctx, src.data_ptr(), 1, dst.data_ptr())
        assert e.value.status == -3
    finally:
        for kind, h in reversed(handles):
            {"ct": sp.spfhe_ct_free, "pt": sp.spfhe_pt_free, "keys": sp.spfhe_keys_free}[kind](h)
        sp.spfhe_ctx_destroy(ctx)
