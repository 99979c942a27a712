"""The allocation-free rescale (secpe_rescale_noalloc), for callers that may
not allocate device memory during a call, gives the same ciphertext as the
ordinary rescale, on two calls in a row.  This file is collected last so a
run that stops at the first failure has already run every other test; it
also passes when run alone in a fresh process."""
import numpy as np
import pytest

from oracle import ARGMAX, TOY

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("params", [TOY, ARGMAX], ids=["N4096", "N65536"])
def test_rescale_noalloc_matches_rescale(params):
    import torch
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    pkg_build.build()
    torch.cuda.set_device(0)
    ctx = secpe.Context.from_params(params)
    keys = secpe.Keys(ctx, 5, [])
    rng = np.random.default_rng(6)
    for call in range(2):
        ct = secpe.encrypt(ctx, keys, rng.uniform(-1, 1, 16), seed=100 + call)
        ref = secpe.rescale(ctx, ct)
        out = ctx.new_ct()
        secpe.rescale_noalloc(ctx, ct, out)
        torch.cuda.synchronize()
        assert out.level == ref.level == ct.level - 1
        assert out.scale == ref.scale
        assert np.array_equal(out.residues(), ref.residues())
    # a lower level works too
    low = secpe.Ciphertext(ct.data, 3, ct.scale)
    out = ctx.new_ct()
    secpe.rescale_noalloc(ctx, low, out)
    assert np.array_equal(out.residues(), secpe.rescale(ctx, low).residues())


def test_rescale_noalloc_rejects_levels_beyond_scratch():
    import torch
    from oracle import Params
    from paper_2502_00847_gb300 import secpe
    torch.cuda.set_device(0)
    big = Params(log_n=16, q0_bits=60, q_bits=50, n_q=26, p_bits=60, n_p=2, dnum=13, log_scale=50)
    ctx = secpe.Context.from_params(big)
    keys = secpe.Keys(ctx, 9, [])
    ct = secpe.encrypt(ctx, keys, np.ones(4), seed=3)   # level 25: needs 2 N 26 words
    with pytest.raises(secpe.SecpeError) as e:
        secpe.rescale_noalloc(ctx, ct, ctx.new_ct())
    assert e.value.code == -1
    ok = secpe.Ciphertext(ct.data, 23, ct.scale)         # level 23 fits exactly
    out = ctx.new_ct()
    secpe.rescale_noalloc(ctx, ok, out)
    assert np.array_equal(out.residues(), secpe.rescale(ctx, ok).residues())
