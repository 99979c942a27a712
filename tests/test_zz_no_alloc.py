"""The allocation-free rescale (secpe_rescale_noalloc) is for callers that may
not allocate device memory during a call: a serving loop that keeps a fixed
device-memory footprint and keeps the allocator off its critical path, or a
host framework that owns all device memory and forbids hidden allocations.

It must give the same ciphertext as the ordinary rescale on two calls in a
row, allocate nothing (the stream-ordered pool's used and reserved bytes and
the device's free memory are unchanged across a call, while the ordinary
rescale does grow the pool), work in place, reject a partly overlapping
output and a level-0 input like secpe_rescale does.  This file is collected
last so a run that stops at the first failure has already run every other
test; it also passes when run alone in a fresh process."""
import numpy as np
import pytest

from oracle import ARGMAX, TOY

pytestmark = pytest.mark.gpu


def _setup(params):
    import torch
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    pkg_build.build()
    torch.cuda.set_device(0)
    ctx = secpe.Context.from_params(params)
    keys = secpe.Keys(ctx, 5, [])
    return torch, secpe, ctx, keys


@pytest.mark.parametrize("params", [TOY, ARGMAX], ids=["N4096", "N65536"])
def test_rescale_noalloc_matches_rescale(params):
    torch, secpe, ctx, keys = _setup(params)
    rng = np.random.default_rng(6)
    # the first call on a device does the one-time set-up (module load, scratch address)
    warm = secpe.encrypt(ctx, keys, rng.uniform(-1, 1, 16), seed=99)
    secpe.rescale_noalloc(ctx, warm, ctx.new_ct())
    for call in range(2):
        ct = secpe.encrypt(ctx, keys, rng.uniform(-1, 1, 16), seed=100 + call)
        ref = secpe.rescale(ctx, ct)
        out = ctx.new_ct()
        torch.cuda.synchronize()
        used0, res0 = secpe.pool_usage(trim=True)
        free0 = torch.cuda.mem_get_info()[0]
        secpe.rescale_noalloc(ctx, ct, out)
        torch.cuda.synchronize()
        used1, res1 = secpe.pool_usage()
        free1 = torch.cuda.mem_get_info()[0]
        assert (used1, res1, free1) == (used0, res0, free0), "secpe_rescale_noalloc allocated device memory"
        assert out.level == ref.level == ct.level - 1
        assert out.scale == ref.scale
        assert np.array_equal(out.residues(), ref.residues())
    # the same probe sees the ordinary rescale take scratch from the pool
    secpe.rescale(ctx, ct)
    torch.cuda.synchronize()
    assert secpe.pool_usage()[1] > res0
    # a lower level works too
    low = secpe.Ciphertext(ct.data, 3, ct.scale)
    out = ctx.new_ct()
    secpe.rescale_noalloc(ctx, low, out)
    assert np.array_equal(out.residues(), secpe.rescale(ctx, low).residues())


@pytest.mark.parametrize("params", [TOY, ARGMAX], ids=["N4096", "N65536"])
def test_rescale_noalloc_in_place_and_overlap(params):
    torch, secpe, ctx, keys = _setup(params)
    rng = np.random.default_rng(7)
    ct = secpe.encrypt(ctx, keys, rng.uniform(-1, 1, 16), seed=200)
    ref = secpe.rescale(ctx, ct)
    # in place: out is in itself (same data and cap)
    inplace = secpe.Ciphertext(ct.data, ct.level, ct.scale)
    secpe.rescale_noalloc(ctx, inplace, inplace)
    torch.cuda.synchronize()
    assert inplace.level == ref.level and inplace.scale == ref.scale
    assert np.array_equal(inplace.residues(), ref.residues())
    # an output that overlaps the input with another layout is rejected before any launch
    ct2 = secpe.encrypt(ctx, keys, rng.uniform(-1, 1, 16), seed=201)
    flat = ct2.data.view(-1)
    cap2 = ct2.cap - 1
    shifted = secpe.Ciphertext(flat[: 2 * cap2 * ctx.n].view(2, cap2, ctx.n), 0, ct2.scale)
    before = ctx.counters()["launches"]
    with pytest.raises(secpe.SecpeError) as e:
        secpe.rescale_noalloc(ctx, ct2, shifted)
    assert e.value.code == -1
    # level 0 has nothing to divide by: the ordinary rescale's SECPE_ELEVEL
    lv0 = secpe.Ciphertext(ct2.data, 0, ct2.scale)
    with pytest.raises(secpe.SecpeError) as e:
        secpe.rescale(ctx, lv0)
    assert e.value.code == -3
    with pytest.raises(secpe.SecpeError) as e:
        secpe.rescale_noalloc(ctx, lv0, ctx.new_ct())
    assert e.value.code == -3
    assert ctx.counters()["launches"] == before


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
