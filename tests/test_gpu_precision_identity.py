"""Precision variant at scale: the NTT/INTT computed as exact 8-bit-limb
contractions on the tensor pipe, and the key switch whose transforms and key
inner product run there, are bit-identical to the CUDA-core path over 1,000
seeded random ciphertexts of the primitive micro-benchmark set (N = 2^16,
24 x 50-bit + 4 x 60-bit special primes, dnum = 3): forward and inverse
transforms of both polynomials, and the relinearisation key switch of
polynomial 0 at the top level.  Seeds 30000 + chunk (transforms) and
40000 + chunk (key switches), as in the benchmark's identity run."""
import pytest

from oracle import MICRO

pytestmark = pytest.mark.gpu

COUNT, CHUNK = 1000, 50


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    pkg_build.build()
    torch.cuda.set_device(0)
    ctx = secpe.Context.from_params(MICRO)
    keys = secpe.Keys(ctx, 2, [])
    return torch, secpe, ctx, keys


def _random_cts(torch, primes, cap, n, count, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    t = torch.empty((count, 2, cap, n), dtype=torch.int64)
    for i in range(cap):
        t[:, :, i] = torch.randint(0, primes[i], (count, 2, n), generator=g, dtype=torch.int64)
    return t.cuda()


def test_tensor_pipe_ntt_identity_1000_ciphertexts(env):
    torch, secpe, ctx, keys = env
    n, cap, L = ctx.n, ctx.L + 1, ctx.L
    primes = ctx.primes()
    mism = 0
    for s0 in range(0, COUNT, CHUNK):
        u = _random_cts(torch, primes, cap, n, CHUNK, 30000 + s0)
        v = u.clone()
        secpe.ntt_cts(ctx, u, CHUNK, 2 * cap * n, cap, L)
        secpe.ntt_cts_tc(ctx, v, CHUNK, 2 * cap * n, cap, L)
        mism += int((u != v).any(dim=(1, 2, 3)).sum().item())
        secpe.ntt_cts(ctx, u, CHUNK, 2 * cap * n, cap, L, inverse=True)
        secpe.ntt_cts_tc(ctx, v, CHUNK, 2 * cap * n, cap, L, inverse=True)
        mism += int((u != v).any(dim=(1, 2, 3)).sum().item())
    assert mism == 0


def test_tensor_pipe_keyswitch_identity_1000_ciphertexts(env):
    torch, secpe, ctx, keys = env
    n, cap, L = ctx.n, ctx.L + 1, ctx.L
    primes = ctx.primes()
    mism = 0
    for s0 in range(0, COUNT, CHUNK):
        d = secpe.CtBatch(_random_cts(torch, primes, cap, n, CHUNK, 40000 + s0), L, ctx.scale)
        u = secpe.CtBatch(torch.zeros_like(d.data), 0, ctx.scale)
        v = secpe.CtBatch(torch.zeros_like(d.data), 0, ctx.scale)
        secpe.keyswitch_batch(ctx, keys, 0, d, u)
        secpe.keyswitch_batch_tc(ctx, keys, 0, d, v)
        assert u.level == v.level == L
        mism += int((u.data != v.data).any(dim=(1, 2, 3)).sum().item())
    assert mism == 0
