"""CKKS bootstrapping on the GPU (secpe_boot_*, secpe_bootstrap*).

* N = 2^12 (bootstrapping toy set, block n = 16): with the oracle's plaintext
  diagonals, every residue of the bootstrapped ciphertext equals the
  oracle's; the sparse secret and the conjugation key are the oracle's; the
  rotation steps agree.
* N = 2^12 with the library's own plan: the result decrypts to the input's
  block sums within 2^-15 at level L - 16, for a batch of ciphertexts.
* N = 2^16 (boot16, block n = 128): a batch of 4 ciphertexts bootstraps to
  their block sums within 2^-12, non-interactively (no secret key used)."""
import numpy as np
import pytest

from oracle import BOOT16, BOOT_TOY, Oracle
from oracle.boot import BootPlan

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def toy():
    import torch
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    pkg_build.build()
    torch.cuda.set_device(0)
    o = Oracle(BOOT_TOY)
    plan = BootPlan(o, 16)
    steps = plan.rotation_steps()
    o.keygen(99, rot_steps=steps)
    ctx = secpe.Context.from_params(BOOT_TOY)
    keys = secpe.Keys(ctx, 99, steps)
    return o, plan, ctx, keys, secpe


def test_toy_bootstrap_bit_exact(toy):
    o, plan, ctx, keys, secpe = toy
    assert secpe.boot_rotation_steps(ctx, 16) == plan.rotation_steps()
    assert np.array_equal(keys.export(0), o.s_ntt)                  # sparse secret
    assert np.array_equal(keys.export(2, secpe.STEP_CONJ), o.gks[2 * o.n - 1])
    rng = np.random.default_rng(12)
    v = rng.uniform(-1, 1, 16)
    ct_o = o.drop(o.encrypt(v, seed=13, level=7), 0)
    z_o = plan.bootstrap(ct_o)
    bs1, gs1 = plan.c2s_bs, plan.c2s_gs
    bs2, gs2 = plan.s2c_bs, plan.s2c_gs
    c2s = [[int(c) for c in plan._pt[("c2s", t, k // bs1, k % bs1)]] for t in range(2) for k in range(16)]
    s2c = [[int(c) for c in plan._pt[("s2c", 0, k // bs2, k % bs2)]] for k in range(32)]
    assert gs1 * bs1 == 16 and gs2 * bs2 == 32
    bt = secpe.Boot(ctx, 16, coeffs=(np.array(c2s, dtype=np.int64), np.array(s2c, dtype=np.int64)))
    ct = secpe.Ciphertext.from_residues(ct_o.c, ct_o.level, ct_o.scale, cap=ctx.L + 1)
    z = bt.bootstrap(keys, ct)
    assert z.level == z_o.level == ctx.L - 16 and z.scale == z_o.scale == ct_o.scale
    assert np.array_equal(z.residues(), z_o.c)
    bt.close()


def test_toy_library_plan_batch(toy):
    import torch
    o, plan, ctx, keys, secpe = toy
    bt = secpe.Boot(ctx, 16)
    rng = np.random.default_rng(14)
    B = 5
    vs = [rng.uniform(-1, 1, 16) for _ in range(B)]
    data = torch.zeros((B, 2, ctx.L + 1, ctx.n), dtype=torch.int64, device="cuda")
    for b in range(B):
        secpe.encrypt(ctx, keys, vs[b], 200 + b, out=secpe.Ciphertext(data[b], 0, ctx.scale))
    x = secpe.CtBatch(data, 1, ctx.scale)           # bootstrapped from limb 0 (level 1 dropped to 0)
    out = secpe.CtBatch(torch.zeros_like(data), 0, 0.0)
    bt.bootstrap_batch(keys, x, out)
    assert out.level == ctx.L - 16 and out.scale == ctx.scale
    for b in range(B):
        z = secpe.decrypt(ctx, keys, secpe.Ciphertext(out.data[b], out.level, out.scale), 64)
        for k in range(4):
            assert np.max(np.abs(z[16 * k:16 * (k + 1)] - vs[b])) < 2.0 ** -15
    bt.close()


def test_full_size_bootstrap_batch():
    import torch
    from paper_2502_00847_gb300 import secpe
    torch.cuda.set_device(0)
    ctx = secpe.Context.from_params(BOOT16)
    n = 128
    keys = secpe.Keys(ctx, 7, secpe.boot_rotation_steps(ctx, n))
    bt = secpe.Boot(ctx, n)
    rng = np.random.default_rng(15)
    B = 4
    vs = [rng.uniform(-1, 1, n) for _ in range(B)]
    data = torch.zeros((B, 2, ctx.L + 1, ctx.n), dtype=torch.int64, device="cuda")
    for b in range(B):
        secpe.encrypt(ctx, keys, vs[b], 300 + b, out=secpe.Ciphertext(data[b], 0, ctx.scale))
    out = secpe.CtBatch(torch.zeros_like(data), 0, 0.0)
    bt.bootstrap_batch(keys, secpe.CtBatch(data, 0, ctx.scale), out)
    assert out.level == ctx.L - 16
    for b in range(B):
        z = secpe.decrypt(ctx, keys, secpe.Ciphertext(out.data[b], out.level, out.scale), 2 * n)
        assert np.max(np.abs(z[:n] - vs[b])) < 2.0 ** -12 and np.max(np.abs(z[n:] - vs[b])) < 2.0 ** -12
    bt.close()
