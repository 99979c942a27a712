"""CKKS bootstrapping on the GPU (secpe_boot_*, secpe_bootstrap*).

* N = 2^12 (bootstrapping toy set, block n = 16): with the oracle's plaintext
  diagonals, every residue of the bootstrapped ciphertext equals the
  oracle's; the sparse secret and the conjugation key are the oracle's; the
  rotation steps agree.
* N = 2^12 with the library's own plan: n-periodic inputs come back
  unchanged within 2^-20 at level L - 16, for a batch of ciphertexts.
* N = 2^16 (boot16, block n = 128): a batch of 4 n-periodic ciphertexts
  bootstraps to itself within 2^-16, non-interactively (no secret key used).
* The non-interactive Argmax (secpe_argmax_batch_boot: every refresh a
  bootstrap) of a C = 3 query at N = 2^12 equals the oracle's, residue for
  residue, with the exact index."""
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
    steps = sorted(set(plan.rotation_steps()) | {1, 2, -4})
    o.keygen(99, rot_steps=steps)
    ctx = secpe.Context.from_params(BOOT_TOY)
    keys = secpe.Keys(ctx, 99, steps)
    return o, plan, ctx, keys, secpe


def _plan_coeffs(plan):
    bs1, bs2 = plan.c2s_bs, plan.s2c_bs
    c2s = [[int(c) for c in plan._pt[("c2s", t, k // bs1, k % bs1)]] for t in range(2) for k in range(plan.n)]
    s2c = [[int(c) for c in plan._pt[("s2c", 0, k // bs2, k % bs2)]] for k in range(2 * plan.n)]
    return np.array(c2s, dtype=np.int64), np.array(s2c, dtype=np.int64)


def test_toy_bootstrap_bit_exact(toy):
    o, plan, ctx, keys, secpe = toy
    assert secpe.boot_rotation_steps(ctx, 16) == plan.rotation_steps()
    assert np.array_equal(keys.export(0), o.s_ntt)                  # sparse secret
    assert np.array_equal(keys.export(2, secpe.STEP_CONJ), o.gks[2 * o.n - 1])
    rng = np.random.default_rng(12)
    v = np.tile(rng.uniform(-1, 1, 16), (o.n // 2) // 16)
    ct_o = o.drop(o.encrypt(v, seed=13, level=7), 0)
    z_o = plan.bootstrap(ct_o)
    assert plan.c2s_bs * plan.c2s_gs == 16 and plan.s2c_bs * plan.s2c_gs == 32
    bt = secpe.Boot(ctx, 16, coeffs=_plan_coeffs(plan))
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
    vs = [np.tile(rng.uniform(-1, 1, 16), ctx.n // 32) for _ in range(B)]
    data = torch.zeros((B, 2, ctx.L + 1, ctx.n), dtype=torch.int64, device="cuda")
    for b in range(B):
        secpe.encrypt(ctx, keys, vs[b], 200 + b, out=secpe.Ciphertext(data[b], 0, ctx.scale))
    x = secpe.CtBatch(data, 1, ctx.scale)           # bootstrapped from limb 0 (level 1 dropped to 0)
    out = secpe.CtBatch(torch.zeros_like(data), 0, 0.0)
    bt.bootstrap_batch(keys, x, out)
    assert out.level == ctx.L - 16 and out.scale == ctx.scale
    for b in range(B):
        z = secpe.decrypt(ctx, keys, secpe.Ciphertext(out.data[b], out.level, out.scale), ctx.n // 2)
        assert np.max(np.abs(z - vs[b])) < 2.0 ** -20
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
    vs = [rng.uniform(-1, 1, n // 2) for _ in range(B)]
    data = torch.zeros((B, 2, ctx.L + 1, ctx.n), dtype=torch.int64, device="cuda")
    for b in range(B):
        # n-periodic: n/2 values and n/2 zeros packed into every block of n slots
        secpe.encrypt_logits_packed(ctx, keys, np.tile(vs[b], (ctx.n // (2 * n), 1)), 0.0, 300 + b,
                                    out=secpe.Ciphertext(data[b], 0, ctx.scale))
    out = secpe.CtBatch(torch.zeros_like(data), 0, 0.0)
    bt.bootstrap_batch(keys, secpe.CtBatch(data, 0, ctx.scale), out)
    assert out.level == ctx.L - 16
    for b in range(B):
        z = secpe.decrypt(ctx, keys, secpe.Ciphertext(out.data[b], out.level, out.scale), 4 * n)
        block = np.concatenate([vs[b], np.zeros(n // 2)])
        assert np.max(np.abs(z - np.tile(block, 4))) < 2.0 ** -16
    bt.close()


def test_toy_noninteractive_argmax_bit_exact(toy):
    """Alg. 1 with every refresh a bootstrap (the oracle's plan and
    plaintexts on both sides): z residues, level, scale and the op counts
    equal the oracle's one-query evaluation."""
    from oracle import plainsim
    from paper_2502_00847_gb300 import workloads
    o, plan, ctx, keys, secpe = toy
    q = workloads.toy_query(seed=3, K=3, C=3)
    lv = ctx.L - 16
    P = o.packed_capacity(q.C)      # the query packed into every block: 2C'-periodic inputs
    cts_o = [o.encrypt(o.pack_slots(np.tile(q.logits[i], (P, 1)), q.d_min), seed=q.enc_seeds[i], level=lv)
             for i in range(q.K)]
    o.boot_plan = plan
    try:
        y_o = o.aggregate(cts_o, q.d_min, q.d_max)
        o.reset_counters()
        z_o = o.argmax(y_o, q.C, qseed=q.qseed)
    finally:
        o.boot_plan = None
    assert o.counters["bootstraps"] >= 4
    bt = secpe.Boot(ctx, 16, coeffs=_plan_coeffs(plan))
    cts = [secpe.Ciphertext.from_residues(c.c, c.level, c.scale, cap=ctx.L + 1) for c in cts_o]
    b = [dict(cts=cts, C=q.C, d_min=q.d_min, d_max=q.d_max, qseed=q.qseed, z_out=ctx.new_ct())]
    ctx.reset_counters()
    secpe.argmax_batch_boot(ctx, keys, bt, b)
    z = b[0]["z_out"]
    cnt = ctx.counters()
    assert cnt["bootstraps"] == o.counters["bootstraps"] and cnt["signs"] == o.counters["signs"]
    assert z.level == z_o.level and z.scale == z_o.scale
    assert np.array_equal(z.residues(), z_o.c)
    zd = secpe.decrypt(ctx, keys, z, q.C)
    assert int(np.argmax(zd)) == int(np.argmax(q.logits.mean(0)))
    bt.close()


def test_toy_noninteractive_packed_distinct_inputs(toy):
    """Non-interactive Argmax on slot-packed inputs: n / (2C') different
    inputs in every n-block (the block repeated over the slots, so every
    bootstrap's n-periodic average keeps it); every input's index exact."""
    from paper_2502_00847_gb300 import workloads
    o, plan, ctx, keys, secpe = toy
    n, S = 16, ctx.n // 2
    (st,) = workloads.packed_queries(1, n, seed=9, K_choices=(2,), C_choices=(3,))
    assert st.P == 2
    lv = ctx.L - 16
    cts = []
    for i in range(st.K):
        c = secpe.encrypt_logits_packed(ctx, keys, np.tile(st.prompt(i), (S // n, 1)), st.d_min, st.enc_seeds[i])
        cts.append(secpe.Ciphertext(c.data, lv, c.scale))
    bt = secpe.Boot(ctx, n)
    b = [dict(cts=cts, C=st.C, d_min=st.d_min, d_max=st.d_max, qseed=st.qseed, z_out=ctx.new_ct())]
    secpe.argmax_batch_boot(ctx, keys, bt, b)
    z = secpe.decrypt_packed(ctx, keys, b[0]["z_out"], S // 8, st.C)
    for j in range(S // 8):
        assert int(np.argmax(z[j])) == int(np.argmax(st.logits[j % st.P].mean(0))), j
    bt.close()

