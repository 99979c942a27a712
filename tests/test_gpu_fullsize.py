"""GPU parity at full size (N = 2^16): the Argmax parameter set (q_0 60-bit +
23 x 50-bit primes, 4 special primes, dnum = 6) and the primitive
micro-benchmark set (24 x 50-bit, 4 special, dnum = 3).  Primitives are
compared bit for bit with the CPU oracle; the batched circuit over a mix of
queries is checked against the plaintext simulation, the exact argmax, and
the one-query path (bit-identical)."""
import numpy as np
import pytest

from oracle import ARGMAX, MICRO, Ct, Oracle, plainsim
from paper_2502_00847_gb300 import workloads

pytestmark = pytest.mark.gpu

ROT = [1, -2]


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    pkg_build.build()
    torch.cuda.set_device(0)
    o = Oracle(ARGMAX)
    o.keygen(2024, rot_steps=ROT)
    ctx = secpe.Context.from_params(ARGMAX)
    keys = secpe.Keys(ctx, 2024, ROT)
    return o, ctx, keys, secpe


def to_gpu(secpe, ctx, ct_o):
    return secpe.Ciphertext.from_residues(ct_o.c, ct_o.level, ct_o.scale, cap=ctx.L + 1)


def same(ct_g, ct_o):
    assert ct_g.level == ct_o.level and ct_g.scale == ct_o.scale
    assert np.array_equal(ct_g.residues(), ct_o.c)


def test_keys_bit_exact(env):
    o, ctx, keys, secpe = env
    assert ctx.primes() == o.primes
    assert np.array_equal(keys.export(0), o.s_ntt)
    assert np.array_equal(keys.export(1), o.rlk)
    assert np.array_equal(keys.export(2, -2), o.gks[o.galois(-2)])


def test_ntt_bit_exact(env):
    import torch
    o, ctx, keys, secpe = env
    rng = np.random.default_rng(16)
    pidx = [(5 * i) % 28 for i in range(37)]
    x = np.stack([rng.integers(0, o.primes[i], o.n, dtype=np.uint64) for i in pidx])
    t = torch.from_numpy(x.view(np.int64)).cuda()
    secpe.ntt(ctx, t, pidx)
    got = t.cpu().numpy().view(np.uint64)
    for r in (0, 1, 17, 36):
        exp = x[r].copy()
        o.ntt(exp, pidx[r])
        assert np.array_equal(got[r], exp)
    # property at every limb: INTT(NTT(x)) = x
    secpe.ntt(ctx, t, pidx, inverse=True)
    assert np.array_equal(t.cpu().numpy().view(np.uint64), x)


def test_encrypt_mul_rotate_rescale_refresh_bit_exact(env):
    o, ctx, keys, secpe = env
    rng = np.random.default_rng(17)
    m = o.encode_coeffs(rng.uniform(-1, 1, 16), o.p.scale)
    a_o = o.encrypt_coeffs(m, o.ctx.L, o.p.scale, seed=71)
    a = secpe.encrypt_coeffs(ctx, keys, np.array([int(v) for v in m], dtype=np.int64), ctx.L, o.p.scale, 71)
    same(a, a_o)
    b_o = o.encrypt(rng.uniform(-1, 1, 16), seed=72)
    b = to_gpu(secpe, ctx, b_o)
    same(secpe.mul_relin(ctx, keys, a, b), o.mul(a_o, b_o))
    low_o = o.drop(b_o, 6)
    same(secpe.mul_relin(ctx, keys, to_gpu(secpe, ctx, low_o), a), o.mul(low_o, a_o))
    same(secpe.rotate(ctx, keys, a, 1), o.rotate(a_o, 1))
    same(secpe.rotate(ctx, keys, to_gpu(secpe, ctx, low_o), -2), o.rotate(low_o, -2))
    same(secpe.rescale(ctx, a), o.rescale(a_o))
    o.ridx = 5
    same(secpe.refresh_testonly(ctx, keys, to_gpu(secpe, ctx, o.drop(a_o, 1)), 8, 5), o.refresh(o.drop(a_o, 1), 8))


def test_hoisted_rotations_bit_exact(env):
    """secpe_rotate_hoisted at N = 2^16 (the fused ModDown path): both
    rotations from one ModUp equal the oracle's rotate_hoisted residue for
    residue, at the top level and at level 6."""
    o, ctx, keys, secpe = env
    a_o = o.encrypt(np.random.default_rng(18).uniform(-1, 1, 16), seed=73)
    a = to_gpu(secpe, ctx, a_o)
    for g, w in zip(secpe.rotate_hoisted(ctx, keys, a, ROT), o.rotate_hoisted(a_o, ROT)):
        same(g, w)
    low_o = o.drop(a_o, 6)
    for g, w in zip(secpe.rotate_hoisted(ctx, keys, to_gpu(secpe, ctx, low_o), ROT), o.rotate_hoisted(low_o, ROT)):
        same(g, w)


def test_micro_keyswitch_dnum3_bit_exact():
    import torch
    from paper_2502_00847_gb300 import secpe
    o = Oracle(MICRO)
    o.keygen(3)
    ctx = secpe.Context.from_params(MICRO)
    keys = secpe.Keys(ctx, 3, [])
    lv = ctx.L
    d = workloads.residues((lv + 1, ctx.n), o.primes[: lv + 1], seed=2)
    k0, k1 = o.keyswitch(d, lv, o.rlk)
    dt = torch.from_numpy(d.view(np.int64)).cuda()
    g0, g1 = secpe.keyswitch(ctx, keys, 0, dt, lv)
    assert np.array_equal(g0.cpu().numpy().view(np.uint64), k0)
    assert np.array_equal(g1.cpu().numpy().view(np.uint64), k1)
    # precision variant (tensor-pipe transforms and 3-digit inner product) against the oracle
    x = torch.zeros((1, 2, lv + 1, ctx.n), dtype=torch.int64, device="cuda")
    x[0, 0] = dt
    out = secpe.CtBatch(torch.zeros_like(x), 0, ctx.scale)
    secpe.keyswitch_batch_tc(ctx, keys, 0, secpe.CtBatch(x, lv, ctx.scale), out)
    assert np.array_equal(out.data[0, 0].cpu().numpy().view(np.uint64), k0)
    assert np.array_equal(out.data[0, 1].cpu().numpy().view(np.uint64), k1)


def test_tensor_pipe_keyswitch_bit_identical(env):
    """Precision variant of key switching: every NTT/INTT and the key inner
    product on the tensor pipe give the residues of the CUDA-core key switch
    (relinearisation and Galois keys; 6 digits at the top level, fewer below;
    ragged batches of 9 and 3 items)."""
    import torch
    o, ctx, keys, secpe = env
    cap = ctx.L + 1
    for lv, B, step in [(ctx.L, 9, 0), (ctx.L, 1, 1), (11, 3, -2), (0, 2, 0)]:
        x = workloads.residues((B, 2, cap, ctx.n), o.primes[:cap], seed=40 + lv)
        xt = torch.from_numpy(x.view(np.int64)).cuda()
        d = secpe.CtBatch(xt, lv, ctx.scale)
        ref = secpe.CtBatch(torch.zeros_like(xt), 0, ctx.scale)
        out = secpe.CtBatch(torch.zeros_like(xt), 0, ctx.scale)
        secpe.keyswitch_batch(ctx, keys, step, d, ref)
        secpe.keyswitch_batch_tc(ctx, keys, step, d, out)
        torch.cuda.synchronize()
        assert out.level == ref.level == lv
        assert torch.equal(ref.data[:, :, : lv + 1], out.data[:, :, : lv + 1]), (lv, B, step)
        assert torch.equal(xt, torch.from_numpy(x.view(np.int64)).cuda())  # input untouched


def test_batched_argmax_mix(env):
    o, ctx, keys, secpe = env
    qs = workloads.argmax_queries(5, seed=4, K_choices=(4, 8), C_choices=(2, 3, 6, 14))
    # and two queries with the largest class count of the mix (6 QuickMax rounds)
    qs += workloads.argmax_queries(2, seed=9, K_choices=(4,), C_choices=(64,))
    rot = sorted({-(1 << (q.C - 1).bit_length()) for q in qs} | {1 << i for i in range(6)})
    k2 = secpe.Keys(ctx, 99, rot)
    inputs = [[secpe.encrypt_logits(ctx, k2, q.logits[i], q.d_min, q.enc_seeds[i]) for i in range(q.K)]
              for q in qs]
    batch = [dict(cts=cts, C=q.C, d_min=q.d_min, d_max=q.d_max, qseed=q.qseed, z_out=ctx.new_ct())
             for q, cts in zip(qs, inputs)]
    secpe.argmax_batch(ctx, k2, batch)
    for q, b, cts in zip(qs, batch, inputs):
        zd = secpe.decrypt(ctx, k2, b["z_out"], q.C)
        zp = plainsim.ensemble_argmax(q.logits, q.d_min, q.d_max, ctx.n // 2)
        assert np.max(np.abs(zd - zp)) < 2.0 ** -12
        assert int(np.argmax(zd)) == int(np.argmax(q.logits.mean(0)))
    # the one-query path gives identical residues for two of them
    for q, b, cts in list(zip(qs, batch, inputs))[:2]:
        y = secpe.ensemble_aggregate(ctx, cts, q.d_min, q.d_max)
        z = secpe.encrypted_argmax(ctx, k2, y, q.C, q.qseed)
        assert z.level == b["z_out"].level and np.array_equal(z.residues(), b["z_out"].residues())
    # the oracle decrypts the GPU output to the same values
    z = batch[0]["z_out"]
    o2 = Oracle(ARGMAX)
    o2.keygen(99)
    zo = o2.decrypt(Ct(z.residues(), z.level, z.scale), qs[0].C)
    assert np.max(np.abs(zo - secpe.decrypt(ctx, k2, z, qs[0].C))) < 2.0 ** -30


def test_tensor_pipe_ntt_bit_identical(env):
    """Precision variant: both passes (columns, twist, rows) as exact
    8-bit-limb contractions on the tensor pipe; forward and inverse
    bit-identical to the CUDA-core NTT and to the oracle's transform."""
    import torch
    o, ctx, keys, secpe = env
    rng = np.random.default_rng(33)
    pidx = [(3 * i) % 28 for i in range(29)]
    x = np.stack([rng.integers(0, o.primes[i], o.n, dtype=np.uint64) for i in pidx])
    # extremes: zeros and q - 1 everywhere in two limbs
    x[0] = 0
    x[1] = o.primes[pidx[1]] - 1
    a = torch.from_numpy(x.view(np.int64)).cuda()
    b = a.clone()
    secpe.ntt(ctx, a, pidx)
    secpe.ntt_tc(ctx, b, pidx)
    assert torch.equal(a, b)
    exp = x[5].copy()
    o.ntt(exp, pidx[5])
    assert np.array_equal(b[5].cpu().numpy().view(np.uint64), exp)
    secpe.ntt(ctx, a, pidx, inverse=True)
    secpe.ntt_tc(ctx, b, pidx, inverse=True)
    assert torch.equal(a, b)
    assert np.array_equal(b.cpu().numpy().view(np.uint64), x)
    # ciphertext layout entry point
    B, cap = 3, ctx.L + 1
    c = torch.from_numpy(workloads.residues((B, 2, cap, ctx.n), o.primes[:cap], seed=7).view(np.int64)).cuda()
    d = c.clone()
    secpe.ntt_cts(ctx, c, B, 2 * cap * ctx.n, cap, ctx.L)
    secpe.ntt_cts_tc(ctx, d, B, 2 * cap * ctx.n, cap, ctx.L)
    assert torch.equal(c, d)


def test_argmax8_parameter_set_bit_exact():
    """8 special primes, dnum = 3: HMult (full and partial last digits),
    rotation and a two-query batched Argmax, bit-exact / decoded against the
    oracle and the plaintext argmax."""
    from oracle import ARGMAX8
    from paper_2502_00847_gb300 import secpe
    o = Oracle(ARGMAX8)
    o.keygen(808, rot_steps=[1, -4])
    ctx = secpe.Context.from_params(ARGMAX8)
    keys = secpe.Keys(ctx, 808, [1, -4])
    assert ctx.primes() == o.primes
    rng = np.random.default_rng(88)
    a_o = o.encrypt(rng.uniform(-1, 1, 8), seed=5)
    b_o = o.drop(o.encrypt(rng.uniform(-1, 1, 8), seed=6), 17)
    a, b = to_gpu(secpe, ctx, a_o), to_gpu(secpe, ctx, b_o)
    same(secpe.mul_relin(ctx, keys, a, b), o.mul(a_o, b_o))
    same(secpe.rotate(ctx, keys, b, -4), o.rotate(b_o, -4))
    # partial last digits of 7 and 6 primes (levels 22, 21) and of 1 (level 8)
    for lv in (22, 21, 8):
        c_o = o.drop(a_o, lv)
        c = to_gpu(secpe, ctx, c_o)
        same(secpe.mul_relin(ctx, keys, c, c), o.mul(c_o, c_o))
    qs = workloads.argmax_queries(2, seed=8, K_choices=(4,), C_choices=(2, 4))
    rot = sorted({-(1 << (q.C - 1).bit_length()) for q in qs} | {1, 2})
    k2 = secpe.Keys(ctx, 5, rot)
    batch = []
    for q in qs:
        cts = [secpe.encrypt_logits(ctx, k2, q.logits[i], q.d_min, q.enc_seeds[i]) for i in range(q.K)]
        batch.append(dict(cts=cts, C=q.C, d_min=q.d_min, d_max=q.d_max, qseed=q.qseed, z_out=ctx.new_ct()))
    secpe.argmax_batch(ctx, k2, batch)
    for q, b in zip(qs, batch):
        zd = secpe.decrypt(ctx, k2, b["z_out"], q.C)
        zp = plainsim.ensemble_argmax(q.logits, q.d_min, q.d_max, ctx.n // 2)
        assert np.max(np.abs(zd - zp)) < 2.0 ** -12
        assert int(np.argmax(zd)) == int(np.argmax(q.logits.mean(0)))


def test_graph_captured_batch_replays_bit_exact(env):
    """The batched Argmax captured as one CUDA graph: a replay gives the same
    residues as the direct call, a replay after the inputs are rewritten in
    place gives the new inputs' results, and the counters count the replays."""
    import torch
    o, ctx, keys, secpe = env
    qs = workloads.argmax_queries(3, seed=12, K_choices=(4,), C_choices=(2, 3))
    rot = sorted({-(1 << (q.C - 1).bit_length()) for q in qs} | {1, 2})
    k2 = secpe.Keys(ctx, 21, rot)
    qs2 = [workloads.argmax_queries(1, seed=100 + i, K_choices=(4,), C_choices=(q.C,))[0] for i, q in enumerate(qs)]
    cts = [[secpe.encrypt_logits(ctx, k2, q.logits[i], q.d_min, q.enc_seeds[i]) for i in range(q.K)] for q in qs]
    batch = [dict(cts=c, C=q.C, d_min=q.d_min, d_max=q.d_max, qseed=q.qseed, z_out=ctx.new_ct())
             for q, c in zip(qs, cts)]
    ref = [dict(b, z_out=ctx.new_ct()) for b in batch]
    secpe.argmax_batch(ctx, k2, ref)
    g = secpe.Graph(ctx, k2, batch)
    assert g.nodes > 100
    ctx.reset_counters()
    g.launch()
    torch.cuda.synchronize()
    cnt = ctx.counters()
    assert cnt["launches"] > 100 and cnt["relins"] > 0
    for b, r in zip(batch, ref):
        assert b["z_out"].level == r["z_out"].level
        assert np.array_equal(b["z_out"].residues(), r["z_out"].residues())
    # new inputs written into the captured buffers (same classes per query)
    for q, q2, c in zip(qs, qs2, cts):
        for i in range(q.K):
            secpe.encrypt_logits(ctx, k2, q2.logits[i], q2.d_min, q2.enc_seeds[i], out=c[i])
    g.launch()
    torch.cuda.synchronize()
    for q, q2, b in zip(qs, qs2, batch):
        zd = secpe.decrypt(ctx, k2, b["z_out"], q.C)
        assert int(np.argmax(zd)) == int(np.argmax(q2.logits.mean(0)))
    g.close()


def test_autotune_and_every_launch_configuration_bit_exact(env):
    """secpe_autotune times both candidates of each tuned kernel and keeps
    one; NTT/INTT and HMult give identical residues under 3 and 4 CTAs/SM."""
    import torch
    o, ctx, keys, secpe = env
    rng = np.random.default_rng(44)
    pidx = [(5 * i) % 28 for i in range(20)]
    x = np.stack([rng.integers(0, o.primes[i], o.n, dtype=np.uint64) for i in pidx])
    a_o = o.encrypt(rng.uniform(-1, 1, 8), seed=71)
    outs = []
    for v in (3, 4):
        for k in range(5):
            ctx.tuning_set(k, v)
        t = torch.from_numpy(x.view(np.int64)).cuda()
        secpe.ntt(ctx, t, pidx)
        f = t.clone()
        secpe.ntt(ctx, t, pidx, inverse=True)
        a = to_gpu(secpe, ctx, a_o)
        outs.append((f.cpu(), t.cpu(), secpe.mul_relin(ctx, keys, a, a).residues()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][1].numpy().view(np.uint64), x)
    assert np.array_equal(outs[0][2], outs[1][2])
    res = ctx.autotune()
    assert set(res) == {"ntt16_colpass", "ntt16_rowpass", "intt16_colpass", "intt16_rowpass", "colpass_bconv"}
    for r in res.values():
        assert r["ctas_per_sm"] in (3, 4) and r["ms_3"] > 0 and r["ms_4"] > 0
        assert r["ctas_per_sm"] == (4 if r["ms_4"] < 0.97 * r["ms_3"] else 3)
    same(secpe.mul_relin(ctx, keys, to_gpu(secpe, ctx, a_o), to_gpu(secpe, ctx, a_o)), o.mul(a_o, a_o))
