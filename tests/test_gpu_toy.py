"""GPU parity at the toy size (N = 2^12, 12 x 40-bit primes + one special):
every primitive and the whole encrypted ensemble Argmax, through the C ABI,
bit-exact against the CPU oracle on the same inputs; decoded values against
the FP64 plaintext simulation; returned index against the exact argmax."""
import numpy as np
import pytest

from oracle import Oracle, Params, TOY, plainsim
from paper_2502_00847_gb300 import workloads

pytestmark = pytest.mark.gpu

ROT = [1, 2, 4, -2, -4, -8, 3, 8, 16, 32, -64]
TOL_Z = 2.0 ** -12


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    pkg_build.build()
    torch.cuda.set_device(0)
    o = Oracle(TOY)
    o.keygen(77, rot_steps=ROT)
    ctx = secpe.Context.from_params(TOY)
    keys = secpe.Keys(ctx, 77, ROT)
    return o, ctx, keys, secpe


def to_gpu(secpe, ctx, ct_o):
    return secpe.Ciphertext.from_residues(ct_o.c, ct_o.level, ct_o.scale, cap=ctx.L + 1)


def same(ct_g, ct_o):
    assert ct_g.level == ct_o.level
    assert ct_g.scale == ct_o.scale
    assert np.array_equal(ct_g.residues(), ct_o.c)


def test_primes_and_keys_bit_exact(env):
    o, ctx, keys, secpe = env
    assert ctx.primes() == o.primes
    assert np.array_equal(keys.export(0), o.s_ntt)
    assert np.array_equal(keys.export(1), o.rlk)
    for r in (1, -2, 3):
        assert np.array_equal(keys.export(2, r), o.gks[o.galois(r)])


@pytest.mark.parametrize("logn", [12, 10, 8])
def test_ntt_bit_exact_random_limbs(logn):
    import torch
    from paper_2502_00847_gb300 import secpe
    p = Params(log_n=logn, q0_bits=60, q_bits=50, n_q=5, p_bits=60, n_p=2, dnum=2, log_scale=50)
    o = Oracle(p)
    ctx = secpe.Context.from_params(p)
    rng = np.random.default_rng(logn)
    # a ragged count of limbs over every prime, twice over
    pidx = [i % 7 for i in range(13)]
    x = np.stack([rng.integers(0, o.primes[i], o.n, dtype=np.uint64) for i in pidx])
    t = torch.from_numpy(x.view(np.int64)).cuda()
    secpe.ntt(ctx, t, pidx)
    got = t.cpu().numpy().view(np.uint64)
    exp = x.copy()
    for r, i in enumerate(pidx):
        o.ntt(exp[r], i)
    assert np.array_equal(got, exp)
    secpe.ntt(ctx, t, pidx, inverse=True)
    assert np.array_equal(t.cpu().numpy().view(np.uint64), x)


def test_encrypt_coeffs_bit_exact(env):
    o, ctx, keys, secpe = env
    m = o.encode_coeffs(np.linspace(-1, 1, 9), o.p.scale)
    ct_o = o.encrypt_coeffs(m, o.ctx.L, o.p.scale, seed=555)
    ct_g = secpe.encrypt_coeffs(ctx, keys, np.array([int(v) for v in m], dtype=np.int64), ctx.L,
                                o.p.scale, 555)
    same(ct_g, ct_o)
    # a lower level too
    ct_o = o.encrypt_coeffs(m, 3, o.p.scale, seed=556)
    ct_g = secpe.encrypt_coeffs(ctx, keys, np.array([int(v) for v in m], dtype=np.int64), 3, o.p.scale, 556)
    same(ct_g, ct_o)


def test_encrypt_decrypt_library_encoding(env):
    o, ctx, keys, secpe = env
    v = np.random.default_rng(3).uniform(-1, 1, 20)
    ct = secpe.encrypt(ctx, keys, v, 91)
    assert np.max(np.abs(secpe.decrypt(ctx, keys, ct, 20) - v)) < 2.0 ** -20
    # the oracle decrypts the library's ciphertext to the same values
    from oracle import Ct
    assert np.max(np.abs(o.decrypt(Ct(ct.residues(), ct.level, ct.scale), 20) - v)) < 2.0 ** -20


def test_linear_ops_bit_exact(env):
    o, ctx, keys, secpe = env
    rng = np.random.default_rng(4)
    a_o = o.encrypt(rng.uniform(-1, 1, 8), seed=21)
    b_o = o.drop(o.encrypt(rng.uniform(-1, 1, 8), seed=22), 9)
    a, b = to_gpu(secpe, ctx, a_o), to_gpu(secpe, ctx, b_o)
    same(secpe.add(ctx, a, b), o.add(a_o, b_o))
    same(secpe.sub(ctx, a, b), o.sub(a_o, b_o))
    same(secpe.add_const(ctx, a, -0.3125), o.add_const(a_o, -0.3125))
    same(secpe.mul_const(ctx, a, 1.7, 2.0 ** 39, 7), o.mul_const(a_o, 1.7, 2.0 ** 39, 7))
    same(secpe.rescale(ctx, a), o.rescale(a_o))


def test_mul_relin_and_rotation_bit_exact(env):
    o, ctx, keys, secpe = env
    rng = np.random.default_rng(5)
    a_o = o.encrypt(rng.uniform(-1, 1, 8), seed=31)
    b_o = o.encrypt(rng.uniform(-1, 1, 8), seed=32)
    a, b = to_gpu(secpe, ctx, a_o), to_gpu(secpe, ctx, b_o)
    same(secpe.mul_relin(ctx, keys, a, b), o.mul(a_o, b_o))
    low_o = o.drop(a_o, 4)
    low = to_gpu(secpe, ctx, low_o)
    same(secpe.mul_relin(ctx, keys, low, low), o.mul(low_o, low_o))
    for r in (1, 3, -4):
        same(secpe.rotate(ctx, keys, a, r), o.rotate(a_o, r))
    same(secpe.rotate(ctx, keys, low, -8), o.rotate(low_o, -8))


def test_hoisted_rotations_bit_exact(env):
    """secpe_rotate_hoisted: one ModUp for several steps, residue for residue
    the oracle's rotate_hoisted, at the top level and at a lower one; host
    errors for a missing key and an output aliasing the input."""
    o, ctx, keys, secpe = env
    a_o = o.encrypt(np.random.default_rng(6).uniform(-1, 1, 8), seed=33)
    a = to_gpu(secpe, ctx, a_o)
    steps = [1, 2, -4, 16, 3]
    for g, w in zip(secpe.rotate_hoisted(ctx, keys, a, steps), o.rotate_hoisted(a_o, steps)):
        same(g, w)
    low_o = o.drop(a_o, 5)
    low = to_gpu(secpe, ctx, low_o)
    for g, w in zip(secpe.rotate_hoisted(ctx, keys, low, [-2, 8]), o.rotate_hoisted(low_o, [-2, 8])):
        same(g, w)
    with pytest.raises(secpe.SecpeError) as e:
        secpe.rotate_hoisted(ctx, keys, a, [1, 5])
    assert e.value.code == -5
    with pytest.raises(secpe.SecpeError) as e:
        secpe.rotate_hoisted(ctx, keys, a, [1], outs=[a])
    assert e.value.code == -1


def test_keyswitch_primitive_bit_exact(env):
    import torch
    o, ctx, keys, secpe = env
    rng = np.random.default_rng(6)
    lv = 7
    d = np.stack([rng.integers(0, o.primes[i], o.n, dtype=np.uint64) for i in range(lv + 1)])
    k0, k1 = o.keyswitch(d, lv, o.rlk)
    dt = torch.zeros((ctx.L + 1, ctx.n), dtype=torch.int64, device="cuda")
    dt[: lv + 1] = torch.from_numpy(d.view(np.int64)).cuda()
    g0, g1 = secpe.keyswitch(ctx, keys, 0, dt, lv)
    assert np.array_equal(g0[: lv + 1].cpu().numpy().view(np.uint64), k0)
    assert np.array_equal(g1[: lv + 1].cpu().numpy().view(np.uint64), k1)


def test_refresh_bit_exact(env):
    o, ctx, keys, secpe = env
    a_o = o.drop(o.encrypt(np.linspace(-0.5, 0.5, 8), seed=41), 2)
    o.ridx = 3
    r_o = o.refresh(a_o, 1234)
    r = secpe.refresh_testonly(ctx, keys, to_gpu(secpe, ctx, a_o), 1234, 3)
    same(r, r_o)


def test_sign_and_max_bit_exact(env):
    o, ctx, keys, secpe = env
    rng = np.random.default_rng(7)
    x_o = o.encrypt(rng.uniform(-0.5, 0.5, 8), seed=51)
    o.qseed, o.ridx = 99, 0
    s_o = o.sign(x_o, 1)
    s, ridx = secpe.sign(ctx, keys, to_gpu(secpe, ctx, x_o), 1, 99, 0)
    same(s, s_o)
    assert ridx == o.ridx
    y_o = o.encrypt(rng.uniform(-0.5, 0.5, 8), seed=52)
    o.qseed, o.ridx = 98, 0
    m_o = o.max(x_o, y_o)
    m, ridx = secpe.vmax(ctx, keys, to_gpu(secpe, ctx, x_o), to_gpu(secpe, ctx, y_o), 98, 0)
    same(m, m_o)
    assert ridx == o.ridx


@pytest.mark.parametrize("C,K,seed", [(2, 5, 1), (3, 4, 2), (4, 2, 3), (2, 1, 4), (33, 3, 21)])
def test_toy_ensemble_argmax_bit_exact(env, C, K, seed):
    o, ctx, keys, secpe = env
    q = workloads.toy_query(seed=seed, K=K, C=C)
    cts_o = [o.encrypt_logits(q.logits[i], C, q.d_min, seed=q.enc_seeds[i]) for i in range(K)]
    y_o = o.aggregate(cts_o, q.d_min, q.d_max)
    o.reset_counters()
    z_o = o.argmax(y_o, C, qseed=q.qseed)
    cts = [to_gpu(secpe, ctx, c) for c in cts_o]
    y = secpe.ensemble_aggregate(ctx, cts, q.d_min, q.d_max)
    same(y, y_o)
    ctx.reset_counters()
    z = secpe.encrypted_argmax(ctx, keys, y, C, q.qseed)
    same(z, z_o)
    cnt = ctx.counters()
    for k in ("rotations", "signs", "relins", "refreshes"):
        assert cnt[k] == o.counters[k], k
    zd = secpe.decrypt(ctx, keys, z, C)
    zp = plainsim.ensemble_argmax(q.logits, q.d_min, q.d_max, ctx.n // 2)
    assert np.max(np.abs(zd - zp)) < TOL_Z
    assert int(np.argmax(zd)) == int(np.argmax(q.logits.mean(0)))


def test_toy_argmax_largest_class_count():
    """The largest Argmax the slots hold at N = 2^12: C = 1000 classes
    (ragged: C' = 1024, 2C' = N/2, 10 QuickMax rounds, every refresh range
    on its level plan), one-query and batched paths bit-exact with the
    oracle, counters equal, the exact index."""
    from paper_2502_00847_gb300 import secpe
    C, K = 1000, 2
    steps = [-1024] + [1 << i for i in range(10)]
    o = Oracle(TOY)
    o.keygen(91, rot_steps=steps)
    ctx = secpe.Context.from_params(TOY)
    keys = secpe.Keys(ctx, 91, steps)
    q = workloads.toy_query(seed=5, K=K, C=C)
    cts_o = [o.encrypt_logits(q.logits[i], C, q.d_min, seed=q.enc_seeds[i]) for i in range(K)]
    y_o = o.aggregate(cts_o, q.d_min, q.d_max)
    o.reset_counters()
    z_o = o.argmax(y_o, C, qseed=q.qseed)
    assert o.counters["refreshes"] >= 10
    cts = [to_gpu(secpe, ctx, c) for c in cts_o]
    ctx.reset_counters()
    z = secpe.encrypted_argmax(ctx, keys, secpe.ensemble_aggregate(ctx, cts, q.d_min, q.d_max), C, q.qseed)
    same(z, z_o)
    cnt = ctx.counters()
    for k in ("rotations", "signs", "relins", "refreshes"):
        assert cnt[k] == o.counters[k], k
    b = [dict(cts=cts, C=C, d_min=q.d_min, d_max=q.d_max, qseed=q.qseed, z_out=ctx.new_ct())]
    secpe.argmax_batch(ctx, keys, b)
    same(b[0]["z_out"], z_o)
    assert int(np.argmax(secpe.decrypt(ctx, keys, z, C))) == int(np.argmax(q.logits.mean(0)))
    with pytest.raises(secpe.SecpeError):
        secpe.encrypted_argmax(ctx, keys, z, 1025, q.qseed)      # 2C' > N/2


def test_toy_batch_equals_single(env):
    o, ctx, keys, secpe = env
    qs = [workloads.toy_query(seed=s, K=k, C=c) for s, k, c in ((11, 3, 2), (12, 2, 4), (13, 4, 3), (14, 2, 2))]
    inputs = []
    for q in qs:
        inputs.append([secpe.encrypt_logits(ctx, keys, q.logits[i], q.d_min, q.enc_seeds[i])
                       for i in range(q.K)])
    singles = []
    for q, cts in zip(qs, inputs):
        y = secpe.ensemble_aggregate(ctx, cts, q.d_min, q.d_max)
        singles.append(secpe.encrypted_argmax(ctx, keys, y, q.C, q.qseed))
    batch = [dict(cts=cts, C=q.C, d_min=q.d_min, d_max=q.d_max, qseed=q.qseed, z_out=ctx.new_ct())
             for q, cts in zip(qs, inputs)]
    secpe.argmax_batch(ctx, keys, batch)
    for s, b, q in zip(singles, batch, qs):
        z = b["z_out"]
        assert z.level == s.level and z.scale == s.scale
        assert np.array_equal(z.residues(), s.residues())
        assert int(np.argmax(secpe.decrypt(ctx, keys, z, q.C))) == int(np.argmax(q.logits.mean(0)))


def test_error_paths(env):
    o, ctx, keys, secpe = env
    ct = secpe.encrypt(ctx, keys, np.ones(4), 5)
    with pytest.raises(secpe.SecpeError) as e:
        secpe.rotate(ctx, keys, ct, 5)            # no Galois key for 5
    assert e.value.code == -5
    with pytest.raises(secpe.SecpeError) as e:
        secpe.encrypted_argmax(ctx, keys, ct, 1, 0)  # C = 1
    assert e.value.code == -1
    low = secpe.Ciphertext(ct.data, 1, ct.scale)
    with pytest.raises(secpe.SecpeError) as e:
        secpe.mul_relin(ctx, keys, low, low)      # level 1 < 1 + reserve
    assert e.value.code == -3
    other = secpe.Ciphertext(ct.data, ct.level, ct.scale * 2)
    with pytest.raises(secpe.SecpeError) as e:
        secpe.add(ctx, ct, other)
    assert e.value.code == -4
    # buffers off a 16-byte boundary are rejected on the host, nothing is launched
    import torch
    flat = torch.zeros(ct.data.numel() + 1, dtype=torch.int64, device="cuda")
    mis = secpe.Ciphertext(flat[1:].view(ct.data.shape), ct.level, ct.scale)
    assert mis.data.data_ptr() % 16 == 8
    before = ctx.counters()["launches"]
    for call in (lambda: secpe.add(ctx, ct, mis), lambda: secpe.rescale(ctx, mis),
                 lambda: secpe.ntt(ctx, flat[1:1 + ctx.n].view(1, ctx.n), [0])):
        with pytest.raises(secpe.SecpeError) as e:
            call()
        assert e.value.code == -1
    assert ctx.counters()["launches"] == before
    assert ctx.stream_status() == 0


def test_seeded_ciphertext_expansion(env):
    import torch
    o, ctx, keys, secpe = env
    rng = np.random.default_rng(9)
    cts = torch.zeros((3, 2, ctx.L + 1, ctx.n), dtype=torch.int64, device="cuda")
    seeds = [901, 902, 903]
    for i in range(3):
        secpe.encrypt_logits(ctx, keys, rng.uniform(-1, 1, 3), -1.0, seeds[i],
                             out=secpe.Ciphertext(cts[i], 0, ctx.scale))
    ref = cts.clone()
    cts[:, 1] = 0
    secpe.expand_seeded(ctx, cts, ctx.L, seeds)
    assert torch.equal(cts, ref)


def test_kernel_profiler_report(env):
    """kprof "*" records every launch under its kernel name; the report's
    launch count equals the context's launch counter for the same range."""
    import torch
    o, ctx, keys, secpe = env
    rng = np.random.default_rng(6)
    a = to_gpu(secpe, ctx, o.encrypt(rng.uniform(-1, 1, 8), seed=41))
    torch.cuda.synchronize()
    ctx.reset_counters()
    ctx.kprof_begin("*", max_launches=4096)
    secpe.mul_relin(ctx, keys, a, a)
    secpe.rotate(ctx, keys, a, 1)
    k = ctx.kprof_end()
    rows = ctx.kprof_report()
    assert rows and all(name.startswith("k_") and n > 0 and ms >= 0 for name, n, ms in rows)
    assert sum(n for _, n, _ in rows) == k["launches"] == ctx.counters()["launches"]
    assert [r[2] for r in rows] == sorted((r[2] for r in rows), reverse=True)


def test_bounded_device_wait_reports_timeout(env):
    """The bounded mbarrier wait of the bulk-copy kernels: with the arrival the
    wait completes (status 0); without it the wait runs out after its poll
    limit, the kernel records SECPE_ETIMEOUT (read and cleared by
    secpe_stream_status) and returns, and the context keeps working."""
    o, ctx, keys, secpe = env
    assert ctx.stream_status() == 0
    ctx.device_wait_selftest(True, polls=1 << 16)
    assert ctx.stream_status() == 0
    ctx.device_wait_selftest(False, polls=1 << 12)
    assert ctx.stream_status() == -7
    assert ctx.stream_status() == 0
    with pytest.raises(secpe.SecpeError) as e:
        ctx.device_wait_selftest(False, polls=0)
    assert e.value.code == -1
    a_o = o.encrypt(np.random.default_rng(9).uniform(-1, 1, 8), seed=91)
    same(secpe.rescale(ctx, to_gpu(secpe, ctx, a_o)), o.rescale(a_o))


def test_toy_batch_many_inputs_sum_in_chunks(env):
    """110 queries of K = 16 (1,760 input ciphertexts, more than one launch of
    the ensemble sum holds): every index is the exact argmax, and queries in
    both chunks equal the one-query path bit for bit."""
    o, ctx, keys, secpe = env
    qs = [workloads.toy_query(seed=300 + i, K=16, C=2 + i % 3) for i in range(110)]
    inputs = [[secpe.encrypt_logits(ctx, keys, q.logits[i], q.d_min, q.enc_seeds[i]) for i in range(q.K)]
              for q in qs]
    batch = [dict(cts=cts, C=q.C, d_min=q.d_min, d_max=q.d_max, qseed=q.qseed, z_out=ctx.new_ct())
             for q, cts in zip(qs, inputs)]
    secpe.argmax_batch(ctx, keys, batch)
    for q, b in zip(qs, batch):
        assert int(np.argmax(secpe.decrypt(ctx, keys, b["z_out"], q.C))) == int(np.argmax(q.logits.mean(0)))
    for i in (0, 95, 109):
        y = secpe.ensemble_aggregate(ctx, inputs[i], qs[i].d_min, qs[i].d_max)
        z = secpe.encrypted_argmax(ctx, keys, y, qs[i].C, qs[i].qseed)
        assert z.level == batch[i]["z_out"].level
        assert np.array_equal(z.residues(), batch[i]["z_out"].residues())
