"""Continuous-batching server (secpe_server_*): every query in flight advances
one phase per step, so queries submitted while others are mid-circuit start
at once and can finish first; each result is bit-identical alone and in the
mix, and equal to the one-query path; admission by HBM budget, missing keys,
cancellation and bounded waits are host-side failure paths (no GPU fault)."""
import numpy as np
import pytest

from oracle import TOY
from paper_2502_00847_gb300 import workloads

pytestmark = pytest.mark.gpu

ROT = [1, 2, -2, -4]


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    pkg_build.build()
    torch.cuda.set_device(0)
    ctx = secpe.Context.from_params(TOY)
    keys = secpe.Keys(ctx, 31, ROT)
    qs = [workloads.toy_query(seed=s, K=k, C=c) for s, k, c in
          ((21, 3, 2), (22, 2, 4), (23, 4, 3), (24, 2, 2), (25, 3, 4))]
    inputs = [[secpe.encrypt_logits(ctx, keys, q.logits[i], q.d_min, q.enc_seeds[i]) for i in range(q.K)]
              for q in qs]
    ref = []
    for q, cts in zip(qs, inputs):
        y = secpe.ensemble_aggregate(ctx, cts, q.d_min, q.d_max)
        ref.append(secpe.encrypted_argmax(ctx, keys, y, q.C, q.qseed).residues())
    return ctx, keys, qs, inputs, ref, secpe


def submit(srv, ctx, q, cts):
    z = ctx.new_ct()
    return srv.submit(cts, q.C, q.d_min, q.d_max, q.qseed, z), z


def test_interleaved_submissions_match_single_query_path(env):
    ctx, keys, qs, inputs, ref, secpe = env
    srv = secpe.Server(ctx, keys, hbm_budget_bytes=8 << 30, max_batch=8)
    tickets = []
    # two queries, a few phases, then the rest arrive while those are in flight
    for i in (0, 1):
        tickets.append(submit(srv, ctx, qs[i], inputs[i]))
    assert srv.step() == 2          # both start at once (two groups: different C')
    assert srv.step() >= 1
    for i in (2, 3, 4):
        tickets.append(submit(srv, ctx, qs[i], inputs[i]))
    batched = 0
    for _ in range(200):
        n = srv.step()
        batched = max(batched, n)
        if n == 0:
            break
    assert batched >= 2, "later arrivals were never batched with earlier ones"
    for i, (t, z) in enumerate(tickets):
        assert srv.wait(t, 60.0) == 1
        assert np.array_equal(z.residues(), ref[i]), i
        d = secpe.decrypt(ctx, keys, z, qs[i].C)
        assert int(np.argmax(d)) == int(np.argmax(qs[i].logits.mean(0)))
        srv.forget(t)
    st = srv.stats()
    assert st["active"] == 0 and st["waiting"] == 0 and st["in_flight_bytes"] == 0


def test_alone_equals_in_mix(env):
    ctx, keys, qs, inputs, ref, secpe = env
    alone = secpe.Server(ctx, keys, hbm_budget_bytes=8 << 30, max_batch=8)
    t, z = submit(alone, ctx, qs[2], inputs[2])
    alone.wait(t, 60.0)
    mixed = secpe.Server(ctx, keys, hbm_budget_bytes=8 << 30, max_batch=8)
    subs = [submit(mixed, ctx, qs[i], inputs[i]) for i in (4, 2, 0, 3)]
    for tk, _ in subs:
        mixed.wait(tk, 60.0)
    assert np.array_equal(z.residues(), subs[1][1].residues())


def test_admission_by_budget(env):
    ctx, keys, qs, inputs, ref, secpe = env
    with pytest.raises(secpe.SecpeError) as e:
        secpe.Server(ctx, keys, hbm_budget_bytes=1 << 20, max_batch=8)
    assert e.value.code == -8
    # room for one query in flight: the second waits until the first is done
    probe = secpe.Server(ctx, keys, hbm_budget_bytes=8 << 30, max_batch=1)
    s0 = probe.stats()
    one = s0["keys_bytes"] + s0["scratch_bytes"] + 3 * 2 * ctx.n * (ctx.L + 1) * 8
    srv = secpe.Server(ctx, keys, hbm_budget_bytes=one + 1, max_batch=1)
    (t0, z0), (t1, z1) = submit(srv, ctx, qs[0], inputs[0]), submit(srv, ctx, qs[3], inputs[3])
    srv.step()
    st = srv.stats()
    assert st["active"] == 1 and st["waiting"] == 1
    srv.wait(t0, 60.0)
    srv.wait(t1, 60.0)
    assert np.array_equal(z0.residues(), ref[0]) and np.array_equal(z1.residues(), ref[3])


def test_missing_key_cancel_and_timeout(env):
    ctx, keys, qs, inputs, ref, secpe = env
    srv = secpe.Server(ctx, keys, hbm_budget_bytes=8 << 30, max_batch=8)
    q = workloads.toy_query(seed=40, K=2, C=6)      # needs RotR(8) and RotL(4): not generated
    cts = [secpe.encrypt_logits(ctx, keys, q.logits[i], q.d_min, q.enc_seeds[i]) for i in range(q.K)]
    with pytest.raises(secpe.SecpeError) as e:
        submit(srv, ctx, q, cts)
    assert e.value.code == -5
    t0, z0 = submit(srv, ctx, qs[1], inputs[1])
    t1, z1 = submit(srv, ctx, qs[0], inputs[0])
    srv.step()
    srv.cancel(t0)
    assert srv.poll(t0) == -1
    with pytest.raises(secpe.SecpeError) as e:
        srv.wait(t1, 0.0)
    assert e.value.code == -7
    assert srv.wait(t1, 60.0) == 1
    assert np.array_equal(z1.residues(), ref[0])
    assert ctx.stream_status() == 0


def test_two_tenants_in_one_server(env):
    """Queries of two tenants (different secret keys) interleaved: each is
    batched only with its own tenant, equals the one-query path with its own
    keys bit for bit, and the second key set is counted as resident."""
    ctx, keys, qs, inputs, ref, secpe = env
    keys_b = secpe.Keys(ctx, 32, ROT)
    inputs_b = [[secpe.encrypt_logits(ctx, keys_b, q.logits[i], q.d_min, q.enc_seeds[i]) for i in range(q.K)]
                for q in qs]
    ref_b = []
    for q, cts in zip(qs, inputs_b):
        y = secpe.ensemble_aggregate(ctx, cts, q.d_min, q.d_max)
        ref_b.append(secpe.encrypted_argmax(ctx, keys_b, y, q.C, q.qseed).residues())
    srv = secpe.Server(ctx, keys, hbm_budget_bytes=8 << 30, max_batch=8)
    kb0 = srv.stats()["keys_bytes"]
    subs = []
    for i in range(len(qs)):
        subs.append(("a", i, submit(srv, ctx, qs[i], inputs[i])))
        z = ctx.new_ct()
        subs.append(("b", i, (srv.submit(inputs_b[i], qs[i].C, qs[i].d_min, qs[i].d_max, qs[i].qseed, z,
                                         keys=keys_b), z)))
    assert srv.stats()["keys_bytes"] == 2 * kb0
    for who, i, (t, z) in subs:
        assert srv.wait(t, 60.0) == 1
        assert np.array_equal(z.residues(), ref[i] if who == "a" else ref_b[i]), (who, i)
        k = keys if who == "a" else keys_b
        assert int(np.argmax(secpe.decrypt(ctx, k, z, qs[i].C))) == int(np.argmax(qs[i].logits.mean(0)))


def test_two_tenants_in_one_batch(env):
    """secpe_argmax_batch over queries of two tenants: one batch per key set,
    bit-identical to the one-query path with each query's keys."""
    ctx, keys, qs, inputs, ref, secpe = env
    keys_b = secpe.Keys(ctx, 33, ROT)
    inputs_b = [[secpe.encrypt_logits(ctx, keys_b, q.logits[i], q.d_min, q.enc_seeds[i]) for i in range(q.K)]
                for q in qs]
    batch = []
    for i, q in enumerate(qs):
        batch.append(dict(cts=inputs[i], C=q.C, d_min=q.d_min, d_max=q.d_max, qseed=q.qseed, z_out=ctx.new_ct()))
        batch.append(dict(cts=inputs_b[i], C=q.C, d_min=q.d_min, d_max=q.d_max, qseed=q.qseed, z_out=ctx.new_ct(),
                          keys=keys_b))
    secpe.argmax_batch(ctx, keys, batch)
    for i, q in enumerate(qs):
        assert np.array_equal(batch[2 * i]["z_out"].residues(), ref[i])
        y = secpe.ensemble_aggregate(ctx, inputs_b[i], q.d_min, q.d_max)
        zb = secpe.encrypted_argmax(ctx, keys_b, y, q.C, q.qseed)
        assert np.array_equal(batch[2 * i + 1]["z_out"].residues(), zb.residues())
        assert int(np.argmax(secpe.decrypt(ctx, keys_b, zb, q.C))) == int(np.argmax(q.logits.mean(0)))


def test_arrival_mid_flight_finishes_before_the_cohort(env):
    """Two queries with C = 16 (six phases) are two phases in when a C = 2
    query (three phases) arrives: it starts in the next step, overlapping the
    cohort's QuickMax rounds, and completes while the cohort is still in
    flight; all three results equal their one-query evaluations bit for bit."""
    ctx, keys, qs, inputs, ref, secpe = env
    rot = [1, 2, 4, 8, -2, -16]
    k2 = secpe.Keys(ctx, 34, rot)
    big = [workloads.toy_query(seed=s, K=2, C=16) for s in (61, 62)]
    small = workloads.toy_query(seed=63, K=3, C=2)
    cts = {id(q): [secpe.encrypt_logits(ctx, k2, q.logits[i], q.d_min, q.enc_seeds[i]) for i in range(q.K)]
           for q in big + [small]}
    solo = {}
    for q in big + [small]:
        y = secpe.ensemble_aggregate(ctx, cts[id(q)], q.d_min, q.d_max)
        solo[id(q)] = secpe.encrypted_argmax(ctx, k2, y, q.C, q.qseed).residues()
    import torch
    srv = secpe.Server(ctx, k2, hbm_budget_bytes=8 << 30, max_batch=8)
    tb = [submit(srv, ctx, q, cts[id(q)]) for q in big]
    assert srv.step() == 2
    assert srv.step() == 2
    ts = submit(srv, ctx, small, cts[id(small)])
    finished_first = False
    for _ in range(20):
        n = srv.step()
        torch.cuda.synchronize()
        if srv.poll(ts[0]) == 1:
            finished_first = all(srv.poll(t) == 0 for t, _ in tb)
            break
        assert n == 3, "the new query did not run beside the cohort"
    assert finished_first, "the mid-flight arrival waited for the cohort"
    for q, (t, z) in zip(big + [small], tb + [ts]):
        assert srv.wait(t, 60.0) == 1
        assert np.array_equal(z.residues(), solo[id(q)])
        assert int(np.argmax(secpe.decrypt(ctx, k2, z, q.C))) == int(np.argmax(q.logits.mean(0)))

