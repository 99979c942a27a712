"""Residue parity on the benchmark's own configuration: N = 2^16, a 60-bit q_0
+ 23 x 50-bit primes, 8 special primes, dnum = 3, Delta = 2^50.

A two-query batch (C = 2 and C = 3, K = 4 each: two values of r = log2 C',
so two phase ranges, and a refresh inside the C = 3 query's second QuickMax
round) runs through secpe_argmax_batch and through the batch captured as one
CUDA graph and replayed.  Every residue of both z, their levels and scales,
and the operation counts are compared with the CPU oracle's one-query
evaluation of the same input ciphertexts (SecPE Sec. 3.1 step 3, Eq. norm,
Alg. 1, Eq. max, Eq. comp).  The oracle's two queries run in spawned worker
processes while the GPU works."""
import multiprocessing

import numpy as np
import pytest

from oracle import ARGMAX8, Oracle, plainsim
from oracle import jobs as ojobs
from paper_2502_00847_gb300 import workloads

pytestmark = pytest.mark.gpu

KEY_SEED = 880
ROT = [1, 2, -2, -4]
TOL_Z = 2.0 ** -12


def _queries():
    q2 = workloads.argmax_queries(1, seed=41, K_choices=(4,), C_choices=(2,))[0]
    q3 = workloads.argmax_queries(1, seed=42, K_choices=(4,), C_choices=(3,))[0]
    return [q2, q3]


@pytest.fixture(scope="module")
def run():
    import torch
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    qs = _queries()
    jobs = [("argmax8", KEY_SEED, ROT, q.logits, q.d_min, q.d_max, q.qseed, q.enc_seeds) for q in qs]
    pool = multiprocessing.get_context("spawn").Pool(len(jobs))
    pending = pool.map_async(ojobs.ensemble_query, jobs)
    try:
        # the same input ciphertexts, encrypted by the oracle in this process
        o = Oracle(ARGMAX8)
        o.keygen(KEY_SEED, rot_steps=ROT)
        cts_o = [[o.encrypt_logits(q.logits[i], q.C, q.d_min, seed=q.enc_seeds[i]) for i in range(q.K)]
                 for q in qs]
        pkg_build.build()
        torch.cuda.set_device(0)
        ctx = secpe.Context.from_params(ARGMAX8)
        keys = secpe.Keys(ctx, KEY_SEED, ROT)
        cts = [[secpe.Ciphertext.from_residues(c.c, c.level, c.scale, cap=ctx.L + 1) for c in row] for row in cts_o]

        def batch():
            return [dict(cts=cts[i], C=q.C, d_min=q.d_min, d_max=q.d_max, qseed=q.qseed, z_out=ctx.new_ct())
                    for i, q in enumerate(qs)]

        direct = batch()
        ctx.reset_counters()
        secpe.argmax_batch(ctx, keys, direct)
        torch.cuda.synchronize()
        counters = ctx.counters()
        graphed = batch()
        g = secpe.Graph(ctx, keys, graphed)
        for _ in range(2):
            g.launch()
        torch.cuda.synchronize()
        g.close()
        ref = pending.get(timeout=1800)
    finally:
        pool.close()
        pool.join()
    return dict(qs=qs, ctx=ctx, keys=keys, direct=direct, graphed=graphed, counters=counters, ref=ref,
                secpe=secpe)


def _same(z, r):
    assert z.level == r["level"]
    assert z.scale == r["scale"]
    assert np.array_equal(z.residues(), r["z"])


def test_batched_argmax_every_residue_equals_oracle(run):
    for b, r in zip(run["direct"], run["ref"]):
        _same(b["z_out"], r)
    # two phase ranges and a refresh inside QuickMax (C = 3: greedy levels run out in QuickMax round k = 2)
    assert [r["counters"]["refreshes"] for r in run["ref"]][1] >= 2
    for k in ("rotations", "signs", "relins", "refreshes"):
        assert run["counters"][k] == sum(r["counters"][k] for r in run["ref"]), k


def test_graph_replay_every_residue_equals_oracle(run):
    for b, r in zip(run["graphed"], run["ref"]):
        _same(b["z_out"], r)


def test_decoded_and_index(run):
    secpe, ctx, keys = run["secpe"], run["ctx"], run["keys"]
    for q, b, r in zip(run["qs"], run["direct"], run["ref"]):
        zd = secpe.decrypt(ctx, keys, b["z_out"], q.C)
        assert np.max(np.abs(zd - r["decoded"])) < 2.0 ** -30
        zp = plainsim.ensemble_argmax(q.logits, q.d_min, q.d_max, ctx.n // 2)
        assert np.max(np.abs(zd - zp)) < TOL_Z
        assert int(np.argmax(zd)) == int(np.argmax(q.logits.mean(0)))
