"""Sampled residue parity of the benchmark's own step, at its full size and in
its launch configuration: the 256-query mix (N = 2^16, the argmax8 set,
K in {4, 8, 16}, C in {2, 3, 4, 6, 14, 64}, seed 4; 2,428 input
ciphertexts) encrypted on the device with the benchmark's key seed and
rotation keys, the N = 2^16 launch configurations chosen by the autotuner,
and the whole batch captured as one CUDA graph and replayed twice.

Two queries of the mix, the cheapest with C = 2 and the cheapest with C = 4
(one and two QuickMax rounds), are evaluated one at a time by the CPU oracle
from the same logits, encryption seeds and query seed, with keys from the
same key seed (each key depends only on that seed and its Galois element,
so the oracle generates only the rotations its query uses).  Their input
ciphertexts in the batch are the oracle's own encryptions (the library's
host encoding may round a coefficient differently; encryption of the same
coefficients is bit-exact), placed at their positions in the mix; every
other query is encrypted on the device, as the benchmark does.  Every residue
of their z, its level and its scale equal the oracle's (SecPE Sec. 3.1
step 3, Eq. norm, Alg. 1, Eq. max, Eq. comp), and the decoded z agrees with
the oracle's decoding and with the FP64 plaintext simulation.  Every query
of the mix gets its exact argmax.  The oracle's queries run in spawned
worker processes while the GPU works."""
import gc
import multiprocessing

import numpy as np
import pytest

from oracle import ARGMAX8, Oracle, plainsim
from oracle import jobs as ojobs
from paper_2502_00847_gb300 import workloads

pytestmark = pytest.mark.gpu

KEY_SEED = 1000                                             # the benchmark's keys (rank 0)
ROT_STEPS = [-2, -4, -8, -16, -64, 1, 2, 4, 8, 16, 32]      # the benchmark's rotation keys
N_QUERIES, MIX_SEED = 256, 4
TOL_Z = 2.0 ** -12


def _sample(qs):
    """Indices of the query with the smallest K (then the lowest index) among
    those with C = 2, and among those with C = 4."""
    out = []
    for C in (2, 4):
        idx = [i for i, q in enumerate(qs) if q.C == C]
        out.append(min(idx, key=lambda i: (qs[i].K, i)))
    return out


def _rotations(C):
    """The rotations Alg. 1 applies for C classes: RotR(C') and RotL(2^i), 2^i < C'."""
    cp = 1 << (C - 1).bit_length()
    return [-cp] + [1 << i for i in range(cp.bit_length() - 1)]


def _gpu_step(qs, sample, own):
    """The benchmark's step on the whole mix; returns host copies only, so that
    every device tensor is released when it returns."""
    import torch
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    from paper_2502_00847_gb300.presets import PRESETS
    pkg_build.build()
    torch.cuda.set_device(0)
    # start from an empty cache and pool: earlier test modules may have left both full
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    secpe.pool_usage(trim=True)
    dev = torch.device("cuda", 0)
    ctx = secpe.Context.from_params(PRESETS["argmax8"])
    keys = secpe.Keys(ctx, KEY_SEED, ROT_STEPS)
    n, cap = ctx.n, ctx.L + 1
    inputs = torch.empty((sum(q.K for q in qs), 2, cap, n), dtype=torch.int64, device=dev)
    views, off = [], 0
    for qi, q in enumerate(qs):
        cts = []
        for i in range(q.K):
            if qi in own:
                co = own[qi][i]
                src = torch.from_numpy(np.ascontiguousarray(co.c, dtype=np.uint64).view(np.int64))
                inputs[off, :, : co.level + 1].copy_(src)
                c = secpe.Ciphertext(inputs[off], co.level, co.scale)
            else:
                c = secpe.Ciphertext(inputs[off], 0, ctx.scale)
                secpe.encrypt_logits(ctx, keys, q.logits[i], q.d_min, q.enc_seeds[i], out=c)
            cts.append(c)
            off += 1
        views.append(cts)
    zbuf = torch.zeros((len(qs), 2, cap, n), dtype=torch.int64, device=dev)
    batch = [dict(cts=views[i], C=q.C, d_min=q.d_min, d_max=q.d_max, qseed=q.qseed,
                  z_out=secpe.Ciphertext(zbuf[i], 0, ctx.scale)) for i, q in enumerate(qs)]
    torch.cuda.synchronize()
    ctx.autotune()
    g = secpe.Graph(ctx, keys, batch)
    for _ in range(2):
        g.launch()
    torch.cuda.synchronize()
    g.close()
    got = {i: dict(level=batch[i]["z_out"].level, scale=batch[i]["z_out"].scale,
                   z=batch[i]["z_out"].residues()) for i in sample}
    decoded = [secpe.decrypt(ctx, keys, batch[i]["z_out"], q.C) for i, q in enumerate(qs)]
    torch.cuda.synchronize()
    keys.close()
    ctx.close()
    secpe.pool_usage(trim=True)   # hand the batch's scratch back to the device for the next tests
    return got, decoded


@pytest.fixture(scope="module")
def run():
    import torch
    qs = workloads.argmax_queries(N_QUERIES, seed=MIX_SEED)
    sample = _sample(qs)
    jobs = [("argmax8", KEY_SEED, _rotations(qs[i].C), qs[i].logits, qs[i].d_min, qs[i].d_max, qs[i].qseed,
             qs[i].enc_seeds) for i in sample]
    pool = multiprocessing.get_context("spawn").Pool(len(jobs))
    pending = pool.map_async(ojobs.ensemble_query, jobs)
    try:
        # the sampled queries' inputs, encrypted by the oracle in this process
        o = Oracle(ARGMAX8)
        o.keygen(KEY_SEED)
        own = {i: [o.encrypt_logits(qs[i].logits[k], qs[i].C, qs[i].d_min, seed=int(qs[i].enc_seeds[k]))
                   for k in range(qs[i].K)] for i in sample}
        del o
        got, decoded = _gpu_step(qs, sample, own)
        torch.cuda.empty_cache()
        ref = pending.get(timeout=1800)
    finally:
        pool.close()
        pool.join()
    return dict(qs=qs, sample=sample, got=got, decoded=decoded, ref=dict(zip(sample, ref)))


def test_sample_covers_one_and_two_quickmax_rounds(run):
    qs, sample = run["qs"], run["sample"]
    assert [qs[i].C for i in sample] == [2, 4]
    assert len(qs) == N_QUERIES and sum(q.K for q in qs) == 2428


def test_sampled_queries_every_residue_equals_oracle(run):
    for i in run["sample"]:
        g, r = run["got"][i], run["ref"][i]
        assert g["level"] == r["level"], i
        assert g["scale"] == r["scale"], i
        assert np.array_equal(g["z"], r["z"]), i


def test_sampled_queries_decoded(run):
    for i in run["sample"]:
        q, zd = run["qs"][i], run["decoded"][i]
        assert np.max(np.abs(zd - run["ref"][i]["decoded"])) < 2.0 ** -30, i
        zp = plainsim.ensemble_argmax(q.logits, q.d_min, q.d_max, 1 << 15)
        assert np.max(np.abs(zd - zp)) < TOL_Z, i


def test_every_query_of_the_mix_exact_index(run):
    for i, (q, zd) in enumerate(zip(run["qs"], run["decoded"])):
        assert int(np.argmax(zd)) == int(np.argmax(q.logits.mean(0))), i
