"""Slot-packed multi-query Argmax on the GPU (SecPE Sec. 3.2, the slot-batching
paragraph after Alg. 1): N/(4C') inputs of one task per ciphertext, Alg. 1
run once for all of them.

* N = 2^12: packed ciphertexts encrypted by the oracle, two packed query sets
  (C = 3 with 64 inputs, C = 2 with 100) through secpe_argmax_batch: every
  residue of both z equals the oracle's, every input's index is exact.
* N = 2^16 (the benchmark's parameter set): packed sets filled to capacity
  (C = 64: 256 inputs; C = 3: 4,096 inputs), encrypted by the library's
  packed encoder, through the batched driver: every one of the 4,352 inputs
  gets its exact argmax, and sampled blocks are within 2^-12 of the
  plaintext pipeline."""
import numpy as np
import pytest

from oracle import ARGMAX8, TOY, Oracle, plainsim
from paper_2502_00847_gb300 import workloads

pytestmark = pytest.mark.gpu

ROT = [1, 2, -2, -4]


def _set(slots, seed, C, K, fill):
    return workloads.packed_queries(1, slots, seed=seed, K_choices=(K,), C_choices=(C,), fill=fill)[0]


def test_toy_packed_batch_bit_exact():
    import torch
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    pkg_build.build()
    torch.cuda.set_device(0)
    o = Oracle(TOY)
    o.keygen(91, rot_steps=ROT)
    ctx = secpe.Context.from_params(TOY)
    keys = secpe.Keys(ctx, 91, ROT)
    sets = [_set(o.n // 2, 21, 3, 3, 0.25), _set(o.n // 2, 22, 2, 2, 100 / 512)]
    assert [s.P for s in sets] == [64, 100]
    batch, zo = [], []
    for pq in sets:
        cts_o = [o.encrypt_logits_packed(pq.prompt(i), pq.d_min, seed=pq.enc_seeds[i]) for i in range(pq.K)]
        z_o = o.argmax(o.aggregate(cts_o, pq.d_min, pq.d_max), pq.C, qseed=pq.qseed)
        zo.append(z_o)
        cts = [secpe.Ciphertext.from_residues(c.c, c.level, c.scale, cap=ctx.L + 1) for c in cts_o]
        batch.append(dict(cts=cts, C=pq.C, d_min=pq.d_min, d_max=pq.d_max, qseed=pq.qseed, z_out=ctx.new_ct()))
    secpe.argmax_batch(ctx, keys, batch)
    for pq, b, z_o in zip(sets, batch, zo):
        z = b["z_out"]
        assert z.level == z_o.level and z.scale == z_o.scale
        assert np.array_equal(z.residues(), z_o.c)
        zd = secpe.decrypt_packed(ctx, keys, z, pq.P, pq.C)
        assert np.max(np.abs(zd - o.decrypt_packed(z_o, pq.P, pq.C))) < 2.0 ** -30
        for i in range(pq.P):
            assert int(np.argmax(zd[i])) == int(np.argmax(pq.logits[i].mean(0))), i


def test_full_size_packed_every_input_correct():
    import torch
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    pkg_build.build()
    torch.cuda.set_device(0)
    ctx = secpe.Context.from_params(ARGMAX8)
    rot = [1, 2, 4, 8, 16, 32, -4, -64]
    keys = secpe.Keys(ctx, 93, rot)
    slots = ctx.n // 2
    sets = [_set(slots, 31, 64, 4, 1.0), _set(slots, 32, 3, 4, 1.0)]
    assert [s.P for s in sets] == [256, 4096]
    assert [secpe.packed_capacity(16, s.C) for s in sets] == [256, 4096]
    batch = []
    for pq in sets:
        cts = [secpe.encrypt_logits_packed(ctx, keys, pq.prompt(i), pq.d_min, pq.enc_seeds[i]) for i in range(pq.K)]
        # the library's encoder round-trips the packed values
        back = secpe.decrypt_packed(ctx, keys, cts[0], pq.P, pq.C)
        assert np.max(np.abs(back - pq.prompt(0))) < 2.0 ** -20
        batch.append(dict(cts=cts, C=pq.C, d_min=pq.d_min, d_max=pq.d_max, qseed=pq.qseed, z_out=ctx.new_ct()))
    secpe.argmax_batch(ctx, keys, batch)
    torch.cuda.synchronize()
    for pq, b in zip(sets, batch):
        zd = secpe.decrypt_packed(ctx, keys, b["z_out"], pq.P, pq.C)
        exact = pq.logits.mean(1).argmax(1)
        assert np.array_equal(zd.argmax(1), exact)
        # a few blocks against the plaintext pipeline (the full packed vector)
        zp = plainsim.ensemble_argmax_packed(pq.logits, pq.d_min, pq.d_max, slots)
        for i in (0, 1, pq.P // 2, pq.P - 1):
            assert np.max(np.abs(zd[i] - zp[i])) < 2.0 ** -12, i
