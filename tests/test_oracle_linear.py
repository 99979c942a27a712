"""The upstream encrypted linear step of CLIP-style prompt ensembling (SecPE
Sec. 2.3: y* = Argmax(sum_i I(x) . T(prompt_i))) in the oracle, on the CPU:
every prompt's logit ciphertext decodes to T_i x (a plain matrix-vector
product) within 2^-20 in the layout one-query Argmax expects (d_min in the
padding slots, zeros beyond C'), and aggregation + Alg. 1 on them return the
exact argmax of the ensembled logits."""
import numpy as np
import pytest

from oracle import Oracle, TOY, plainsim
from paper_2502_00847_gb300 import workloads


@pytest.fixture(scope="module")
def lin_oracle():
    o = Oracle(TOY)
    o.keygen(515, rot_steps=[16, 32, 64, 128, 256, 512, -16, 1, 2, 4, 8])
    return o


def test_replicated_layout_and_plaintexts(lin_oracle):
    o = lin_oracle
    task = workloads.clip_task(d=64, C=10, K=2, seed=3)
    slots = o.replicated_slots(task.x, task.C)
    assert slots.shape == (64 * 16,) and np.array_equal(slots[16 * 5: 16 * 6], np.full(16, task.x[5]))
    Wm, mask, pad = o.linear_plaintexts(task.T, task.d_min)
    # the weight plaintext decodes to T_i[c][j] at slot j C' + c
    w = o.decode_coeffs(Wm[1], float(o.primes[o.ctx.L]), 64 * 16).reshape(64, 16)
    assert np.max(np.abs(w[:, :10] - task.T[1].T)) < 2.0 ** -30 and np.max(np.abs(w[:, 10:])) < 2.0 ** -30


@pytest.mark.parametrize("seed", [3, 4])
def test_linear_logits_decode_to_matrix_vector_products(lin_oracle, seed):
    o = lin_oracle
    task = workloads.clip_task(d=64, C=10, K=3, seed=seed)
    x = o.encrypt_replicated(task.x, task.C, seed=task.enc_seed)
    pts = o.linear_plaintexts(task.T, task.d_min)
    outs = o.linear_logits(x, pts, task.C, task.d)
    logits = task.logits()
    for i, y in enumerate(outs):
        assert y.level == o.ctx.L - 2 and abs(y.scale - o.p.scale) <= o.p.scale * 2.0 ** -40
        v = o.decrypt(y, 32)
        assert np.max(np.abs(v[:10] - logits[i])) < 2.0 ** -20
        assert np.max(np.abs(v[10:16] - task.d_min)) < 2.0 ** -20
        assert np.max(np.abs(v[16:32])) < 2.0 ** -20
    z = o.argmax(o.aggregate(outs, task.d_min, task.d_max), task.C, qseed=task.qseed)
    zd = o.decrypt(z, task.C)
    zp = plainsim.ensemble_argmax(logits, task.d_min, task.d_max, o.n // 2)
    assert np.max(np.abs(zd - zp)) < 2.0 ** -12
    assert int(np.argmax(zd)) == int(np.argmax(logits.mean(0)))
