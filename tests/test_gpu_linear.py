"""The upstream encrypted linear step (CLIP-style prompt ensembling, SecPE
Sec. 2.3) on the GPU: at N = 2^12 every residue of every prompt's logit
ciphertext, and of the Argmax run on them by the batched driver, equals the
oracle's (same input ciphertext, same plaintext coefficients); at N = 2^16
with the library's encoders (d = 512, C = 10, K = 16 prompts) the logits
decode to T_i x within 2^-20 and every task's index is the exact argmax."""
import numpy as np
import pytest

from oracle import ARGMAX8, TOY, Oracle
from paper_2502_00847_gb300 import workloads

pytestmark = pytest.mark.gpu


def test_toy_linear_step_and_argmax_bit_exact():
    import torch
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    pkg_build.build()
    torch.cuda.set_device(0)
    rot = [16, 32, 64, 128, 256, 512, -16, 1, 2, 4, 8]
    o = Oracle(TOY)
    o.keygen(616, rot_steps=rot)
    ctx = secpe.Context.from_params(TOY)
    keys = secpe.Keys(ctx, 616, rot)
    task = workloads.clip_task(d=64, C=10, K=3, seed=5)
    x_o = o.encrypt_replicated(task.x, task.C, seed=task.enc_seed)
    pts = o.linear_plaintexts(task.T, task.d_min)
    outs_o = o.linear_logits(x_o, pts, task.C, task.d)
    Wm = np.array([[int(v) for v in m] for m in pts[0]], dtype=np.int64)
    mask = np.array([int(v) for v in pts[1]], dtype=np.int64)
    pad = np.array([int(v) for v in pts[2]], dtype=np.int64)
    lin = secpe.Linear(ctx, coeffs=(Wm, mask, pad), K=task.K, C=task.C, d=task.d)
    x = secpe.Ciphertext.from_residues(x_o.c, x_o.level, x_o.scale, cap=ctx.L + 1)
    outs = lin.apply(keys, x)
    for y, y_o in zip(outs, outs_o):
        assert y.level == y_o.level and y.scale == y_o.scale
        assert np.array_equal(y.residues(), y_o.c)
    z_o = o.argmax(o.aggregate(outs_o, task.d_min, task.d_max), task.C, qseed=task.qseed)
    b = [dict(cts=outs, C=task.C, d_min=task.d_min, d_max=task.d_max, qseed=task.qseed, z_out=ctx.new_ct())]
    secpe.argmax_batch(ctx, keys, b)
    z = b[0]["z_out"]
    assert z.level == z_o.level and np.array_equal(z.residues(), z_o.c)
    assert int(np.argmax(secpe.decrypt(ctx, keys, z, task.C))) == int(np.argmax(task.logits().mean(0)))
    lin.close()


def test_full_size_linear_step_clip_shapes():
    import torch
    from paper_2502_00847_gb300 import secpe
    torch.cuda.set_device(0)
    ctx = secpe.Context.from_params(ARGMAX8)
    d, C, K = 512, 10, 16
    rot = [16 << t for t in range(9)] + [-16, 1, 2, 4, 8]
    keys = secpe.Keys(ctx, 617, rot)
    tasks = [workloads.clip_task(d=d, C=C, K=K, seed=40 + i) for i in range(3)]
    batch = []
    for t in tasks:
        lin = secpe.Linear(ctx, T=t.T, d_min=t.d_min)
        x = secpe.encrypt_replicated(ctx, keys, t.x, C, t.enc_seed)
        outs = lin.apply(keys, x)
        logits = t.logits()
        for i in (0, K - 1):
            v = secpe.decrypt(ctx, keys, outs[i], 32)
            assert np.max(np.abs(v[:C] - logits[i])) < 2.0 ** -20
            assert np.max(np.abs(v[C:16] - t.d_min)) < 2.0 ** -20 and np.max(np.abs(v[16:])) < 2.0 ** -20
        batch.append(dict(cts=outs, C=C, d_min=t.d_min, d_max=t.d_max, qseed=t.qseed, z_out=ctx.new_ct()))
        lin.close()
    secpe.argmax_batch(ctx, keys, batch)
    for t, b in zip(tasks, batch):
        zd = secpe.decrypt(ctx, keys, b["z_out"], C)
        assert int(np.argmax(zd)) == int(np.argmax(t.logits().mean(0)))
