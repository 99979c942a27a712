"""Whole-query jobs of the CPU oracle, runnable in worker processes.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only tests/, the smoke check and the
benchmark's CPU-baseline and reference legs may call this module.

A job is a plain tuple (picklable for a process pool started with spawn), so
several queries can run concurrently on the host cores while the GPU works.
`ensemble_query` runs the server side of SecPE's workflow for one query
(Sec. 3.1 steps 1-3: encrypted logits, ensemble aggregation with the Eq. norm
scale, Alg. 1), exactly as the oracle defines it one query at a time.
"""
import time

import numpy as np

from . import params as _params
from .ckks import Oracle


_CACHE = {}


def make_oracle(preset, key_seed, rot_steps):
    """An oracle with its keys; kept per worker process, so that repeated
    jobs with the same keys pay keygen once."""
    key = (preset, key_seed, tuple(rot_steps))
    if key not in _CACHE:
        o = Oracle(_params.PRESETS[preset])
        o.keygen(key_seed, rot_steps=list(rot_steps))
        _CACHE.clear()
        _CACHE[key] = o
    return _CACHE[key]


def ensemble_query(job):
    """job = (preset, key_seed, rot_steps, logits [K][C], d_min, d_max, qseed,
    enc_seeds).  Returns a dict with the input ciphertexts' residues
    (`inputs`, optional), z's residues, level and scale, the oracle's op
    counters and the seconds spent in aggregation + Argmax (keygen and the
    client-side encryption excluded)."""
    preset, key_seed, rot_steps, logits, d_min, d_max, qseed, enc_seeds = job[:8]
    want_inputs = len(job) > 8 and bool(job[8])
    o = make_oracle(preset, key_seed, rot_steps)
    logits = np.asarray(logits, dtype=np.float64)
    K, C = logits.shape
    cts = [o.encrypt_logits(logits[i], C, d_min, seed=int(enc_seeds[i])) for i in range(K)]
    o.reset_counters()
    t0 = time.perf_counter()
    y = o.aggregate(cts, d_min, d_max)
    z = o.argmax(y, C, qseed=int(qseed))
    seconds = time.perf_counter() - t0
    out = {"z": z.c, "level": z.level, "scale": z.scale, "counters": dict(o.counters), "seconds": seconds,
           "decoded": o.decrypt(z, C)}
    if want_inputs:
        out["inputs"] = [(c.c, c.level, c.scale) for c in cts]
    return out


def hmult_sample(job):
    """job = (preset, key_seed, rot_steps, level, seed): seconds of one HMult +
    relinearisation + rescale at `level` (the circuit's dominant operation)."""
    preset, key_seed, rot_steps, level, seed = job
    o = make_oracle(preset, key_seed, rot_steps)
    rng = np.random.default_rng(seed)
    a = o.drop(o.encrypt(rng.uniform(-1, 1, 8), seed=seed, level=max(level, 1)), level)
    t0 = time.perf_counter()
    o.mul(a, a)
    return time.perf_counter() - t0
