"""Slot packing (SecPE Sec. 3.2, the slot-batching paragraph after Alg. 1),
checked on the CPU:

* the packed plaintext pipeline gives every input exactly the z its own
  one-query pipeline gives (Alg. 1's rotations by C' and 2^i < C' never read
  across blocks of 2C' slots where the result is taken);
* the library's O(N log N) host encoder and decoder agree with the direct
  canonical-embedding sums (the oracle's encoder, the definition written
  out) to within rounding;
* the oracle's encrypted Argmax on packed ciphertexts returns every packed
  input's exact argmax, within 2^-12 of the plaintext pipeline."""
import numpy as np
import pytest

from oracle import Oracle, TOY, plainsim
from paper_2502_00847_gb300 import workloads


def _sets(n, slots, seed, C, K, fill):
    return workloads.packed_queries(n, slots, seed=seed, K_choices=(K,), C_choices=(C,), fill=fill)


@pytest.mark.parametrize("C,K", [(2, 3), (3, 4), (6, 2), (14, 2), (64, 4)])
def test_packed_pipeline_equals_one_query_pipeline(C, K):
    slots = 2048
    pq = _sets(1, slots, 7, C, K, 1.0)[0]
    zp = plainsim.ensemble_argmax_packed(pq.logits, pq.d_min, pq.d_max, slots)
    assert zp.shape == (pq.P, C) and pq.P == slots // (2 * (1 << (C - 1).bit_length()))
    for b in range(pq.P):
        zs = plainsim.ensemble_argmax(pq.logits[b], pq.d_min, pq.d_max, slots)
        assert np.array_equal(zp[b], zs), b
        assert int(np.argmax(zp[b])) == int(np.argmax(pq.logits[b].mean(0)))


def test_packed_capacity_rule():
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    pkg_build.build()
    o = Oracle(TOY)
    for C in (1, 2, 3, 4, 5, 64, 512, 1024, 1025):
        cp = 1 << max(0, (C - 1).bit_length())
        assert secpe.packed_capacity(12, C) == (2048 // (2 * cp) if 2 * cp <= 2048 else 0)
        if 2 * cp <= 2048 and C > 1:
            assert o.packed_capacity(C) == secpe.packed_capacity(12, C)
    assert secpe.packed_capacity(16, 64) == 256 and secpe.packed_capacity(16, 2) == 8192
    # class counts far beyond any slot count (C' would overflow 32 bits) fit nowhere
    for C in (2 ** 30, 2 ** 30 + 1, 2 ** 31 - 1):
        assert secpe.packed_capacity(16, C) == 0 and secpe.packed_capacity(17, C) == 0
    # ... and the encoder refuses them before reading its input
    import ctypes
    one = np.zeros(1)
    m = np.zeros(1 << 12, dtype=np.int64)
    code = secpe.lib().secpe_encode_packed(12, ctypes.c_double(2.0 ** 40),
                                           one.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1, 2 ** 31 - 1,
                                           ctypes.c_double(-1.0), m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    assert code == -1


@pytest.mark.parametrize("log_n,C,fill", [(8, 3, 1.0), (12, 2, 1.0), (12, 14, 0.5)])
def test_fft_encoder_matches_direct_sums(log_n, C, fill):
    from oracle import Params
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    pkg_build.build()
    p = Params(log_n=log_n, q0_bits=40, q_bits=40, n_q=3, p_bits=60, n_p=1, dnum=3, log_scale=40)
    o = Oracle(p)
    n = 1 << log_n
    pq = _sets(1, n // 2, 9, C, 2, fill)[0]
    V = pq.prompt(0)
    direct = np.array([int(x) for x in o.encode_coeffs(o.pack_slots(V, pq.d_min), p.scale)], dtype=np.int64)
    fast = secpe.encode_packed(log_n, p.scale, V, pq.d_min)
    # the two summation orders round a handful of coefficients differently, by one unit
    assert np.max(np.abs(fast - direct)) <= 1
    assert np.mean(fast != direct) < 0.01
    # decoding either encoding returns the packed values (errors ~ N / scale)
    for m in (fast, direct):
        dec = secpe.decode_packed(log_n, p.scale, m.astype(np.float64), pq.P, C)
        assert np.max(np.abs(dec - V)) < 2.0 ** -25
    # the decoder against the oracle's direct decoding sums
    ref = o.decode_coeffs(direct, p.scale, pq.P * 2 * (1 << (C - 1).bit_length()))
    cp = 1 << (C - 1).bit_length()
    ref_blocks = np.stack([ref[b * 2 * cp: b * 2 * cp + C] for b in range(pq.P)])
    dec = secpe.decode_packed(log_n, p.scale, direct.astype(np.float64), pq.P, C)
    assert np.max(np.abs(dec - ref_blocks)) < 2.0 ** -30


def test_oracle_packed_argmax_every_input(toy_oracle):
    o = toy_oracle
    pq = _sets(1, o.n // 2, 11, 3, 3, 0.25)[0]     # 64 inputs of C = 3 (capacity 256)
    cts = [o.encrypt_logits_packed(pq.prompt(i), pq.d_min, seed=pq.enc_seeds[i]) for i in range(pq.K)]
    y = o.aggregate(cts, pq.d_min, pq.d_max)
    z = o.argmax(y, pq.C, qseed=pq.qseed)
    zd = o.decrypt_packed(z, pq.P, pq.C)
    zp = plainsim.ensemble_argmax_packed(pq.logits, pq.d_min, pq.d_max, o.n // 2)
    assert np.max(np.abs(zd - zp)) < 2.0 ** -12
    for b in range(pq.P):
        assert int(np.argmax(zd[b])) == int(np.argmax(pq.logits[b].mean(0))), b
