"""CKKS bootstrapping in the oracle (the reading of SecPE Sec. 2.2 / 4.1: it
relies on bootstrapping without describing it), pinned step by step against
what the mathematics fixes, on the bootstrapping toy set (N = 2^12, q0
50-bit, 7 x 40-bit computation primes, 16 x 60-bit bootstrapping primes,
sparse secret of weight 32), block n = 16:

* the sparse secret has exactly h nonzero coefficients in {-1, 1}; the
  conjugation key conjugates complex slots; the complex encoder agrees
  with the real one on real vectors and round-trips complex ones;
* ModRaise: the lifted ciphertext decrypts to m + q0 I exactly, |I| <= (h+1)/2;
* SubSum: the slots become the n-periodic block sums;
* CoeffToSlot: slots [0, 2n) hold the subring coefficients of the raised
  plaintext divided by q0 (big-integer decryption);
* EvalMod: sin(2 pi u) of its input slots;
* the whole bootstrap returns an n-periodic input unchanged (the block
  average) at level L - 16 within 2^-20."""
import numpy as np
import pytest

from oracle import BOOT_TOY, Oracle
from oracle.boot import BootPlan
from oracle.ckks import STEP_CONJ

N_BLOCK = 16
TOL_BOOT = 2.0 ** -20


@pytest.fixture(scope="module")
def boot():
    o = Oracle(BOOT_TOY)
    plan = BootPlan(o, N_BLOCK)
    o.keygen(99, rot_steps=plan.rotation_steps())
    rng = np.random.default_rng(1)
    v = rng.uniform(-1, 1, N_BLOCK)
    ct = o.drop(o.encrypt(np.tile(v, (o.n // 2) // N_BLOCK), seed=5, level=7), 0)
    x = plan.mod_raise(ct)
    xs = plan.sub_sum(x)
    u = plan.coeff_to_slot(xs)
    f = plan.eval_mod(u)
    z = plan.slot_to_coeff(f, ct.scale)
    return dict(o=o, plan=plan, v=v, ct=ct, x=x, xs=xs, u=u, f=f, z=z)


def test_sparse_secret_and_primes(boot):
    o = boot["o"]
    s = o.s_coeffs
    assert np.count_nonzero(s) == BOOT_TOY.secret_hw and set(np.unique(s)) <= {-1, 0, 1}
    bits = [p.bit_length() for p in o.primes]
    assert bits[0] == 50 and all(b in (40, 41) for b in bits[1:8])
    assert all(b == 60 for b in bits[8:24]) and len(bits) == 28 and all(b == 60 for b in bits[24:])


def test_complex_encoding_and_conjugation(boot):
    o = boot["o"]
    rng = np.random.default_rng(3)
    re = rng.uniform(-1, 1, 8)
    assert np.array_equal(np.array(o.encode_complex(re, 2.0 ** 30), dtype=object),
                          np.array(o.encode_coeffs(re, 2.0 ** 30), dtype=object))
    z = rng.uniform(-1, 1, 8) + 1j * rng.uniform(-1, 1, 8)
    m = o.encode_complex(z, 2.0 ** 40)
    assert np.max(np.abs(o.decode_complex(m, 2.0 ** 40, 8) - z)) < 2.0 ** -30
    ct = o.encrypt_coeffs(m, 10, 2.0 ** 40, seed=8)
    zc = o.decode_complex(o.decrypt_coeffs(o.rotate(ct, STEP_CONJ)), 2.0 ** 40, 8)
    assert np.max(np.abs(zc - np.conj(z))) < 2.0 ** -20


def test_mod_raise_exact(boot):
    o, ct, x = boot["o"], boot["ct"], boot["x"]
    q0 = o.primes[0]
    t = o.decrypt_coeffs(x)
    m = o.decrypt_coeffs(ct)
    assert x.level == o.ctx.L
    d = [int(a) - int(b) for a, b in zip(t, m)]
    assert all(v % q0 == 0 for v in d)
    assert max(abs(v // q0) for v in d) <= (BOOT_TOY.secret_hw + 1) // 2


def test_sub_sum_is_block_sum(boot):
    o, plan = boot["o"], boot["plan"]
    rng = np.random.default_rng(4)
    v = rng.uniform(-1, 1, 100)
    ct = o.encrypt(v, seed=9)
    w = o.decrypt(plan.sub_sum(ct), o.n // 2)
    full = np.zeros(o.n // 2)
    full[:100] = v
    exp = sum(np.roll(full, -k * N_BLOCK) for k in range((o.n // 2) // N_BLOCK))
    assert np.max(np.abs(w - exp)) < 2.0 ** -20


def test_coeff_to_slot_gives_subring_coefficients(boot):
    o, xs, u = boot["o"], boot["xs"], boot["u"]
    q0 = o.primes[0]
    t = o.decrypt_coeffs(boot["x"])
    step = o.n // (2 * N_BLOCK)
    p = np.array([float(t[a * step]) for a in range(2 * N_BLOCK)]) / q0
    got = o.decrypt(u, 4 * N_BLOCK)
    assert u.level == o.ctx.L - 1 and u.scale == xs.scale
    assert np.max(np.abs(got[:2 * N_BLOCK] - p)) < 2.0 ** -30
    assert np.max(np.abs(got[2 * N_BLOCK:] - p)) < 2.0 ** -30   # the next 2n-block repeats it


def test_eval_mod_is_sine(boot):
    o, u, f = boot["o"], boot["u"], boot["f"]
    uu = o.decrypt(u, 2 * N_BLOCK)
    assert f.level == u.level - 14
    assert np.max(np.abs(o.decrypt(f, 2 * N_BLOCK) - np.sin(2 * np.pi * uu))) < 2.0 ** -30


def test_bootstrap_returns_periodic_input(boot):
    o, v, z, ct = boot["o"], boot["v"], boot["z"], boot["ct"]
    assert z.level == o.ctx.L - 16 and z.scale == ct.scale
    zd = o.decrypt(z, o.n // 2)
    assert np.max(np.abs(zd - np.tile(v, (o.n // 2) // N_BLOCK))) < TOL_BOOT
