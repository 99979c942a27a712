"""Pins of the oracle's CKKS layer and of the SecPE circuit: encoding against
closed forms, homomorphic ops against plaintext numpy, rescale and ModDown
against big-integer rounded division, the Argmax circuit against the FP64
plaintext simulation and the exact argmax, and the paper's op counts."""
import json
import os

import numpy as np
import pytest

from oracle import Oracle, Params, plainsim
from oracle.ckks import round_half_away

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")
TOL_LINEAR = 2.0 ** -20


def _crt(o, res_list, level):
    """Big-integer CRT of coefficient-form limbs (centred)."""
    qs = o.ctx.q[: level + 1]
    Q = 1
    for q in qs:
        Q *= q
    out = []
    for k in range(o.n):
        acc = 0
        for i, q in enumerate(qs):
            Mi = Q // q
            acc += int(res_list[i][k]) * Mi * pow(Mi % q, -1, q)
        acc %= Q
        out.append(acc - Q if acc > Q // 2 else acc)
    return out, Q


def test_round_half_away():
    assert round_half_away(2.5) == 3 and round_half_away(-2.5) == -3
    assert round_half_away(2.4999) == 2 and round_half_away(-0.5) == -1
    assert round_half_away(float(2**52 + 1)) == 2**52 + 1
    assert round_half_away(float(2**60)) == 2**60


def test_encode_constant_vector_is_constant_polynomial():
    o = Oracle(Params(log_n=6, q0_bits=30, q_bits=30, n_q=3, p_bits=40, n_p=1, dnum=3,
                      log_scale=20))
    m = o.encode_coeffs(np.full(o.n // 2, 0.75), 2.0**20)
    assert int(m[0]) == round(0.75 * 2**20)
    assert all(int(x) == 0 for x in m[1:])


def test_decode_of_monomial_is_root_ordering():
    # slot j of X is zeta^(5^j), zeta = exp(i pi / N): pins the 5^j order
    o = Oracle(Params(log_n=6, q0_bits=30, q_bits=30, n_q=3, p_bits=40, n_p=1, dnum=3,
                      log_scale=20))
    m = np.zeros(o.n, dtype=object)
    m[1] = 1
    got = o.decode_coeffs(m, 1.0, o.n // 2)
    exp = [np.cos(np.pi * pow(5, j, 2 * o.n) / o.n) for j in range(o.n // 2)]
    assert np.allclose(got, exp, atol=1e-12)


def test_encode_decode_roundtrip(toy_oracle):
    o = toy_oracle
    v = np.random.default_rng(2).uniform(-1, 1, 37)
    m = o.encode_coeffs(v, o.p.scale)
    assert np.max(np.abs(o.decode_coeffs(m, o.p.scale, 37) - v)) < 2.0**-30


def test_encrypt_decrypt_and_linear_ops(toy_oracle):
    o = toy_oracle
    rng = np.random.default_rng(3)
    v, w = rng.uniform(-1, 1, 16), rng.uniform(-1, 1, 16)
    a, b = o.encrypt(v, seed=11), o.encrypt(w, seed=12)
    assert np.max(np.abs(o.decrypt(a, 16) - v)) < TOL_LINEAR
    assert np.max(np.abs(o.decrypt(o.add(a, b), 16) - (v + w))) < TOL_LINEAR
    assert np.max(np.abs(o.decrypt(o.sub(a, b), 16) - (v - w))) < TOL_LINEAR
    assert np.max(np.abs(o.decrypt(o.add_const(a, 0.375), 16) - (v + 0.375))) < TOL_LINEAR
    mc = o.mul_const(a, -1.7, o.p.scale, a.level - 1)
    assert mc.level == a.level - 1 and mc.scale == o.p.scale
    assert np.max(np.abs(o.decrypt(mc, 16) - (-1.7 * v))) < TOL_LINEAR
    pr = o.mul(a, b)
    assert pr.level == a.level - 1
    assert np.max(np.abs(o.decrypt(pr, 16) - v * w)) < TOL_LINEAR
    # a linear combination of operands at different levels and scales lands
    # at one level with the declared scale and decrypts to the combination
    lc = o.lincomb([(a, 0.8125), (pr, -2.5)], o.p.scale, pr.level - 1)
    assert lc.level == pr.level - 1 and lc.scale == o.p.scale
    assert np.max(np.abs(o.decrypt(lc, 16) - (0.8125 * v - 2.5 * v * w))) < TOL_LINEAR
    # one term is exactly the constant multiply
    one = o.lincomb([(a, -1.7)], o.p.scale, a.level - 1)
    assert np.array_equal(one.c, mc.c)


def test_rotation_direction(toy_oracle):
    o = toy_oracle
    v = np.random.default_rng(4).uniform(-1, 1, 24)
    full = np.zeros(o.n // 2)
    full[:24] = v
    ct = o.encrypt(v, seed=13)
    for r in (1, 2, 3):
        got = o.decrypt(o.rotate(ct, r), 40)
        assert np.max(np.abs(got - np.roll(full, -r)[:40])) < TOL_LINEAR
    for r in (2, 4, 8):
        got = o.decrypt(o.rotate(ct, -r), 40)
        assert np.max(np.abs(got - np.roll(full, r)[:40])) < TOL_LINEAR
    with pytest.raises(KeyError):
        o.rotate(ct, 5)


def test_hoisted_rotations(toy_oracle):
    """Rotations sharing one ModUp (bootstrapping's baby steps) rotate the
    slots like rotate does, and within the linear tolerance of rotate's
    result; each of them also decrypts to the rotated vector at a lower level."""
    o = toy_oracle
    v = np.random.default_rng(5).uniform(-1, 1, 24)
    full = np.zeros(o.n // 2)
    full[:24] = v
    ct = o.encrypt(v, seed=15)
    outs = o.rotate_hoisted(ct, [1, 2, -2, -4])
    for r, c in zip([1, 2, -2, -4], outs):
        assert c.level == ct.level and c.scale == ct.scale
        got = o.decrypt(c, 40)
        assert np.max(np.abs(got - np.roll(full, -r)[:40])) < TOL_LINEAR
        assert np.max(np.abs(got - o.decrypt(o.rotate(ct, r), 40))) < TOL_LINEAR
    low = o.drop(ct, 3)
    (c,) = o.rotate_hoisted(low, [1])
    assert np.max(np.abs(o.decrypt(c, 40) - np.roll(full, -1)[:40])) < TOL_LINEAR
    with pytest.raises(KeyError):
        o.rotate_hoisted(ct, [5])


def test_rescale_is_rounded_division(toy_oracle):
    o = toy_oracle
    ct = o.encrypt(np.linspace(-1, 1, 8), seed=14)
    lv = ct.level
    r = o.rescale(ct)
    ql = o.primes[lv]
    # the scale is divided by q_l, and a ciphertext at scale Delta q_l keeps its
    # slot values at scale Delta
    assert r.level == lv - 1 and r.scale == ct.scale / ql
    big = o.encrypt(np.linspace(-1, 1, 8), seed=14, scale=o.p.scale * ql)
    rb = o.rescale(big)
    assert rb.scale == big.scale / ql
    assert np.max(np.abs(o.decrypt(rb, 8) - np.linspace(-1, 1, 8))) < TOL_LINEAR
    for k in range(2):
        before = []
        for pi in range(lv + 1):
            x = ct.c[k, pi].copy()
            o.intt(x, pi)
            before.append(x)
        after = []
        for pi in range(lv):
            x = r.c[k, pi].copy()
            o.intt(x, pi)
            after.append(x)
        cb, Qb = _crt(o, before, lv)
        ca, Qa = _crt(o, after, lv - 1)
        for x, y in zip(cb[:64], ca[:64]):
            # floor((x + floor(q/2)) / q) with x taken in [0, Q)
            xn = x % Qb
            assert (xn + ql // 2) // ql % Qa == y % Qa


def test_moddown_is_rounded_division_by_P(toy_oracle):
    o = toy_oracle
    rng = np.random.default_rng(5)
    lv = 3
    tgt = list(range(lv + 1)) + o.ctx.special_idx()
    QP = o.ctx.P
    for pi in range(lv + 1):
        QP *= o.primes[pi]
    xs = [int(rng.integers(0, 2**62)) ** 3 % QP for _ in range(o.n)]
    acc = {}
    for t in tgt:
        limb = np.array([x % o.primes[t] for x in xs], dtype=np.uint64)
        o.ntt(limb, t)
        acc[t] = limb
    out = o.moddown(acc, lv)
    res = []
    for pi in range(lv + 1):
        x = out[pi].copy()
        o.intt(x, pi)
        res.append(x)
    Q = QP // o.ctx.P
    for c in range(0, o.n, 97):
        exp = (xs[c] + o.ctx.P // 2) // o.ctx.P
        # one special prime: FastBConv from P is exact, so the result is the
        # exact rounded quotient mod Q
        assert all(int(res[pi][c]) == exp % o.primes[pi] for pi in range(lv + 1))
        assert exp < Q


def test_keyswitch_noise_small(toy_oracle):
    o = toy_oracle
    v = np.random.default_rng(6).uniform(-1, 1, 8)
    ct = o.encrypt(v, seed=15)
    sq = o.mul(ct, ct)
    assert np.max(np.abs(o.decrypt(sq, 8) - v * v)) < 2.0**-24


def test_refresh_preserves_value(toy_oracle):
    o = toy_oracle
    v = np.random.default_rng(7).uniform(-1, 1, 8)
    ct = o.encrypt(v, seed=16)
    low = o.drop(ct, 2)
    o.qseed, o.ridx = 77, 0
    r = o.refresh(low, 77)
    assert r.level == o.ctx.L and r.scale == low.scale
    assert np.max(np.abs(o.decrypt(r, 8) - o.decrypt(low, 8))) < 2.0**-30
    assert o.ridx == 1


def test_op_counts_match_paper_formula():
    facts = json.load(open(GOLDEN))
    for ex in facts["op_count_examples"]:
        n = ex["n"]
        r = (n - 1).bit_length()
        assert r + 1 == ex["sign_calls"] == ex["rotations"]
    sb = facts["slot_batching"]
    assert sb["slots"] // (2 * sb["input_length"]) == sb["inputs_per_ciphertext"]
    assert Params(log_n=16, q0_bits=60, q_bits=50, n_q=2, p_bits=60, n_p=1, dnum=1,
                  log_scale=50).slots == sb["slots"]


@pytest.mark.parametrize("C,seed", [(2, 1), (3, 2), (33, 3)])
def test_toy_argmax_circuit(C, seed):
    from oracle import TOY
    o = Oracle(TOY)
    cp = 1 << (C - 1).bit_length()
    r = cp.bit_length() - 1
    o.keygen(500 + seed, rot_steps=[-cp] + [1 << i for i in range(r)])
    rng = np.random.default_rng(seed)
    K = 5
    while True:
        logits = rng.uniform(-1, 1, (K, C))
        srt = np.sort(logits.mean(0))
        if srt[-1] - srt[-2] >= 0.05:
            break
    cts = [o.encrypt_logits(logits[i], C, -1.0, seed=1000 + i) for i in range(K)]
    y = o.aggregate(cts, -1.0, 1.0)
    assert y.level == o.ctx.L - 1
    assert np.max(np.abs(o.decrypt(y, C) - logits.sum(0) / (K * 2.0))) < TOL_LINEAR
    o.reset_counters()
    z = o.argmax(y, C, qseed=9)
    assert o.counters["rotations"] == r + 1 and o.counters["signs"] == r + 1
    zd = o.decrypt(z, C)
    zp = plainsim.ensemble_argmax(logits, -1.0, 1.0, o.n // 2)
    assert np.max(np.abs(zd - zp)) < 2.0**-12
    assert int(np.argmax(zd)) == int(np.argmax(logits.mean(0)))
    assert zd.max() > 0.5 and np.sort(zd)[-2] < 0.5


def test_max_keeps_the_scale(toy_oracle):
    """Max folds its 1/2 into Sign's last polynomial: the output scale stays
    the input scale (up to the q_l / Delta drift of one rescale), so QuickMax
    rounds do not inflate it, and the value is Max within the Sign bound."""
    o = toy_oracle
    rng = np.random.default_rng(12)
    v, w = rng.uniform(-0.5, 0.5, 32), rng.uniform(-0.5, 0.5, 32)
    a, y = o.encrypt(v, seed=51), o.encrypt(w, seed=52)
    o.qseed, o.ridx = 5, 0
    m = o.max(a, y)
    assert abs(np.log2(m.scale) - np.log2(o.p.scale)) < 1e-3
    assert np.max(np.abs(o.decrypt(m, 32) - plainsim.vmax(v, w))) < 2.0**-12
    m2 = o.max(o.rotate(m, 1), m)
    assert abs(np.log2(m2.scale) - np.log2(o.p.scale)) < 1e-3


def test_plainsim_argmax_exact_on_margins():
    rng = np.random.default_rng(8)
    for C in (2, 3, 4, 6, 14, 64):
        for _ in range(20):
            y = rng.uniform(-1, 1, C)
            srt = np.sort(y)
            if srt[-1] - srt[-2] < 2e-3 * 2:
                continue
            yp = plainsim.pad_logits(y, C, -1.0) / 2.0
            full = np.zeros(4096)
            full[: len(yp)] = yp
            z = plainsim.argmax_slots(full, C)[:C]
            assert int(np.argmax(z)) == int(np.argmax(y))


def test_moddown_rescale_is_exact_division_definition(toy_oracle):
    """Relinearisation's fused ModDown + rescale against its big-integer
    definition: out = (x + h - FastBConv([x + h]_M)) / M, M = P q_l,
    x = P d + acc (CRT value over Q_l P), FastBConv from the primes of M."""
    o = toy_oracle
    rng = np.random.default_rng(12)
    lv = 4
    P = o.ctx.P
    ql = o.primes[lv]
    M = P * ql
    h = M // 2
    q_idx = list(range(lv + 1))
    tgt = q_idx + o.ctx.special_idx()
    QP = P
    for i in q_idx:
        QP *= o.primes[i]
    d_big = [int(rng.integers(0, 2**62)) ** 2 % (QP // P) for _ in range(o.n)]
    a_big = [int(rng.integers(0, 2**62)) ** 3 % QP for _ in range(o.n)]
    dk = np.empty((lv + 1, o.n), dtype=np.uint64)
    for i in q_idx:
        dk[i] = np.array([v % o.primes[i] for v in d_big], dtype=np.uint64)
        o.ntt(dk[i], i)
    acc = {}
    for t in tgt:
        limb = np.array([v % o.primes[t] for v in a_big], dtype=np.uint64)
        o.ntt(limb, t)
        acc[t] = limb
    out = o.moddown_rescale(acc, dk, lv)
    res = []
    for i in range(lv):
        x = out[i].copy()
        o.intt(x, i)
        res.append(x)
    src = o.ctx.special_idx() + [lv]
    Qo = QP // P // ql
    for c in range(0, o.n, 61):
        x = (P * d_big[c] + a_big[c]) % QP
        conv = 0
        for t in src:
            s = o.primes[t]
            mh = M // s
            conv += ((x + h) % s) * pow(mh % s, -1, s) % s * mh
        assert (x + h - conv) % M == 0
        exact = (x + h - conv) // M
        for i in range(lv):
            assert int(res[i][c]) == exact % o.primes[i]
        assert 0 <= exact < Qo * (P + 1)


def test_lazy_relinearisation_counts(toy_oracle):
    """4 relinearisations per degree-9 polynomial (x^2, x^4, x^5 and the lazily
    relinearised sum of the two giant-step products): 16 per Sign with (2, 2)."""
    o = toy_oracle
    x = o.encrypt(np.linspace(-0.4, 0.4, 8), seed=60)
    o.reset_counters()
    o.qseed, o.ridx = 3, 0
    s = o.sign(x, 0)
    assert o.counters["relins"] == 16 and s.level >= o.p.reserve
    from oracle import plainsim
    ref = plainsim.sign(np.linspace(-0.4, 0.4, 8))
    assert np.max(np.abs(o.decrypt(s, 8) - ref)) < 2.0 ** -12


@pytest.mark.parametrize("C,seed", [(2, 4), (4, 5)])
def test_level_aware_final_sign_keeps_refreshes(C, seed, monkeypatch):
    """Alg. 1's final Sign evaluated at the lowest sufficient levels (each
    polynomial's input dropped to 4 (polynomials left) + reserve), with the
    level plan: the same refresh count as with the greedy levels throughout,
    z at the reserve level, and the same decoded result within the Sign
    tolerance."""
    from oracle import TOY
    o = Oracle(TOY)
    cp = 1 << (C - 1).bit_length()
    r = cp.bit_length() - 1
    o.keygen(700 + seed, rot_steps=[-cp] + [1 << i for i in range(r)])
    rng = np.random.default_rng(seed)
    logits = rng.uniform(-1, 1, (3, C))
    cts = [o.encrypt_logits(logits[i], C, -1.0, seed=2000 + i) for i in range(3)]
    y = o.aggregate(cts, -1.0, 1.0)
    o.reset_counters()
    z = o.argmax(y, C, qseed=9)
    low_refreshes = o.counters["refreshes"]
    assert z.level == o.p.reserve
    zd = o.decrypt(z, C)
    greedy = Oracle.sign
    monkeypatch.setattr(Oracle, "sign", lambda self, x, out_levels, last_factor=1.0, lowest=False:
                        greedy(self, x, out_levels, last_factor, False))
    # greedy levels throughout: no level plan either
    monkeypatch.setattr(Oracle, "level_plan", lambda self, r, entry: [entry])
    o.reset_counters()
    zg = o.argmax(y, C, qseed=9)
    assert o.counters["refreshes"] == low_refreshes
    assert zg.level > z.level
    assert np.max(np.abs(o.decrypt(zg, C) - zd)) < 2.0**-12
