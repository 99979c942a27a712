"""Pins of the oracle's ring layer against definitions that do not depend on
it: primality by independent means, the NTT against the direct evaluation of
its definition, the convolution theorem against the schoolbook negacyclic
product, basis conversion and the automorphism against big-integer
definitions, and the SplitMix64 sampler against its published outputs."""
import numpy as np
import pytest

from oracle import _lib
from oracle.params import (Context, Params, TOY, ARGMAX, MICRO, find_psi, is_prime,
                           primes_above, primes_below)

L = _lib.lib()
ptr = _lib.ptr


def _trial_division_prime(n):
    if n < 2:
        return False
    d = 2
    while d * d <= n:
        if n % d == 0:
            return False
        d += 1
    return True


def test_is_prime_small_matches_trial_division():
    for n in range(0, 5000):
        assert is_prime(n) == _trial_division_prime(n), n


def test_is_prime_matches_sympy():
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(3)
    for _ in range(300):
        n = int(rng.integers(2**40, 2**62))
        assert is_prime(n) == bool(sympy.isprime(n)), n
    # strong pseudoprimes to several bases
    for n in (3215031751, 2152302898747, 3474749660383, 341550071728321):
        assert not is_prime(n)


@pytest.mark.parametrize("params", [TOY, MICRO, ARGMAX], ids=["toy", "micro", "argmax"])
def test_prime_selection_rule(params):
    ctx = Context(params)
    m = 2 * params.n
    allp = ctx.q + ctx.special
    assert len(set(allp)) == len(allp)
    assert len(ctx.q) == params.n_q and len(ctx.special) == params.n_p
    for p in allp:
        assert p % m == 1 and is_prime(p)
        assert p < 2**60 or params.q_bits < 60  # every prime stays below 2^60
    # special primes: no prime = 1 mod 2N between the smallest special prime
    # and 2^p_bits is skipped
    lo = min(ctx.special)
    k = lo // m + 1
    count = 0
    while k * m + 1 < 2**params.p_bits:
        if is_prime(k * m + 1):
            count += 1
        k += 1
    assert count == params.n_p - 1
    # alternating nearest primes around 2^q_bits
    rest = ctx.q[1:] if params.q0_bits != params.q_bits else ctx.q
    below = [p for p in rest if p < 2**params.q_bits]
    above = [p for p in rest if p > 2**params.q_bits]
    assert abs(len(below) - len(above)) <= 1
    assert below == sorted(below, reverse=True)
    assert above == sorted(above)
    # nothing skipped between 2^b and the extreme picks
    if below:
        k = min(below) // m + 1
        n_between = sum(1 for kk in range(k, (2**params.q_bits) // m + 1)
                        if kk * m + 1 < 2**params.q_bits and is_prime(kk * m + 1)
                        and kk * m + 1 not in allp)
        assert n_between == 0
    if above:
        n_between = sum(1 for kk in range((2**params.q_bits) // m + 1, max(above) // m)
                        if is_prime(kk * m + 1) and kk * m + 1 not in allp)
        assert n_between == 0


def test_psi_is_primitive_and_smallest():
    for params in (TOY, ARGMAX):
        ctx = Context(params)
        n = params.n
        for q, psi in zip(ctx.all_primes, ctx.psi):
            assert pow(psi, n, q) == q - 1
            assert pow(psi, 2 * n, q) == 1
            e = (q - 1) // (2 * n)
            x = 2
            while pow(x, e, q) != psi:
                assert pow(pow(x, e, q), n, q) != q - 1
                x += 1


def _rand_limb(rng, n, q):
    return rng.integers(0, q, n, dtype=np.uint64)


@pytest.mark.parametrize("logn", [1, 2, 3, 5, 8, 10])
def test_ntt_matches_definition(logn):
    n = 1 << logn
    rng = np.random.default_rng(logn)
    for bits in (30, 50, 60):
        q = primes_below(2**bits, 2 * n, 1)[0]
        psi = find_psi(q, n)
        a = _rand_limb(rng, n, q)
        ref = np.empty(n, dtype=np.uint64)
        L.or_ntt_naive(ptr(a), ptr(ref), logn, q, psi)
        b = a.copy()
        L.or_ntt_fwd(ptr(b), logn, q, psi)
        assert np.array_equal(b, ref)
        L.or_ntt_inv(ptr(b), logn, q, psi)
        assert np.array_equal(b, a)


def test_ntt_definition_is_evaluation_at_odd_powers():
    # brute force with Python ints: out[j] = a(psi^(2 brv(j) + 1))
    logn, n = 4, 16
    q = primes_below(2**20, 2 * n, 1)[0]
    psi = find_psi(q, n)
    a = np.arange(1, n + 1, dtype=np.uint64) * 7919 % q
    out = np.empty(n, dtype=np.uint64)
    L.or_ntt_naive(ptr(a), ptr(out), logn, q, psi)
    for j in range(n):
        brv = int(format(j, "04b")[::-1], 2)
        x = pow(psi, 2 * brv + 1, q)
        assert int(out[j]) == sum(int(a[k]) * pow(x, k, q) for k in range(n)) % q


@pytest.mark.parametrize("logn", [2, 4, 6, 8])
def test_convolution_theorem(logn):
    n = 1 << logn
    rng = np.random.default_rng(100 + logn)
    q = primes_below(2**50, 2 * n, 1)[0]
    psi = find_psi(q, n)
    a, b = _rand_limb(rng, n, q), _rand_limb(rng, n, q)
    ref = np.empty(n, dtype=np.uint64)
    L.or_negacyclic_naive(ptr(a), ptr(b), ptr(ref), logn, q)
    # Python big-int schoolbook as a second, independent reference
    pyref = [0] * n
    for i in range(n):
        for k in range(n):
            v = int(a[i]) * int(b[k])
            if i + k < n:
                pyref[i + k] += v
            else:
                pyref[i + k - n] -= v
    assert [x % q for x in pyref] == [int(x) for x in ref]
    fa, fb = a.copy(), b.copy()
    L.or_ntt_fwd(ptr(fa), logn, q, psi)
    L.or_ntt_fwd(ptr(fb), logn, q, psi)
    prod = np.empty(n, dtype=np.uint64)
    L.or_vmul(ptr(fa), ptr(fb), ptr(prod), n, q)
    L.or_ntt_inv(ptr(prod), logn, q, psi)
    assert np.array_equal(prod, ref)


def test_from_signed_and_vector_ops():
    q = primes_below(2**59, 2**13, 1)[0]
    vals = np.array([0, 1, -1, 2**62, -2**62, -2**63, 2**63 - 1, 12345, -q], dtype=np.int64)
    out = np.empty(len(vals), dtype=np.uint64)
    L.or_vfrom_signed(ptr(vals), ptr(out), len(vals), q)
    assert [int(x) for x in out] == [int(v) % q for v in vals]
    rng = np.random.default_rng(5)
    a, b = _rand_limb(rng, 64, q), _rand_limb(rng, 64, q)
    r = np.empty(64, dtype=np.uint64)
    for fn, op in ((L.or_vmul, lambda x, y: x * y), (L.or_vadd, lambda x, y: x + y),
                   (L.or_vsub, lambda x, y: x - y)):
        fn(ptr(a), ptr(b), ptr(r), 64, q)
        assert [int(x) for x in r] == [op(int(x), int(y)) % q for x, y in zip(a, b)]


def test_fast_bconv_definition_and_error_bound():
    rng = np.random.default_rng(7)
    n = 32
    src = primes_below(2**50, 64, 4)
    dst = primes_below(2**60, 64, 3)
    Q = 1
    for q in src:
        Q *= q
    xs = [int(rng.integers(0, 2**62)) * int(rng.integers(0, 2**62)) * int(rng.integers(0, 2**60)) % Q
          for _ in range(n)]
    x = np.array([[v % q for v in xs] for q in src], dtype=np.uint64)
    out = np.empty((len(dst), n), dtype=np.uint64)
    L.or_fast_bconv(ptr(x), ptr(_lib.u64arr(src)), len(src), ptr(_lib.u64arr(dst)), len(dst),
                    ptr(out), n)
    for c in range(n):
        # big-integer definition
        s = 0
        for i, q in enumerate(src):
            qhat = Q // q
            s += (xs[c] % q) * pow(qhat % q, -1, q) % q * qhat
        # FastBConv = x + u*Q with 0 <= u < len(src)
        u = (s - xs[c]) // Q
        assert (s - xs[c]) % Q == 0 and 0 <= u < len(src)
        for t, p in enumerate(dst):
            assert int(out[t, c]) == s % p


def test_automorphism_on_monomials_and_composition():
    logn, n = 5, 32
    q = primes_below(2**40, 2 * n, 1)[0]
    for g in (5, 25, 2 * n - 1, 3):
        for k in range(n):
            a = np.zeros(n, dtype=np.uint64)
            a[k] = 1
            out = np.empty(n, dtype=np.uint64)
            L.or_automorph_coeff(ptr(a), ptr(out), logn, q, g)
            e = k * g % (2 * n)
            exp = np.zeros(n, dtype=np.uint64)
            if e < n:
                exp[e] = 1
            else:
                exp[e - n] = q - 1
            assert np.array_equal(out, exp)
    rng = np.random.default_rng(9)
    a = _rand_limb(rng, n, q)
    t1, t2, t12 = (np.empty(n, dtype=np.uint64) for _ in range(3))
    L.or_automorph_coeff(ptr(a), ptr(t1), logn, q, 5)
    L.or_automorph_coeff(ptr(t1), ptr(t2), logn, q, 25)
    L.or_automorph_coeff(ptr(a), ptr(t12), logn, q, 125)
    assert np.array_equal(t2, t12)


def test_splitmix64_published_outputs():
    # SplitMix64 seeded with 0 (Vigna's splitmix64.c): first three outputs.
    expected = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(L.or_sm_word(0, c)) for c in range(3)] == expected


def test_samplers_ranges_and_moments():
    n = 1 << 16
    key = int(L.or_sm_stream(42, 1, 0))
    t = np.empty(n, dtype=np.int64)
    L.or_sample_ternary(key, ptr(t), n)
    assert set(np.unique(t)) <= {-1, 0, 1}
    for v in (-1, 0, 1):
        assert abs(np.mean(t == v) - 1 / 3) < 0.01
    e = np.empty(n, dtype=np.int64)
    L.or_sample_cbd21(key, ptr(e), n)
    assert e.min() >= -21 and e.max() <= 21
    assert abs(e.mean()) < 0.05 and abs(e.var() - 10.5) < 0.3
    q = primes_below(2**50, 2**17, 1)[0]
    u = np.empty(n, dtype=np.uint64)
    L.or_sample_uniform(key, 0, q, ptr(u), n)
    assert int(u.max()) < q
    assert abs(float(np.mean(u.astype(np.float64))) / q - 0.5) < 0.01
    # the uniform sample is floor((w1*2^64 + w2) * q / 2^128) of the stream words
    w = [int(L.or_sm_word(key, c)) for c in range(6)]
    for i in range(3):
        assert int(u[i]) == ((w[2 * i] << 64) + w[2 * i + 1]) * q >> 128
