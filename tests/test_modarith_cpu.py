"""The library's 64-bit modular arithmetic (csrc/modarith.cuh), compiled for
the host and checked against big-integer definitions, no GPU involved:

* Shoup's product by a fixed w (w' = floor(w 2^64 / q)) is x w mod q for
  every 64-bit x, and its lazy form is congruent and below 2q;
* Montgomery reduction of hi:lo < q 2^64 is hi:lo 2^-64 mod q, and a product
  through two reductions (with 2^128 mod q) is a b mod q;
* the 128-bit multiply-accumulate is the exact sum mod 2^128, and 15
  products of residues by values below q (the dot products of the base
  conversion) stay below q 2^64, so one reduction suffices;
* reduction by floor(2^64 / q) is x mod q;
* the lazy butterfly ranges of the transforms: forward values in [0, 4q),
  inverse in [0, 2q), stay within the word for the 60-bit primes (64-bit
  words) and the primes below 2^30 of the 32-bit word-size probe.

Inputs are the real prime chains of the argmax8 set (60- and 50-bit) and
the 32-bit probe set, at the extremes of each range and at random.  The
device build replaces the 128-bit host product by a 32-bit carry chain;
its results are checked bit for bit against the oracle by the GPU tests."""
import os
import random
import shutil
import subprocess

import pytest

from oracle.params import ARGMAX8, WORD32, select_primes

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2502_00847_gb300", "csrc")
M64 = (1 << 64) - 1

HARNESS = r"""
#include <cstdio>
#include <cstring>
#include "modarith.cuh"
int main() {
    char op[4];
    while (std::scanf("%3s", op) == 1) {
        unsigned long long a, b, c, d, e, f;
        if (!std::strcmp(op, "S")) {            // x w wp q
            std::scanf("%llu %llu %llu %llu", &a, &b, &c, &d);
            std::printf("%llu %llu\n", mul_shoup(a, b, c, d), mul_shoup_lazy(a, b, c, d));
        } else if (!std::strcmp(op, "R")) {     // hi lo q qinv_neg
            std::scanf("%llu %llu %llu %llu", &a, &b, &c, &d);
            std::printf("%llu\n", redc(a, b, c, d));
        } else if (!std::strcmp(op, "M")) {     // a b q qinv_neg r2
            std::scanf("%llu %llu %llu %llu %llu", &a, &b, &c, &d, &e);
            std::printf("%llu %llu\n", mont_mul(a, b, c, d), mul_mod(a, b, c, d, e));
        } else if (!std::strcmp(op, "B")) {     // x q mu
            std::scanf("%llu %llu %llu", &a, &b, &c);
            std::printf("%llu\n", reduce64(a, b, c));
        } else if (!std::strcmp(op, "A")) {     // count, then count pairs
            std::scanf("%llu", &f);
            acc128 acc = {0, 0};
            for (unsigned long long i = 0; i < f; ++i) {
                std::scanf("%llu %llu", &a, &b);
                mac(acc, a, b);
            }
            std::printf("%llu %llu\n", acc.hi, acc.lo);
        } else {
            return 2;
        }
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("modarith")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             check=True).stdout.split("\n")
        return [[int(t) for t in ln.split()] for ln in out if ln.strip()]
    return run


def _primes():
    qs, sp = select_primes(ARGMAX8)
    qs32, sp32 = select_primes(WORD32)
    return sorted(set(qs + sp)), sorted(set(qs32 + sp32))


def _mont(q):
    return (-pow(q, -1, 1 << 64)) % (1 << 64), pow(2, 128, q)


def test_shoup_product_every_64_bit_input(harness):
    ps, _ = _primes()
    rng = random.Random(1)
    cases = []
    for q in ps:
        for w in (0, 1, q - 1, q // 2, rng.randrange(q)):
            wp = (w << 64) // q
            for x in (0, 1, q - 1, q, 2 * q - 1, 4 * q - 1, M64, M64 - q, rng.randrange(1 << 64)):
                cases.append((x, w, wp, q))
    got = harness(["S %d %d %d %d" % c for c in cases])
    for (x, w, wp, q), (full, lazy) in zip(cases, got):
        assert full == x * w % q, (x, w, q)
        assert lazy < 2 * q and lazy % q == full, (x, w, q)
        # the lazy value is exactly x w - floor(x w' / 2^64) q, taken mod 2^64
        assert lazy == (x * w - ((x * wp) >> 64) * q) & M64


def test_montgomery_reduction_and_products(harness):
    ps, _ = _primes()
    rng = random.Random(2)
    red, prod = [], []
    for q in ps:
        qinv, r2 = _mont(q)
        top = q * (1 << 64) - 1                      # largest admissible hi:lo
        for t in (0, 1, q, (1 << 64) - 1, 1 << 64, top, rng.randrange(top), rng.randrange(1 << 64)):
            red.append((t >> 64, t & M64, q, qinv))
        for a, b in ((0, 0), (q - 1, q - 1), (1, q - 1), (rng.randrange(q), rng.randrange(q))):
            prod.append((a, b, q, qinv, r2))
    got = harness(["R %d %d %d %d" % c for c in red])
    for (hi, lo, q, _), (r,) in zip(red, got):
        assert r == ((hi << 64) | lo) * pow(2, -64, q) % q, (hi, lo, q)
    got = harness(["M %d %d %d %d %d" % c for c in prod])
    for (a, b, q, _, _), (mm, m) in zip(prod, got):
        assert mm == a * b * pow(2, -64, q) % q and m == a * b % q, (a, b, q)


def test_multiply_accumulate_and_dot_product_bound(harness):
    ps, _ = _primes()
    rng = random.Random(3)
    lines, want = [], []
    for n in (1, 2, 15, 40):
        pairs = [(M64, M64)] * n if n == 40 else [(rng.randrange(1 << 64), rng.randrange(1 << 64)) for _ in range(n)]
        lines.append("A %d " % n + " ".join("%d %d" % p for p in pairs))
        want.append(sum(a * b for a, b in pairs) % (1 << 128))
    got = harness(lines)
    for (hi, lo), w in zip(got, want):
        assert (hi << 64) | lo == w
    # 15 products of residues (< 2^60) by values below q stay below q 2^64
    for q in ps:
        assert 15 * ((1 << 60) - 1) * (q - 1) < q << 64


def test_reduce64(harness):
    ps, _ = _primes()
    rng = random.Random(4)
    cases = [(x, q, (1 << 64) // q) for q in ps for x in (0, q - 1, q, M64, rng.randrange(1 << 64))]
    got = harness(["B %d %d %d" % c for c in cases])
    for (x, q, _), (r,) in zip(cases, got):
        assert r == x % q


def _butterfly_ranges(q, word, rng, rounds=2000):
    """Forward (Cooley-Tukey, values in [0, 4q)) and inverse
    (Gentleman-Sande, values in [0, 2q)) lazy butterflies with Shoup products
    in the given word size: every intermediate stays in its range and below
    2^word, and the outputs are congruent to the exact butterfly."""
    m = (1 << word) - 1
    for _ in range(rounds):
        w = rng.randrange(q)
        wp = (w << word) // q
        shoup = lambda x: (x * w - ((x * wp) >> word) * q) & m  # noqa: E731
        x, y = rng.randrange(4 * q), rng.randrange(4 * q)
        u = x - 2 * q if x >= 2 * q else x
        t = shoup(y)
        assert t < 2 * q
        a, b = u + t, u - t + 2 * q
        assert a < 4 * q and 0 < b < 4 * q and 4 * q <= m + 1
        assert (a - x - w * y) % q == 0 and (b - x + w * y) % q == 0
        x, y = rng.randrange(2 * q), rng.randrange(2 * q)
        s = x + y
        s = s - 2 * q if s >= 2 * q else s
        d = shoup(x - y + 2 * q)
        assert s < 2 * q and d < 2 * q
        assert (s - x - y) % q == 0 and (d - (x - y) * w) % q == 0


def test_lazy_butterfly_ranges_both_word_sizes():
    ps, ps32 = _primes()
    rng = random.Random(5)
    for q in (min(ps), max(ps)):
        _butterfly_ranges(q, 64, rng)
    assert max(ps32) < 1 << 30
    for q in (min(ps32), max(ps32)):
        _butterfly_ranges(q, 32, rng)
