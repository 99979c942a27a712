"""RNS-CKKS parameter sets and prime/root selection for the oracle.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.

SecPE (Sec. 2.2) works in R_Q = Z_Q[X]/(X^N+1) with Q a product of distinct
primes, and uses N = 2^16 on SEAL (Sec. 4.1).  The paper does not say how the
primes are chosen; the reading implemented here (and, independently, in the
CUDA library) is:

* every prime is = 1 (mod 2N), so that the negacyclic NTT exists;
* the special primes are the n_p largest such primes below 2^p_bits;
* if q0 has its own bit size, it is the largest such prime below 2^q0_bits
  not already taken; otherwise it is the first of the sequence below;
* the remaining ciphertext primes alternate between the nearest such primes
  below and above 2^q_bits (below first), skipping primes already taken, so
  that the running product stays close to a power of the scale;
* psi_q, the primitive 2N-th root used by the NTT, is x^((q-1)/2N) for the
  smallest integer x >= 2 for which that power satisfies psi^N = -1 (mod q).
"""
from dataclasses import dataclass, field

# Deterministic Miller-Rabin bases, sufficient for every n < 3.3e24.
_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n):
    """Miller-Rabin with a fixed base set (deterministic below 3.3e24)."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x == 1 or x == n - 1:
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def primes_below(bound, m, count, taken=()):
    """The `count` largest primes p < bound with p = 1 (mod m), not in taken."""
    out = []
    k = (bound - 2) // m
    while len(out) < count:
        c = k * m + 1
        if c < 2:
            raise ValueError("ran out of primes")
        if c < bound and c not in taken and is_prime(c):
            out.append(c)
        k -= 1
    return out


def primes_above(bound, m, count, taken=()):
    """The `count` smallest primes p > bound with p = 1 (mod m), not in taken."""
    out = []
    k = bound // m + 1
    while len(out) < count:
        c = k * m + 1
        if c > bound and c not in taken and is_prime(c):
            out.append(c)
        k += 1
    return out


def find_psi(q, n):
    """Smallest-base primitive 2n-th root of unity mod q (see module doc)."""
    two_n = 2 * n
    assert (q - 1) % two_n == 0
    e = (q - 1) // two_n
    x = 2
    while True:
        psi = pow(x, e, q)
        if pow(psi, n, q) == q - 1:
            return psi
        x += 1


@dataclass(frozen=True)
class Params:
    """One RNS-CKKS parameter set.

    n_q ciphertext primes q_0..q_L (L = n_q - 1 levels), n_p special primes
    for hybrid key switching with dnum digits of alpha = ceil(n_q/dnum)
    primes, scale 2^log_scale, Sign = f^df(g^dg(x)) (SecPE Eq. comp).
    `reserve` levels are kept below every polynomial block (C-9 reading).
    """
    log_n: int
    q0_bits: int
    q_bits: int
    n_q: int
    p_bits: int
    n_p: int
    dnum: int
    log_scale: int
    sign_dg: int = 2
    sign_df: int = 2
    reserve: int = 1
    secret_hw: int = 0   # 0: uniform ternary secret; h > 0: exactly h nonzero coefficients
    boot_primes: int = 0  # top ciphertext primes of boot_bits bits for bootstrapping's levels
    boot_bits: int = 0

    @property
    def n(self):
        return 1 << self.log_n

    @property
    def slots(self):
        return self.n // 2

    @property
    def alpha(self):
        return -(-self.n_q // self.dnum)

    @property
    def max_level(self):
        return self.n_q - 1

    @property
    def scale(self):
        return float(2 ** self.log_scale)


def select_primes(p):
    """Ciphertext primes (q_0 first) and special primes for a Params.  With
    boot_primes = b > 0 the top b ciphertext primes are the b largest below
    2^boot_bits (taken after the special primes, before q_0), in decreasing
    order, above the q_bits-sized ones."""
    m = 2 * p.n
    special = primes_below(1 << p.p_bits, m, p.n_p)
    taken = set(special)
    boot = primes_below(1 << p.boot_bits, m, p.boot_primes, taken) if p.boot_primes else []
    taken.update(boot)
    qs = []
    if p.q0_bits != p.q_bits:
        q0 = primes_below(1 << p.q0_bits, m, 1, taken)[0]
        qs.append(q0)
        taken.add(q0)
    need = p.n_q - p.boot_primes - len(qs)
    # alternate below / above 2^q_bits; enough candidates of each kind
    below = primes_below(1 << p.q_bits, m, need, taken)
    above = primes_above(1 << p.q_bits, m, need, taken)
    seq = []
    for b, a in zip(below, above):
        seq.append(b)
        seq.append(a)
    qs.extend(seq[:need])
    qs.extend(boot)
    return qs, special


# Named presets.  TOY: N=2^12, 12 x 40-bit primes + one 60-bit special prime
# (non-secure test parameters).  MICRO: N=2^16, 24 x ~50-bit + 4 special,
# dnum=3 (timing only: with alpha=8 the digit modulus exceeds P, so key
# switching noise is too large to decrypt).  ARGMAX: N=2^16, a 60-bit q0 +
# 23 x ~50-bit primes, 4 special, dnum=6 (alpha=4 <= n_p, P > each digit).
TOY = Params(log_n=12, q0_bits=40, q_bits=40, n_q=12, p_bits=60, n_p=1,
             dnum=12, log_scale=40)
MICRO = Params(log_n=16, q0_bits=50, q_bits=50, n_q=24, p_bits=60, n_p=4,
               dnum=3, log_scale=50)
ARGMAX = Params(log_n=16, q0_bits=60, q_bits=50, n_q=24, p_bits=60, n_p=4,
                dnum=6, log_scale=50)
# ARGMAX8: the same ciphertext primes with 8 special primes and dnum = 3
# (alpha = 8 = n_p, P > every digit; log2(QP) = 1690 <= 1763, the paper's
# 128-bit budget at N = 2^16): half the extended limbs of ARGMAX's ModUp.
ARGMAX8 = Params(log_n=16, q0_bits=60, q_bits=50, n_q=24, p_bits=60, n_p=8,
                 dnum=3, log_scale=50)
# BOOT_TOY / BOOT16: bootstrapping sets.  q0 50-bit, computation primes of
# 40 bits (Delta = 2^40), the top 16 primes 60-bit for bootstrapping's 16
# levels (CoeffToSlot 1, EvalMod 14, SlotToCoeff 1), so its working labels
# (near 2^60) stay at the primes' size; a sparse secret of weight 32 bounds
# the ModRaise overflow by 16.5; 60-bit special primes, n_p > alpha, so that P
# exceeds every digit by a whole prime or more and key switching adds only
# rounding noise to the 2^60-sized labels.  BOOT16 leaves 10 computation
# levels above q0 after a bootstrap (two Sign polynomials of 4 levels plus
# the reserve) within log2 QP = 1715 <= 1763 at N = 2^16: 27 ciphertext
# primes, 5 special, 7 digits of at most 4 primes.
BOOT_TOY = Params(log_n=12, q0_bits=50, q_bits=40, n_q=24, p_bits=60, n_p=4, dnum=8,
                  log_scale=40, secret_hw=32, boot_primes=16, boot_bits=60)
BOOT16 = Params(log_n=16, q0_bits=50, q_bits=40, n_q=27, p_bits=60, n_p=5, dnum=7,
                log_scale=40, secret_hw=32, boot_primes=16, boot_bits=60)
# WORD32: the word-size probe's primes: 48 + 8 primes of about 29 bits
# (below 2^30, so Harvey's lazy butterflies fit 32-bit words), a modulus of
# the size of ARGMAX8's (1392 + 232 bits against 1210 + 480); used for the
# 32-bit transform and base conversion only, not for the circuit.
WORD32 = Params(log_n=16, q0_bits=29, q_bits=29, n_q=48, p_bits=29, n_p=8, dnum=4,
                log_scale=58)
PRESETS = {"toy": TOY, "micro": MICRO, "argmax": ARGMAX, "argmax8": ARGMAX8, "boot_toy": BOOT_TOY,
           "boot16": BOOT16, "word32": WORD32}


class Context:
    """Primes, roots and digit layout for one Params."""

    def __init__(self, params):
        self.p = params
        self.n = params.n
        self.log_n = params.log_n
        self.q, self.special = select_primes(params)
        self.all_primes = self.q + self.special       # prime index order
        self.psi = [find_psi(x, self.n) for x in self.all_primes]
        self.P = 1
        for x in self.special:
            self.P *= x
        self.L = params.max_level

    def digits(self, level):
        """Digit j at `level`: prime indices {j*alpha, ..} cut at `level`."""
        a = self.p.alpha
        out = []
        j = 0
        while j * a <= level:
            out.append(list(range(j * a, min((j + 1) * a, level + 1))))
            j += 1
        return out

    def special_idx(self):
        return list(range(len(self.q), len(self.all_primes)))
