"""Named parameter sets of the library (numbers only; each side of the
build selects its primes from them independently: the library in
csrc/hostmath.cpp, the oracle in its own code).

Field names are those of secpe_params in include/secpe.h.  RNS-CKKS over
R_Q = Z_Q[X]/(X^N + 1) (SecPE Sec. 2.2); 128-bit security at N = 2^16 allows
log2(QP) <= 1763 (Sec. 4.1).

* toy:     N = 2^12, 12 x 40-bit primes + one 60-bit special prime, dnum = 12,
           Delta = 2^40 (non-secure test parameters);
* micro:   N = 2^16, 24 x ~50-bit + 4 x 60-bit special primes, dnum = 3,
           Delta = 2^50 (primitive micro-benchmark; timing only);
* argmax:  N = 2^16, a 60-bit q_0 + 23 x ~50-bit, 4 special, dnum = 6;
* argmax8: the same ciphertext primes, 8 special, dnum = 3
           (log2(QP) = 1690), the Argmax benchmark's default.
"""
from dataclasses import dataclass


@dataclass(frozen=True)
class ParamSet:
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
    secret_hw: int = 0
    boot_primes: int = 0
    boot_bits: int = 0


TOY = ParamSet(log_n=12, q0_bits=40, q_bits=40, n_q=12, p_bits=60, n_p=1, dnum=12, log_scale=40)
MICRO = ParamSet(log_n=16, q0_bits=50, q_bits=50, n_q=24, p_bits=60, n_p=4, dnum=3, log_scale=50)
ARGMAX = ParamSet(log_n=16, q0_bits=60, q_bits=50, n_q=24, p_bits=60, n_p=4, dnum=6, log_scale=50)
ARGMAX8 = ParamSet(log_n=16, q0_bits=60, q_bits=50, n_q=24, p_bits=60, n_p=8, dnum=3, log_scale=50)
# Bootstrapping sets: q0 50-bit, 40-bit computation primes (Delta = 2^40),
# the top 16 primes 60-bit for the bootstrapping levels, sparse secret of
# weight 32 (boot_toy N = 2^12, boot16 N = 2^16).
BOOT_TOY = ParamSet(log_n=12, q0_bits=50, q_bits=40, n_q=24, p_bits=60, n_p=4, dnum=8, log_scale=40,
                    secret_hw=32, boot_primes=16, boot_bits=60)
BOOT16 = ParamSet(log_n=16, q0_bits=50, q_bits=40, n_q=27, p_bits=60, n_p=5, dnum=7, log_scale=40,
                  secret_hw=32, boot_primes=16, boot_bits=60)
# The word-size probe's prime chain: 48 + 8 primes of about 29 bits (below
# 2^30), for the 32-bit transform and base conversion only.
WORD32 = ParamSet(log_n=16, q0_bits=29, q_bits=29, n_q=48, p_bits=29, n_p=8, dnum=4, log_scale=58)
PRESETS = {"toy": TOY, "micro": MICRO, "argmax": ARGMAX, "argmax8": ARGMAX8, "boot_toy": BOOT_TOY,
           "boot16": BOOT16, "word32": WORD32}
