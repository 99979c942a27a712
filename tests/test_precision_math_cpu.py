"""Exactness of the precision variant's arithmetic, checked on the CPU
against definitions (no GPU, no library code):

* the four-step factorisation that the tensor-pipe transform uses (a fixed
  matrix on every column, an element-wise twist, a fixed matrix on every
  row, and the inverse in reverse order) equals the negacyclic transform of
  the ring R_Q (Sec. 2.2), out[j] = sum_k a[k] psi^((2 brv(j) + 1) k), here
  at N = 2^8 (16 x 16; the library uses 256 x 256, the algebra is the same);
* the key inner product's 8-bit-limb GEMM, with the m16n8k32 u8 fragment
  layout and the Toeplitz band of key bytes, reproduces sum_j x_j k_j mod p
  for 1..8 digits and ragged item counts, every s32 partial staying below
  2^31.
"""
import random

import pytest


def brv(x, bits):
    return int(format(x, "0%db" % bits)[::-1], 2)


def _prime_and_psi(n):
    q = (1 << 30) // (2 * n) * (2 * n) + 1
    while any(q % p == 0 for p in range(2, int(q ** 0.5) + 1)):
        q += 2 * n
    for x in range(2, q):
        psi = pow(x, (q - 1) // (2 * n), q)
        if pow(psi, n, q) == q - 1:
            return q, psi


def test_four_step_factorisation_equals_negacyclic_definition():
    h = 4
    R = 1 << h
    N = R * R
    q, psi = _prime_and_psi(N)
    rng = random.Random(5)
    a = [rng.randrange(q) for _ in range(N)]
    ref = [sum(a[k] * pow(psi, (2 * brv(j, 2 * h) + 1) * k, q) for k in range(N)) % q for j in range(N)]
    # forward: columns (W), twist, rows (F)
    W = [[pow(psi, R * (2 * brv(r, h) + 1) * k2, q) for k2 in range(R)] for r in range(R)]
    v = [[sum(W[r][k2] * a[c + R * k2] for k2 in range(R)) % q for c in range(R)] for r in range(R)]
    v = [[v[r][c] * pow(psi, (2 * brv(r, h) + 1) * c, q) % q for c in range(R)] for r in range(R)]
    om = pow(psi, 2 * R, q)
    F = [[pow(om, brv(t, h) * c, q) for c in range(R)] for t in range(R)]
    out = [sum(F[t][c] * v[r][c] for c in range(R)) % q for r in range(R) for t in range(R)]
    assert out == ref
    # inverse: rows (F*), inverse twist, columns (W^-1 with the remaining 1/R)
    psi_i, om_i, n_inv = pow(psi, q - 2, q), pow(om, q - 2, q), pow(N, q - 2, q)
    z = [[sum(pow(om_i, brv(t, h) * c, q) * ref[R * r + t] for t in range(R)) % q for c in range(R)]
         for r in range(R)]
    z = [[z[r][c] * pow(psi_i, (2 * brv(r, h) + 1) * c, q) % q for c in range(R)] for r in range(R)]
    back = [0] * N
    for c in range(R):
        for k2 in range(R):
            # W^-1[k2][r] = R^-1 psi^-(R (2 brv(r) + 1) k2); the row part carried no 1/R
            back[c + R * k2] = sum(pow(psi_i, R * (2 * brv(r, h) + 1) * k2, q) * z[r][c] for r in range(R)) \
                * n_inv % q
    assert back == a
    # a dropped twist or a transposed row matrix is detected
    F_t = [[F[c][t] for c in range(R)] for t in range(R)]
    bad = [sum(F_t[t][c] * v[r][c] for c in range(R)) % q for r in range(R) for t in range(R)]
    assert bad != ref


def _band4(k, u):
    sh = 8 * (u - 3)
    w = 0 if sh >= 64 else ((k >> sh) if sh >= 0 else (k << -sh)) & ((1 << 64) - 1)
    w &= 0xFFFFFFFF
    b = [(w >> (8 * i)) & 255 for i in range(4)]
    return [b[3 - i] for i in range(4)]  # byte permutation 0x0123


def _ip_by_fragments(key, x, nkc, p):
    """Per-lane m16n8k32 fragments as the kernel builds them; returns
    {(item, s): result} and the largest s32 partial."""
    ndig, nitem = len(key), len(x)
    out, biggest = {}, 0
    for ig in range((nitem + 7) // 8):
        S = {lane: [[0] * 4, [0] * 4] for lane in range(32)}
        for kc in range(nkc):
            for s in range(2):
                A = [[0] * 32 for _ in range(16)]
                B = [[0] * 8 for _ in range(32)]
                for lane in range(32):
                    g, tq = lane >> 2, lane & 3
                    a0 = 4 * (tq & 1)
                    jl, jh = 4 * kc + (tq >> 1), 4 * kc + 2 + (tq >> 1)
                    kl = key[jl][s] if jl < ndig else 0
                    kh = key[jh][s] if jh < ndig else 0
                    regs = [_band4(kl, g - a0), _band4(kl, g + 8 - a0), _band4(kh, g - a0), _band4(kh, g + 8 - a0)]
                    for i in range(4):
                        A[g][4 * tq + i], A[g + 8][4 * tq + i] = regs[0][i], regs[1][i]
                        A[g][16 + 4 * tq + i], A[g + 8][16 + 4 * tq + i] = regs[2][i], regs[3][i]
                    item = ig * 8 + g

                    def xv(j):
                        return x[item][j] if j < ndig and item < nitem else 0
                    b0 = (xv(jl) >> 32) if tq & 1 else xv(jl) & 0xFFFFFFFF
                    b1 = (xv(jh) >> 32) if tq & 1 else xv(jh) & 0xFFFFFFFF
                    for i in range(4):
                        B[4 * tq + i][g] = (b0 >> (8 * i)) & 255
                        B[16 + 4 * tq + i][g] = (b1 >> (8 * i)) & 255
                C = [[sum(A[r][k] * B[k][c] for k in range(32)) for c in range(8)] for r in range(16)]
                for lane in range(32):
                    g, tq = lane >> 2, lane & 3
                    S[lane][s][0] += C[g][2 * tq]
                    S[lane][s][1] += C[g][2 * tq + 1]
                    S[lane][s][2] += C[g + 8][2 * tq]
                    S[lane][s][3] += C[g + 8][2 * tq + 1]
        cp = [pow(2, 8 * d, p) if d < 15 else 0 for d in range(16)]
        for lane in range(32):
            biggest = max(biggest, *S[lane][0], *S[lane][1])
        for tq in range(4):
            for s in range(2):
                for ip in range(2):
                    tot = sum(S[4 * g + tq][s][ip] * cp[g] + S[4 * g + tq][s][2 + ip] * cp[g + 8] for g in range(8))
                    item = ig * 8 + 2 * tq + ip
                    if item < nitem:
                        out[(item, s)] = tot % p
    return out, biggest


@pytest.mark.parametrize("ndig,nitem", [(1, 3), (3, 9), (4, 8), (6, 2), (8, 5)])
def test_key_inner_product_fragments_reproduce_dot_product(ndig, nitem):
    rng = random.Random(ndig * 100 + nitem)
    p = (1 << 60) - 93  # any modulus below 2^60 (the arithmetic identity does not need a prime)
    key = [[rng.randrange(p) for _ in range(2)] for _ in range(ndig)]
    x = [[rng.randrange(p) for _ in range(ndig)] for _ in range(nitem)]
    key[0][0] = p - 1  # extremes
    x[0][0] = p - 1
    out, biggest = _ip_by_fragments(key, x, 1 if ndig <= 4 else 2, p)
    assert biggest < 2 ** 31
    for b in range(nitem):
        for s in range(2):
            assert out[(b, s)] == sum(x[b][j] * key[j][s] for j in range(ndig)) % p
