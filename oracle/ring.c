/*
 * Plain CPU oracle for the RNS-CKKS ring arithmetic used by SecPE's encrypted
 * Argmax (SecPE Sec. 2.2: R_Q = Z_Q[X]/(X^N+1), Q = prod q_i).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load this file.  It shares no code
 * with the CUDA library: every routine here is the textbook definition written
 * with unsigned __int128 products and the plain `%` operator, radix-2 loops
 * and no Montgomery/Shoup/Barrett tricks, so that it can be checked by eye.
 *
 * All polynomials are arrays of N = 2^logn residues in [0, q).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef unsigned __int128 u128;

static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 addmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
static u64 submod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + q - b) % q); }

static u64 powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

static u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); } /* q prime */

static u64 bitrev(u64 x, int bits) {
    u64 r = 0;
    for (int i = 0; i < bits; i++) {
        r = (r << 1) | (x & 1);
        x >>= 1;
    }
    return r;
}

u64 or_powmod(u64 a, u64 e, u64 q) { return powmod(a, e, q); }
u64 or_bitrev(u64 x, int bits) { return bitrev(x, bits); }

/* ---------------------------------------------------------------------- */
/* Negacyclic NTT.  Definition: out[j] = sum_k a[k] * psi^((2*brv(j)+1)*k),  */
/* i.e. evaluation of a(X) at the odd powers of a primitive 2N-th root psi,  */
/* stored in bit-reversed order.  The INTT is its exact inverse.              */
/* ---------------------------------------------------------------------- */

/* Direct O(N^2) evaluation of the definition above. */
void or_ntt_naive(const u64 *a, u64 *out, int logn, u64 q, u64 psi) {
    u64 n = 1ull << logn;
    for (u64 j = 0; j < n; j++) {
        u64 e = 2 * bitrev(j, logn) + 1;
        u64 w = powmod(psi, e, q);
        u64 acc = 0, wk = 1;
        for (u64 k = 0; k < n; k++) {
            acc = addmod(acc, mulmod(a[k], wk, q), q);
            wk = mulmod(wk, w, q);
        }
        out[j] = acc;
    }
}

/* Schoolbook product in Z_q[X]/(X^N + 1). */
void or_negacyclic_naive(const u64 *a, const u64 *b, u64 *out, int logn, u64 q) {
    u64 n = 1ull << logn;
    for (u64 i = 0; i < n; i++) out[i] = 0;
    for (u64 i = 0; i < n; i++)
        for (u64 k = 0; k < n; k++) {
            u64 p = mulmod(a[i], b[k], q);
            u64 d = i + k;
            if (d < n) out[d] = addmod(out[d], p, q);
            else out[d - n] = submod(out[d - n], p, q);
        }
}

static u64 *power_table(u64 w, u64 n, u64 q) {
    /* tab[i] = w^i mod q for 0 <= i < n */
    u64 *tab = (u64 *)malloc(sizeof(u64) * n);
    tab[0] = 1 % q;
    for (u64 i = 1; i < n; i++) tab[i] = mulmod(tab[i - 1], w, q);
    return tab;
}

/* Radix-2 Cooley-Tukey, natural order in, bit-reversed order out.  Twiddle  */
/* of the butterfly block starting at group index m+i is psi^brv(m+i).        */
void or_ntt_fwd(u64 *a, int logn, u64 q, u64 psi) {
    u64 n = 1ull << logn;
    u64 *pw = power_table(psi, n, q);
    u64 t = n;
    for (u64 m = 1; m < n; m <<= 1) {
        t >>= 1;
        for (u64 i = 0; i < m; i++) {
            u64 w = pw[bitrev(m + i, logn)];
            u64 j1 = 2 * i * t;
            for (u64 j = j1; j < j1 + t; j++) {
                u64 u = a[j];
                u64 v = mulmod(a[j + t], w, q);
                a[j] = addmod(u, v, q);
                a[j + t] = submod(u, v, q);
            }
        }
    }
    free(pw);
}

/* Radix-2 Gentleman-Sande, bit-reversed order in, natural order out, then  */
/* multiplication by N^{-1}: the exact inverse of or_ntt_fwd.                */
void or_ntt_inv(u64 *a, int logn, u64 q, u64 psi) {
    u64 n = 1ull << logn;
    u64 *pw = power_table(invmod(psi, q), n, q);
    u64 t = 1;
    for (u64 m = n >> 1; m >= 1; m >>= 1) {
        for (u64 i = 0; i < m; i++) {
            u64 w = pw[bitrev(m + i, logn)];
            u64 j1 = 2 * i * t;
            for (u64 j = j1; j < j1 + t; j++) {
                u64 u = a[j];
                u64 v = a[j + t];
                a[j] = addmod(u, v, q);
                a[j + t] = mulmod(submod(u, v, q), w, q);
            }
        }
        t <<= 1;
    }
    u64 ninv = invmod(n % q, q);
    for (u64 j = 0; j < n; j++) a[j] = mulmod(a[j], ninv, q);
    free(pw);
}

/* ---------------------------------------------------------------------- */
/* Coefficient-wise arithmetic mod q.                                        */
/* ---------------------------------------------------------------------- */
void or_vmul(const u64 *a, const u64 *b, u64 *out, u64 n, u64 q) {
    for (u64 i = 0; i < n; i++) out[i] = mulmod(a[i], b[i], q);
}
void or_vadd(const u64 *a, const u64 *b, u64 *out, u64 n, u64 q) {
    for (u64 i = 0; i < n; i++) out[i] = addmod(a[i], b[i], q);
}
void or_vsub(const u64 *a, const u64 *b, u64 *out, u64 n, u64 q) {
    for (u64 i = 0; i < n; i++) out[i] = submod(a[i], b[i], q);
}
void or_vscale(const u64 *a, u64 c, u64 *out, u64 n, u64 q) {
    for (u64 i = 0; i < n; i++) out[i] = mulmod(a[i], c % q, q);
}
void or_vaddc(const u64 *a, u64 c, u64 *out, u64 n, u64 q) {
    for (u64 i = 0; i < n; i++) out[i] = addmod(a[i], c % q, q);
}
/* x mod q for arbitrary 64-bit x. */
void or_vreduce(const u64 *a, u64 *out, u64 n, u64 q) {
    for (u64 i = 0; i < n; i++) out[i] = a[i] % q;
}
/* Signed 64-bit integers to residues mod q. */
void or_vfrom_signed(const int64_t *a, u64 *out, u64 n, u64 q) {
    for (u64 i = 0; i < n; i++) {
        int64_t x = a[i];
        if (x >= 0) out[i] = ((u64)x) % q;
        else out[i] = (q - (((u64)(-(x + 1)) + 1) % q)) % q;
    }
}

/* ---------------------------------------------------------------------- */
/* Fast basis conversion (Bajard et al. / Halevi-Polyakov-Shoup), no       */
/* correction: for x given by residues x_i mod q_i (i in D),                */
/*   conv_t(x) = sum_i [x_i * (Qhat_i)^{-1}]_{q_i} * Qhat_i  mod t,          */
/* with Qhat_i = prod_{j != i} q_j.  in: [nin][n], out: [nout][n].          */
/* ---------------------------------------------------------------------- */
void or_fast_bconv(const u64 *in, const u64 *qin, int nin, const u64 *qout, int nout,
                   u64 *out, u64 n) {
    u64 *inv = (u64 *)malloc(sizeof(u64) * nin);
    u64 *hat = (u64 *)malloc(sizeof(u64) * nin * nout);
    for (int i = 0; i < nin; i++) {
        u64 prod = 1 % qin[i];
        for (int j = 0; j < nin; j++)
            if (j != i) prod = mulmod(prod, qin[j] % qin[i], qin[i]);
        inv[i] = invmod(prod, qin[i]);
        for (int t = 0; t < nout; t++) {
            u64 h = 1 % qout[t];
            for (int j = 0; j < nin; j++)
                if (j != i) h = mulmod(h, qin[j] % qout[t], qout[t]);
            hat[i * nout + t] = h;
        }
    }
    for (u64 c = 0; c < n; c++) {
        for (int t = 0; t < nout; t++) {
            u64 acc = 0;
            for (int i = 0; i < nin; i++) {
                u64 y = mulmod(in[(u64)i * n + c], inv[i], qin[i]);
                acc = addmod(acc, mulmod(y % qout[t], hat[i * nout + t], qout[t]), qout[t]);
            }
            out[(u64)t * n + c] = acc;
        }
    }
    free(inv);
    free(hat);
}

/* ---------------------------------------------------------------------- */
/* Ring automorphism X -> X^g (g odd) on a coefficient-form polynomial:    */
/* X^k maps to X^(k*g mod 2N), with X^N = -1.                              */
/* ---------------------------------------------------------------------- */
void or_automorph_coeff(const u64 *a, u64 *out, int logn, u64 q, u64 g) {
    u64 n = 1ull << logn, two_n = 2 * n;
    for (u64 k = 0; k < n; k++) {
        u64 e = (u64)(((u128)k * g) % two_n);
        if (e < n) out[e] = a[k];
        else out[e - n] = (q - a[k]) % q;
    }
}

/* ---------------------------------------------------------------------- */
/* Counter-based sampling from SplitMix64 (Steele, Lea, Flood, OOPSLA 2014). */
/* A generator with state `key` emits, as its c-th output (c = 0, 1, ...),   */
/* mix64(key + (c+1)*GAMMA), which needs no sequential state.                */
/* ---------------------------------------------------------------------- */
#define SM_GAMMA 0x9E3779B97F4A7C15ull
static u64 mix64(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
u64 or_sm_word(u64 key, u64 c) { return mix64(key + (c + 1) * SM_GAMMA); }
/* Key of the stream (seed, domain, index). */
u64 or_sm_stream(u64 seed, u64 domain, u64 index) {
    return mix64(mix64(seed + domain * SM_GAMMA) + index * SM_GAMMA);
}

/* Ternary value in {-1, 0, 1} from one word: floor(w * 3 / 2^64) - 1. */
void or_sample_ternary(u64 key, int64_t *out, u64 n) {
    for (u64 i = 0; i < n; i++) {
        u64 w = or_sm_word(key, i);
        out[i] = (int64_t)(u64)(((u128)w * 3) >> 64) - 1;
    }
}
/* Sparse ternary vector with exactly h nonzero entries: word c = 0, 1, ..   */
/* places sign (w & 1 ? -1 : +1) at position (w >> 1) mod n unless that     */
/* position already holds one.  n is a power of two, h <= n.                */
void or_sample_sparse(u64 key, int64_t *out, u64 n, u64 h) {
    u64 placed = 0;
    for (u64 i = 0; i < n; i++) out[i] = 0;
    for (u64 c = 0; placed < h; c++) {
        u64 w = or_sm_word(key, c);
        u64 pos = (w >> 1) % n;
        if (out[pos] != 0) continue;
        out[pos] = (w & 1) ? -1 : 1;
        placed++;
    }
}

/* Centred binomial with eta = 21: popcount of 21 bits minus popcount of the */
/* next 21 bits of one word.                                                 */
void or_sample_cbd21(u64 key, int64_t *out, u64 n) {
    for (u64 i = 0; i < n; i++) {
        u64 w = or_sm_word(key, i);
        int a = 0, b = 0;
        for (int k = 0; k < 21; k++) {
            a += (int)((w >> k) & 1);
            b += (int)((w >> (21 + k)) & 1);
        }
        out[i] = a - b;
    }
}
/* Uniform residue mod q from two words (w1, w2) = outputs 2i and 2i+1 of the */
/* stream, offset by `start`: floor((w1 * 2^64 + w2) * q / 2^128).            */
void or_sample_uniform(u64 key, u64 start, u64 q, u64 *out, u64 n) {
    for (u64 i = 0; i < n; i++) {
        u64 w1 = or_sm_word(key, 2 * (start + i));
        u64 w2 = or_sm_word(key, 2 * (start + i) + 1);
        /* the 192-bit product (w1*2^64 + w2) * q, top 64 bits of its lower... */
        u128 hi = (u128)w1 * q;              /* contributes at 2^64 */
        u128 lo = (u128)w2 * q;              /* contributes at 2^0  */
        u128 mid = hi + (lo >> 64);          /* = floor(x*q / 2^64), < 2^64 * q */
        out[i] = (u64)(mid >> 64);
    }
}
