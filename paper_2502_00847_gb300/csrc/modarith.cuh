// Modular arithmetic on 64-bit residues for primes q < 2^60.
//
//  * mul_shoup(x, w, w', q): x * w mod q for a fixed w with w' = floor(w 2^64 / q)
//    (V. Shoup's precomputed-quotient multiplication); any 64-bit x.
//  * redc(T): Montgomery reduction T * 2^-64 mod q for T < q * 2^64
//    (P. Montgomery, "Modular multiplication without trial division", 1985),
//    with qinv_neg = -q^-1 mod 2^64.
//  * Sums of up to 15 products of residues (< 2^60) by Montgomery-form
//    constants stay below q * 2^64, so a dot product needs one redc.
#pragma once
#include <cstdint>

typedef unsigned long long u64;
typedef unsigned __int128 u128;

#if defined(__CUDACC__)
#define SECPE_HD __host__ __device__ __forceinline__
#else
#define SECPE_HD inline
#endif

SECPE_HD u64 mulhi64(u64 a, u64 b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (u64)(((u128)a * b) >> 64);
#endif
}

SECPE_HD u64 add_mod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}

SECPE_HD u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// x * w mod q, result in [0, q).
SECPE_HD u64 mul_shoup(u64 x, u64 w, u64 wp, u64 q) {
    u64 hq = mulhi64(x, wp);
    u64 r = x * w - hq * q;
    return r >= q ? r - q : r;
}

// x * w mod q, result in [0, 2q) (lazy variant).
SECPE_HD u64 mul_shoup_lazy(u64 x, u64 w, u64 wp, u64 q) {
    u64 hq = mulhi64(x, wp);
    return x * w - hq * q;
}

// 128-bit accumulator.
struct acc128 {
    u64 lo, hi;
};

SECPE_HD void mac(acc128 &a, u64 x, u64 y) {
    u64 plo = x * y;
    u64 phi = mulhi64(x, y);
    u64 lo = a.lo + plo;
    a.hi += phi + (lo < plo ? 1ull : 0ull);
    a.lo = lo;
}

// (hi:lo) * 2^-64 mod q, for hi:lo < q * 2^64.
SECPE_HD u64 redc(u64 hi, u64 lo, u64 q, u64 qinv_neg) {
    u64 m = lo * qinv_neg;
    u64 mh = mulhi64(m, q);
    u64 t = hi + mh + (lo != 0 ? 1ull : 0ull);
    return t >= q ? t - q : t;
}

// a * b mod q for a, b < q via two Montgomery reductions (r2 = 2^128 mod q).
SECPE_HD u64 mul_mod(u64 a, u64 b, u64 q, u64 qinv_neg, u64 r2) {
    u64 t = redc(mulhi64(a, b), a * b, q, qinv_neg);  // a b 2^-64
    return redc(mulhi64(t, r2), t * r2, q, qinv_neg);  // a b
}

// x mod q for x < 2^64 with mu = floor(2^64 / q).
SECPE_HD u64 reduce64(u64 x, u64 q, u64 mu) {
    u64 qq = mulhi64(x, mu);
    u64 r = x - qq * q;
    while (r >= q) r -= q;
    return r;
}
