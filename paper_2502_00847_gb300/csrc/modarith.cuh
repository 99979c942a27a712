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

// a += x * y (mod 2^128).  On the device the 128-bit product is built from
// the four 32 x 32 partial products with one carry chain (multiply-add with
// carry on 32-bit words), which shares the partial products between the two
// halves instead of forming the low and the high half separately.
SECPE_HD void mac(acc128 &a, u64 x, u64 y) {
#if defined(__CUDA_ARCH__)
    uint32_t r0 = (uint32_t)a.lo, r1 = (uint32_t)(a.lo >> 32), r2 = (uint32_t)a.hi, r3 = (uint32_t)(a.hi >> 32);
    const uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32), y0 = (uint32_t)y, y1 = (uint32_t)(y >> 32);
    asm("mad.lo.cc.u32 %0, %4, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %7, %2;\n\t"
        "madc.hi.u32 %3, %5, %7, %3;\n\t"
        "mad.lo.cc.u32 %1, %4, %7, %1;\n\t"
        "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
        "addc.u32 %3, %3, 0;\n\t"
        "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
        "addc.u32 %3, %3, 0;"
        : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3)
        : "r"(x0), "r"(x1), "r"(y0), "r"(y1));
    a.lo = ((u64)r1 << 32) | r0;
    a.hi = ((u64)r3 << 32) | r2;
#else
    u64 plo = x * y;
    u64 phi = mulhi64(x, y);
    u64 lo = a.lo + plo;
    a.hi += phi + (lo < plo ? 1ull : 0ull);
    a.lo = lo;
#endif
}

// x * y as (hi, lo), the same carry chain as mac from a zero accumulator.
SECPE_HD acc128 mul_full(u64 x, u64 y) {
    acc128 a = {0, 0};
    mac(a, x, y);
    return a;
}

// (hi:lo) * 2^-64 mod q, for hi:lo < q * 2^64.
SECPE_HD u64 redc(u64 hi, u64 lo, u64 q, u64 qinv_neg) {
    u64 m = lo * qinv_neg;
    u64 mh = mulhi64(m, q);
    u64 t = hi + mh + (lo != 0 ? 1ull : 0ull);
    return t >= q ? t - q : t;
}

// a * b * 2^-64 mod q (one Montgomery product), for a * b < q * 2^64.
SECPE_HD u64 mont_mul(u64 a, u64 b, u64 q, u64 qinv_neg) {
    const acc128 p = mul_full(a, b);
    return redc(p.hi, p.lo, q, qinv_neg);
}

// a * b mod q for a, b < q via two Montgomery reductions (r2 = 2^128 mod q).
SECPE_HD u64 mul_mod(u64 a, u64 b, u64 q, u64 qinv_neg, u64 r2) {
    const acc128 p = mul_full(a, b);
    u64 t = redc(p.hi, p.lo, q, qinv_neg);  // a b 2^-64
    const acc128 p2 = mul_full(t, r2);
    return redc(p2.hi, p2.lo, q, qinv_neg);  // a b
}

// x mod q for x < 2^64 with mu = floor(2^64 / q).
SECPE_HD u64 reduce64(u64 x, u64 q, u64 mu) {
    u64 qq = mulhi64(x, mu);
    u64 r = x - qq * q;
    while (r >= q) r -= q;
    return r;
}
