// Element-wise, sampling, CRT and key-switching building-block kernels.
//
// Layout conventions: a limb is N consecutive residues; a polynomial is a
// stack of limbs (limb i modulo prime index i for ciphertext primes, nq + j
// for special prime j); a ciphertext batch is [B][2][cap][N] (CtB).
// Per-limb kernels use blockIdx.y for the limb and blockIdx.x * 256 +
// threadIdx.x for a pair of coefficients (one 128-bit load per operand).
#include "internal.h"
#include "kernels.h"
#include "launch.h"

namespace {

__device__ __forceinline__ ulonglong2 ld2(const u64 *p) { return *reinterpret_cast<const ulonglong2 *>(p); }
__device__ __forceinline__ void st2(u64 *p, ulonglong2 v) { *reinterpret_cast<ulonglong2 *>(p) = v; }

// residue of a signed 64-bit integer modulo q
__device__ __forceinline__ u64 signed_mod(long long k, u64 q, u64 mu) {
    if (k >= 0) return reduce64((u64)k, q, mu);
    u64 r = reduce64((u64)(-(k + 1)) + 1, q, mu);
    return r == 0 ? 0 : q - r;
}

// ------------------------------------------------------------ add / sub
__global__ void k_addsub(DevCtx c, const u64 *a, long long as, const u64 *b, long long bs,
                         u64 *o, long long os, int cap_a, int cap_b, int cap_o, int nl, int sub, int npoly) {
    const int li = blockIdx.y;
    const int i = li % nl, k = (li / nl) % npoly, item = li / (npoly * nl);
    const int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= c.n) return;
    const u64 q = c.q[i];
    const long long ao = item * as + ((long long)k * cap_a + i) * c.n + e;
    const long long bo = item * bs + ((long long)k * cap_b + i) * c.n + e;
    const long long oo = item * os + ((long long)k * cap_o + i) * c.n + e;
    ulonglong2 x = ld2(a + ao), y = ld2(b + bo);
    if (sub) {
        x.x = sub_mod(x.x, y.x, q);
        x.y = sub_mod(x.y, y.y, q);
    } else {
        x.x = add_mod(x.x, y.x, q);
        x.y = add_mod(x.y, y.y, q);
    }
    st2(o + oo, x);
}

// ------------------------------------------------------------ sum of ciphertexts
// dst[qy] = sum of the ciphertexts src[qoff[qy] .. qoff[qy+1]) over limbs
// 0..nl-1 of both polynomials (the ensemble sum of every query of a batch in
// one launch); 8 residues per thread.
constexpr int SUM_MAXP = 1536;
struct SumArgs {
    const u64 *src[SUM_MAXP];
    int cap[SUM_MAXP];
    int qoff[SECPE_MAX_BATCH_CONST + 1];
    u64 *dst;
    long long dstride;
    int dcap, nl;
};

__global__ void __launch_bounds__(256) k_sum_cts(DevCtx c, const __grid_constant__ SumArgs a) {
    const int qy = blockIdx.z;
    const int i = blockIdx.y % a.nl, k = blockIdx.y / a.nl;
    const u64 q = c.q[i];
    const int p0 = a.qoff[qy], p1 = a.qoff[qy + 1];
    u64 *D = a.dst + qy * a.dstride + ((long long)k * a.dcap + i) * c.n;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int e = 2 * (threadIdx.x + 256 * (blockIdx.x * 4 + j));
        if (e >= c.n) break;
        ulonglong2 s = ld2(a.src[p0] + ((long long)k * a.cap[p0] + i) * c.n + e);
        for (int p = p0 + 1; p < p1; p++) {
            const ulonglong2 v = ld2(a.src[p] + ((long long)k * a.cap[p] + i) * c.n + e);
            s.x = add_mod(s.x, v.x, q);
            s.y = add_mod(s.y, v.y, q);
        }
        st2(D + e, s);
    }
}

// ------------------------------------------------------------ tensor
// d[item][0..2][i] = (a0 b0, a0 b1 + a1 b0, a1 b1), d has cap nl.  b0, b1 are
// first brought to Montgomery form (b R), so that each product needs one
// reduction: a b = redc(a * bR), and a0 b1 + a1 b0 = redc(a0 b1R + a1 b0R).
// Each thread takes 8 residues (four 16-byte accesses a block-width apart).
__global__ void __launch_bounds__(256) k_tensor(DevCtx c, const u64 *a, long long as, int cap_a, const u64 *b,
                                                long long bs, int cap_b, u64 *d, int nl) {
    const int li = blockIdx.y;
    const int i = li % nl, item = li / nl;
    const u64 q = c.q[i], qi = c.qinv_neg[i], r2 = c.r2[i];
    const u64 *A = a + item * as + (long long)i * c.n;
    const u64 *Bp = b + item * bs + (long long)i * c.n;
    u64 *D = d + (long long)item * 3 * nl * c.n + (long long)i * c.n;
    const long long ps = (long long)nl * c.n, pa = (long long)cap_a * c.n, pb = (long long)cap_b * c.n;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int e = 2 * (threadIdx.x + 256 * (blockIdx.x * 4 + j));
        if (e >= c.n) break;
        const ulonglong2 a0 = ld2(A + e), a1 = ld2(A + pa + e);
        const ulonglong2 b0 = ld2(Bp + e), b1 = ld2(Bp + pb + e);
        ulonglong2 r0, r1, r2v;
#define SECPE_TENSOR_LANE(f)                                   \
    {                                                          \
        const u64 b0m = mont_mul(b0.f, r2, q, qi);             \
        const u64 b1m = mont_mul(b1.f, r2, q, qi);             \
        r0.f = mont_mul(a0.f, b0m, q, qi);                     \
        r2v.f = mont_mul(a1.f, b1m, q, qi);                    \
        acc128 s = mul_full(a0.f, b1m);                        \
        mac(s, a1.f, b0m);                                     \
        r1.f = redc(s.hi, s.lo, q, qi);                        \
    }
        SECPE_TENSOR_LANE(x)
        SECPE_TENSOR_LANE(y)
#undef SECPE_TENSOR_LANE
        st2(D + e, r0);
        st2(D + ps + e, r1);
        st2(D + 2 * ps + e, r2v);
    }
}

// d = a (x) b + c (x) e (two 3-component products and their sum, one pass):
// each output residue is one Montgomery reduction of the summed 128-bit
// products (at most 4 of them, below q 2^64), so it equals the sum of the
// two separate products residue for residue.
struct Tensor2Args {
    const u64 *p[4];  // a, b, c, e: item stride s[k], poly 1 at cap[k] N
    long long s[4];
    int cap[4];
    u64 *d;
    int nl;
};

__global__ void __launch_bounds__(256) k_tensor2(DevCtx c, const __grid_constant__ Tensor2Args t) {
    const int li = blockIdx.y;
    const int i = li % t.nl, item = li / t.nl;
    const u64 q = c.q[i], qi = c.qinv_neg[i], r2 = c.r2[i];
    const u64 *P[4];
    long long pp[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        P[k] = t.p[k] + item * t.s[k] + (long long)i * c.n;
        pp[k] = (long long)t.cap[k] * c.n;
    }
    u64 *D = t.d + (long long)item * 3 * t.nl * c.n + (long long)i * c.n;
    const long long ps = (long long)t.nl * c.n;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int e = 2 * (threadIdx.x + 256 * (blockIdx.x * 4 + j));
        if (e >= c.n) break;
        const ulonglong2 a0 = ld2(P[0] + e), a1 = ld2(P[0] + pp[0] + e);
        const ulonglong2 b0 = ld2(P[1] + e), b1 = ld2(P[1] + pp[1] + e);
        const ulonglong2 c0 = ld2(P[2] + e), c1 = ld2(P[2] + pp[2] + e);
        const ulonglong2 e0 = ld2(P[3] + e), e1 = ld2(P[3] + pp[3] + e);
        ulonglong2 r0, r1, r2v;
#define SECPE_TENSOR2_LANE(f)                                  \
    {                                                          \
        const u64 b0m = mont_mul(b0.f, r2, q, qi);             \
        const u64 b1m = mont_mul(b1.f, r2, q, qi);             \
        const u64 e0m = mont_mul(e0.f, r2, q, qi);             \
        const u64 e1m = mont_mul(e1.f, r2, q, qi);             \
        acc128 s0 = mul_full(a0.f, b0m);                       \
        mac(s0, c0.f, e0m);                                    \
        r0.f = redc(s0.hi, s0.lo, q, qi);                      \
        acc128 s2 = mul_full(a1.f, b1m);                       \
        mac(s2, c1.f, e1m);                                    \
        r2v.f = redc(s2.hi, s2.lo, q, qi);                     \
        acc128 s1 = mul_full(a0.f, b1m);                       \
        mac(s1, a1.f, b0m);                                    \
        mac(s1, c0.f, e1m);                                    \
        mac(s1, c1.f, e0m);                                    \
        r1.f = redc(s1.hi, s1.lo, q, qi);                      \
    }
        SECPE_TENSOR2_LANE(x)
        SECPE_TENSOR2_LANE(y)
#undef SECPE_TENSOR2_LANE
        st2(D + e, r0);
        st2(D + ps + e, r1);
        st2(D + 2 * ps + e, r2v);
    }
}

// ------------------------------------------------------------ constants
struct KArr {
    long long k[SECPE_MAX_BATCH_CONST];
};

// out = sum_t x_t * k_{t,item} mod q_i on both polynomials, limbs 0..nl-1
// (NT = 1: a constant multiple).  Each thread takes 8 residues (four
// 16-byte accesses one block-width apart), so the per-thread Montgomery form
// of the constants is amortised; one reduction per residue for all terms.
struct LinArgs {
    const u64 *x[2];
    long long xs[2];
    int cap[2];
    u64 *o;
    long long os;
    int cap_o, nl, per_item;
    long long k[2][SECPE_MAX_BATCH_CONST];
};

template <int NT>
__global__ void __launch_bounds__(256) k_lincomb(DevCtx c, const __grid_constant__ LinArgs a) {
    const int li = blockIdx.y;
    const int i = li % a.nl, kk = (li / a.nl) & 1, item = li / (2 * a.nl);
    const u64 q = c.q[i], qi = c.qinv_neg[i], r2 = c.r2[i];
    u64 wm[NT];
    const u64 *xp[NT];
#pragma unroll
    for (int t = 0; t < NT; t++) {
        const u64 w = signed_mod(a.k[t][a.per_item ? item : 0], q, c.mu[i]);
        wm[t] = mont_mul(w, r2, q, qi);  // w * 2^64 mod q
        xp[t] = a.x[t] + item * a.xs[t] + ((long long)kk * a.cap[t] + i) * c.n;
    }
    u64 *op = a.o + item * a.os + ((long long)kk * a.cap_o + i) * c.n;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int e = 2 * (threadIdx.x + 256 * (blockIdx.x * 4 + j));
        if (e >= c.n) break;
        acc128 s0 = {0, 0}, s1 = {0, 0};
#pragma unroll
        for (int t = 0; t < NT; t++) {
            const ulonglong2 v = ld2(xp[t] + e);
            mac(s0, v.x, wm[t]);
            mac(s1, v.y, wm[t]);
        }
        ulonglong2 r;
        r.x = redc(s0.hi, s0.lo, q, qi);
        r.y = redc(s1.hi, s1.lo, q, qi);
        st2(op + e, r);
    }
}

// out = x with k_item added to every NTT value of c0 (the constant polynomial)
__global__ void k_addconst(DevCtx c, const u64 *x, long long xs, int cap_x, u64 *o, long long os,
                           int cap_o, int nl, const __grid_constant__ KArr ka, int per_item) {
    const int li = blockIdx.y;
    const int i = li % nl, kk = (li / nl) & 1, item = li / (2 * nl);
    const int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= c.n) return;
    const u64 q = c.q[i];
    ulonglong2 v = ld2(x + item * xs + ((long long)kk * cap_x + i) * c.n + e);
    if (kk == 0) {
        const u64 w = signed_mod(ka.k[per_item ? item : 0], q, c.mu[i]);
        v.x = add_mod(v.x, w, q);
        v.y = add_mod(v.y, w, q);
    }
    st2(o + item * os + ((long long)kk * cap_o + i) * c.n + e, v);
}

// ------------------------------------------------------------ automorphism
// In NTT form (bit-reversed evaluations at psi^(2 brv(j) + 1)), X -> X^g
// is the permutation out[j] = in[sigma(j)], 2 brv(sigma(j)) + 1 = g (2 brv(j) + 1) mod 2N.
__global__ void k_automorph(DevCtx c, const u64 *x, long long xs, int cap_x, u64 *o, long long os,
                            int cap_o, int nl, unsigned g) {
    const int li = blockIdx.y;
    const int i = li % nl, kk = (li / nl) & 1, item = li / (2 * nl);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= c.n) return;
    const unsigned sh = 32 - c.log_n;
    const unsigned ev = 2u * (__brev((unsigned)j) >> sh) + 1u;
    const unsigned e2 = (unsigned)(((unsigned long long)ev * g) & (2ull * c.n - 1));
    const unsigned src = __brev((e2 - 1u) >> 1) >> sh;
    o[item * os + ((long long)kk * cap_o + i) * c.n + j] = x[item * xs + ((long long)kk * cap_x + i) * c.n + src];
}

// The same permutation on contiguous limbs [count][N] (any primes: it only
// moves residues).
__global__ void k_automorph_flat(DevCtx c, const u64 *x, u64 *o, unsigned g) {
    const long long li = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= c.n) return;
    const unsigned sh = 32 - c.log_n;
    const unsigned ev = 2u * (__brev((unsigned)j) >> sh) + 1u;
    const unsigned e2 = (unsigned)(((unsigned long long)ev * g) & (2ull * c.n - 1));
    const unsigned src = __brev((e2 - 1u) >> 1) >> sh;
    o[li * c.n + j] = x[li * c.n + src];
}

// ------------------------------------------------------------ rescale
// y: coefficient form of the last limb (level l) of both polys, [item][2][N].
// z[item][2][i] = ([y + h]_{q_l} - h) mod q_i for i < l (coefficient form).
__global__ void k_rescale_prep(DevCtx c, const u64 *y, u64 *z, int lv) {
    const int li = blockIdx.y;  // (item, poly, i), i < lv
    const int i = li % lv, kp = li / lv;  // kp = item*2 + poly
    const int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= c.n) return;
    const u64 ql = c.q[lv], h = ql >> 1;
    const u64 qi = c.q[i], mui = c.mu[i];
    const u64 hm = c.rs_hmod[(size_t)lv * c.nq + i];
    ulonglong2 v = ld2(y + (long long)kp * c.n + e);
    u64 y0 = add_mod(v.x, h, ql), y1 = add_mod(v.y, h, ql);
    ulonglong2 r;
    r.x = sub_mod(reduce64(y0, qi, mui), hm, qi);
    r.y = sub_mod(reduce64(y1, qi, mui), hm, qi);
    st2(z + ((long long)kp * lv + i) * c.n + e, r);
}

// out_i = (x_i - Z_i) * q_l^-1 mod q_i (NTT form), i < lv
__global__ void k_rescale_fin(DevCtx c, const u64 *x, long long xs, int cap_x, const u64 *z, u64 *o,
                              long long os, int cap_o, int lv) {
    const int li = blockIdx.y;
    const int i = li % lv, kk = (li / lv) & 1, item = li / (2 * lv);
    const int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= c.n) return;
    const u64 q = c.q[i];
    const ulonglong2 w = c.rs_qinv[(size_t)lv * c.nq + i];
    ulonglong2 a = ld2(x + item * xs + ((long long)kk * cap_x + i) * c.n + e);
    const ulonglong2 b = ld2(z + (((long long)item * 2 + kk) * lv + i) * c.n + e);
    a.x = mul_shoup(sub_mod(a.x, b.x, q), w.x, w.y, q);
    a.y = mul_shoup(sub_mod(a.y, b.y, q), w.x, w.y, q);
    st2(o + item * os + ((long long)kk * cap_o + i) * c.n + e, a);
}

// ------------------------------------------------------------ key switching
// ModUp base conversion of digit j: x = coefficient-form limbs of d
// ([item][lv+1][N]); ext_j[item][t'] for the targets of digit j.
#define BCONV_TG 6
// ND > 0: digit size known at compile time (registers); ND = 0: generic.
template <int ND>
__global__ void k_modup_bconv(DevCtx c, const u64 *x, u64 *ext, long long ext_item_stride,
                              int ext_off, int lv, int j, int lo, int hi, int ntgt) {
    const int ngrp = (ntgt + BCONV_TG - 1) / BCONV_TG;
    const int item = blockIdx.y / ngrp, grp = blockIdx.y % ngrp;
    const int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= c.n) return;
    const int nd = ND > 0 ? ND : hi - lo;
    const size_t tb = ((size_t)lv * c.dnum + j) * c.alpha;
    ulonglong2 y[ND > 0 ? ND : 16];
#pragma unroll
    for (int r = 0; r < nd; r++) {
        const ulonglong2 w = c.mu_inv[tb + r];
        const u64 q = c.q[lo + r];
        const ulonglong2 v = ld2(x + ((long long)item * (lv + 1) + lo + r) * c.n + e);
        y[r] = make_ulonglong2(mul_shoup(v.x, w.x, w.y, q), mul_shoup(v.y, w.x, w.y, q));
    }
    u64 *out = ext + item * ext_item_stride + (long long)ext_off * c.n + e;
    const int t0 = grp * BCONV_TG, t1 = min(ntgt, t0 + BCONV_TG);
    for (int tt = t0; tt < t1; tt++) {
        // compact target index tt -> position t in [0, lv + 1 + k) skipping the digit
        const int t = tt < lo ? tt : tt + nd;
        const int pt = t <= lv ? t : c.nq + (t - lv - 1);
        const u64 q = c.q[pt], qinv = c.qinv_neg[pt];
        acc128 sa = {0, 0}, sb = {0, 0};
#pragma unroll
        for (int r = 0; r < nd; r++) {
            const u64 h = c.mu_hat[(tb + r) * c.nprimes + pt];
            mac(sa, y[r].x, h);
            mac(sb, y[r].y, h);
        }
        st2(out + (long long)tt * c.n, make_ulonglong2(redc(sa.hi, sa.lo, q, qinv), redc(sb.hi, sb.lo, q, qinv)));
    }
}

// Inner product with the key over digits: acc[item][0/1][t] for targets
// t = 0..lv (q_t) and lv+1.. (special primes); key in Montgomery form.
// With gal != 0 the extended limbs are read through the automorphism
// X -> X^gal (NTT form: a gather, as k_automorph), so that a hoisted
// rotation needs no permuted copy of them.
__device__ __forceinline__ unsigned automorph_src(unsigned j, unsigned g, int log_n, int n) {
    const unsigned sh = 32 - log_n;
    const unsigned ev = 2u * (__brev(j) >> sh) + 1u;
    const unsigned e2 = (unsigned)(((unsigned long long)ev * g) & (2ull * n - 1));
    return __brev((e2 - 1u) >> 1) >> sh;
}

__global__ void k_ksk_ip(DevCtx c, const u64 *d, long long d_item_stride, const u64 *ext,
                         long long ext_item_stride, const __grid_constant__ KsDigits dg,
                         const u64 *key, u64 *acc, int lv, unsigned gal) {
    const int nt = lv + 1 + c.np_special;
    const int nitem = gridDim.y / nt;
    // target-major order: the items sharing one key limb run back to back
    const int t = blockIdx.y / nitem, item = blockIdx.y % nitem;
    const int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= c.n) return;
    const unsigned g0 = gal ? automorph_src((unsigned)e, gal, c.log_n, c.n) : 0u;
    const unsigned g1 = gal ? automorph_src((unsigned)e + 1u, gal, c.log_n, c.n) : 0u;
    const int pt = t <= lv ? t : c.nq + (t - lv - 1);
    const u64 q = c.q[pt], qi = c.qinv_neg[pt];
    acc128 s0a = {0, 0}, s0b = {0, 0}, s1a = {0, 0}, s1b = {0, 0};
    const long long kpoly = (long long)c.nprimes * c.n;
    for (int j = 0; j < dg.ndig; j++) {
        const int lo = dg.lo[j], hi = dg.hi[j];
        ulonglong2 xv;
        if (t >= lo && t < hi) {
            xv = ld2(d + item * d_item_stride + (long long)t * c.n + e);
        } else {
            const int tt = t < lo ? t : t - (hi - lo);
            const u64 *xl = ext + item * ext_item_stride + (long long)(dg.off[j] + tt) * c.n;
            xv = gal ? make_ulonglong2(xl[g0], xl[g1]) : ld2(xl + e);
        }
        const u64 *kb = key + (long long)j * 2 * kpoly + (long long)pt * c.n + e;
        const ulonglong2 k0 = ld2(kb), k1 = ld2(kb + kpoly);
        mac(s0a, xv.x, k0.x);
        mac(s0b, xv.y, k0.y);
        mac(s1a, xv.x, k1.x);
        mac(s1b, xv.y, k1.y);
    }
    u64 *o = acc + (long long)item * 2 * nt * c.n + (long long)t * c.n + e;
    st2(o, make_ulonglong2(redc(s0a.hi, s0a.lo, q, qi), redc(s0b.hi, s0b.lo, q, qi)));
    st2(o + (long long)nt * c.n,
        make_ulonglong2(redc(s1a.hi, s1a.lo, q, qi), redc(s1b.hi, s1b.lo, q, qi)));
}

// ModDown base conversion: P-part limbs (coefficient form) of acc ->
// conv[item][poly][i] = FastBConv([x + h]_P -> q_i) - h mod q_i.
template <int KS>
__global__ void k_moddown_bconv(DevCtx c, const u64 *acc, u64 *conv, int lv) {
    const int nt = lv + 1 + c.np_special;
    const int ngrp = (lv + 1 + BCONV_TG - 1) / BCONV_TG;
    const int kp = blockIdx.y / ngrp, grp = blockIdx.y % ngrp;  // kp = item*2 + poly
    const int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= c.n) return;
    const int k = KS > 0 ? KS : c.np_special;
    ulonglong2 y[KS > 0 ? KS : 8];
#pragma unroll
    for (int j = 0; j < k; j++) {
        const int pj = c.nq + j;
        const u64 q = c.q[pj];
        ulonglong2 v = ld2(acc + ((long long)kp * nt + lv + 1 + j) * c.n + e);
        v.x = add_mod(v.x, c.md_hP[pj], q);
        v.y = add_mod(v.y, c.md_hP[pj], q);
        const ulonglong2 w = c.md_inv[j];
        y[j] = make_ulonglong2(mul_shoup(v.x, w.x, w.y, q), mul_shoup(v.y, w.x, w.y, q));
    }
    const int i0 = grp * BCONV_TG, i1 = min(lv + 1, i0 + BCONV_TG);
    for (int i = i0; i < i1; i++) {
        acc128 sa = {0, 0}, sb = {0, 0};
#pragma unroll
        for (int j = 0; j < k; j++) {
            const u64 h = c.md_hat[(size_t)j * c.nq + i];
            mac(sa, y[j].x, h);
            mac(sb, y[j].y, h);
        }
        const u64 q = c.q[i], qinv = c.qinv_neg[i];
        ulonglong2 r = make_ulonglong2(redc(sa.hi, sa.lo, q, qinv), redc(sb.hi, sb.lo, q, qinv));
        r.x = sub_mod(r.x, c.md_hP[i], q);
        r.y = sub_mod(r.y, c.md_hP[i], q);
        st2(conv + ((long long)kp * (lv + 1) + i) * c.n + e, r);
    }
}

// out[item][poly][i] (+)= (acc_i - conv_i) * P^-1 mod q_i (NTT form)
__global__ void k_moddown_fin(DevCtx c, const u64 *acc, const u64 *conv, u64 *o, long long os, int cap_o,
                              int lv, int accum0, int accum1) {
    const int nl = lv + 1, nt = lv + 1 + c.np_special;
    const int li = blockIdx.y;
    const int i = li % nl, kp = li / nl, kk = kp & 1, item = kp >> 1;
    const int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= c.n) return;
    const u64 q = c.q[i];
    const ulonglong2 w = c.md_pinv[i];
    const ulonglong2 a = ld2(acc + ((long long)kp * nt + i) * c.n + e);
    const ulonglong2 b = ld2(conv + ((long long)kp * nl + i) * c.n + e);
    ulonglong2 r;
    r.x = mul_shoup(sub_mod(a.x, b.x, q), w.x, w.y, q);
    r.y = mul_shoup(sub_mod(a.y, b.y, q), w.x, w.y, q);
    u64 *op = o + item * os + ((long long)kk * cap_o + i) * c.n + e;
    if (kk == 0 ? accum0 : accum1) {
        const ulonglong2 old = ld2(op);
        r.x = add_mod(r.x, old.x, q);
        r.y = add_mod(r.y, old.y, q);
    }
    st2(op, r);
}

// ------------------------------------------------------------ sampling
__device__ __forceinline__ u64 sm_mix(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ u64 sm_word(u64 key, u64 ctr) { return sm_mix(key + (ctr + 1) * 0x9E3779B97F4A7C15ull); }

// uniform residues: out limb r (prime prime_of[r]) at offset r*N of item `it`
__global__ void k_sample_uniform(DevCtx c, const __grid_constant__ KeyArr keys, u64 *out,
                                 long long item_stride, const __grid_constant__ PrimeList pl) {
    const int r = blockIdx.y % pl.n, it = blockIdx.y / pl.n;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= c.n) return;
    const int pi = pl.p[r];
    const u64 q = c.q[pi];
    const u64 key = keys.k[it];
    const u64 ctr = 2ull * ((u64)pi * c.n + t);
    const u64 w1 = sm_word(key, ctr), w2 = sm_word(key, ctr + 1);
    const u128 hi = (u128)w1 * q;
    const u64 lo_hi = mulhi64(w2, q);
    out[it * item_stride + (long long)r * c.n + t] = (u64)((hi + lo_hi) >> 64);
}

// small integers: kind 0 = ternary, 1 = centred binomial eta = 21
__global__ void k_sample_small(DevCtx c, const __grid_constant__ KeyArr keys, long long *out, int kind) {
    const int it = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= c.n) return;
    const u64 w = sm_word(keys.k[it], t);
    long long v;
    if (kind == 0) {
        v = (long long)mulhi64(w, 3ull) - 1;
    } else {
        v = (long long)__popcll(w & 0x1FFFFFull) - (long long)__popcll((w >> 21) & 0x1FFFFFull);
    }
    out[(long long)it * c.n + t] = v;
}

// out[it][r][t] = (m[it][t] + e[it][t]) mod prime pl.p[r]  (e optional)
__global__ void k_signed_to_limbs(DevCtx c, const long long *m, const long long *e, u64 *out,
                                  long long item_stride, const __grid_constant__ PrimeList pl) {
    const int r = blockIdx.y % pl.n, it = blockIdx.y / pl.n;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= c.n) return;
    const int pi = pl.p[r];
    long long v = m ? m[(long long)it * c.n + t] : 0;
    if (e) v += e[(long long)it * c.n + t];
    out[it * item_stride + (long long)r * c.n + t] = signed_mod(v, c.q[pi], c.mu[pi]);
}

// c0 = M - a*s, c1 = a (NTT form), limbs 0..nl-1, prime index = limb index
__global__ void k_enc_finish(DevCtx c, const u64 *M, long long ms, const u64 *a, long long as,
                             const u64 *s, u64 *o, long long os, int cap_o, int nl) {
    const int li = blockIdx.y;
    const int i = li % nl, it = li / nl;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= c.n) return;
    const u64 q = c.q[i];
    const u64 av = a[it * as + (long long)i * c.n + e];
    const u64 as_ = mul_mod(av, s[(long long)i * c.n + e], q, c.qinv_neg[i], c.r2[i]);
    u64 *op = o + it * os + (long long)i * c.n + e;
    op[0] = sub_mod(M[it * ms + (long long)i * c.n + e], as_, q);
    op[(long long)cap_o * c.n] = av;
}

// m_i = c0_i + c1_i * s_i
__global__ void k_dec_dot(DevCtx c, const u64 *x, long long xs, int cap_x, const u64 *s, u64 *m, int nl) {
    const int li = blockIdx.y;
    const int i = li % nl, it = li / nl;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= c.n) return;
    const u64 q = c.q[i];
    const u64 *p = x + it * xs + (long long)i * c.n + e;
    const u64 cs = mul_mod(p[(long long)cap_x * c.n], s[(long long)i * c.n + e], q, c.qinv_neg[i], c.r2[i]);
    m[((long long)it * nl + i) * c.n + e] = add_mod(p[0], cs, q);
}

// Mixed-radix digits v_0..v_l of the residues x_0..x_l (Garner).
__device__ __forceinline__ void mixed_radix(const DevCtx &c, const u64 *x, int lv, u64 *v) {
    for (int i = 0; i <= lv; i++) {
        const u64 q = c.q[i];
        u64 a = x[i];
        for (int j = 0; j < i; j++) {
            const ulonglong2 w = c.mr_inv[(size_t)j * c.nq + i];
            a = mul_shoup(sub_mod(a, reduce64(v[j], q, c.mu[i]), q), w.x, w.y, q);
        }
        v[i] = a;
    }
}

// is X > (Q_l - 1)/2 ?  (compare mixed-radix digits from the top)
__device__ __forceinline__ bool mr_greater_half(const DevCtx &c, const u64 *v, int lv) {
    for (int i = lv; i >= 0; i--) {
        const u64 h = c.mr_H[(size_t)lv * c.nq + i];
        if (v[i] != h) return v[i] > h;
    }
    return false;
}

// Centred integer value of each coefficient as a double.
__global__ void k_crt_double(DevCtx c, const u64 *m, int lv, double *out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= c.n) return;
    u64 x[SECPE_MAX_PRIMES], v[SECPE_MAX_PRIMES];
    for (int i = 0; i <= lv; i++) x[i] = m[(long long)i * c.n + e];
    mixed_radix(c, x, lv, v);
    const bool neg = mr_greater_half(c, v, lv);
    double acc = 0.0;
    for (int i = lv; i >= 0; i--) {
        const double d = neg ? (double)(c.q[i] - 1 - v[i]) : (double)v[i];
        acc = acc * (double)c.q[i] + d;
    }
    out[e] = neg ? -(acc + 1.0) : acc;
}

// Exact centred lift of m (coefficient form, level lv) plus e, reduced
// modulo every ciphertext prime: out[it][t] for t = 0..ntop-1.
__global__ void k_crt_lift(DevCtx c, const u64 *m, int lv, const long long *e, u64 *out,
                           long long out_item_stride, int ntop) {
    const int it = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= c.n) return;
    u64 x[SECPE_MAX_PRIMES], v[SECPE_MAX_PRIMES];
    for (int i = 0; i <= lv; i++) x[i] = m[((long long)it * (lv + 1) + i) * c.n + t];
    mixed_radix(c, x, lv, v);
    const bool neg = mr_greater_half(c, v, lv);
    const long long ev = e[(long long)it * c.n + t];
    for (int p = 0; p < ntop; p++) {
        const u64 q = c.q[p], qi = c.qinv_neg[p], r2 = c.r2[p];
        u64 acc = 0;
        for (int i = 0; i <= lv; i++)
            acc = add_mod(acc, mul_mod(reduce64(v[i], q, c.mu[p]), c.mr_M[(size_t)i * c.nq + p], q, qi, r2), q);
        if (neg) acc = sub_mod(acc, c.mr_Q[(size_t)lv * c.nq + p], q);
        acc = add_mod(acc, signed_mod(ev, q, c.mu[p]), q);
        out[it * out_item_stride + (long long)p * c.n + t] = acc;
    }
}

// Key-switching key of digit [lo, hi): over every prime t,
// b = -a s + e + (lo <= t < hi ? [P]_{q_t} s' : 0), stored (b, a) in
// Montgomery form at key[0][t], key[1][t].
__global__ void k_ksk_gen(DevCtx c, const u64 *a, const u64 *e_ntt, const u64 *s, const u64 *sp,
                          const u64 *pmod, u64 *key, int lo, int hi) {
    const int t = blockIdx.y;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= c.n) return;
    const u64 q = c.q[t], qi = c.qinv_neg[t], r2 = c.r2[t];
    const long long o = (long long)t * c.n + x;
    const u64 av = a[o];
    u64 b = sub_mod(e_ntt[o], mul_mod(av, s[o], q, qi, r2), q);
    if (t >= lo && t < hi) b = add_mod(b, mul_mod(pmod[t], sp[o], q, qi, r2), q);
    const long long kp = (long long)c.nprimes * c.n;
    key[o] = mont_mul(b, r2, q, qi);
    key[kp + o] = mont_mul(av, r2, q, qi);
}

// Montgomery form -> plain residues (key export)
__global__ void k_from_mont(DevCtx c, const u64 *in, u64 *out, int nlimb_total) {
    const int li = blockIdx.y;
    const int t = li % c.nprimes;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= c.n) return;
    const long long o = (long long)li * c.n + x;
    out[o] = redc(0, in[o], c.q[t], c.qinv_neg[t]);
}

// elementwise product of two limb stacks over primes 0..np-1 (s*s)
__global__ void k_limb_mul(DevCtx c, const u64 *a, const u64 *b, u64 *o) {
    const int t = blockIdx.y;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= c.n) return;
    const long long i = (long long)t * c.n + x;
    o[i] = mul_mod(a[i], b[i], c.q[t], c.qinv_neg[t], c.r2[t]);
}

// automorphism of one limb stack over all primes (NTT form)
__global__ void k_limb_automorph(DevCtx c, const u64 *in, u64 *o, unsigned g) {
    const int t = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= c.n) return;
    const unsigned sh = 32 - c.log_n;
    const unsigned ev = 2u * (__brev((unsigned)j) >> sh) + 1u;
    const unsigned e2 = (unsigned)(((unsigned long long)ev * g) & (2ull * c.n - 1));
    const unsigned src = __brev((e2 - 1u) >> 1) >> sh;
    o[(long long)t * c.n + j] = in[(long long)t * c.n + src];
}

// ------------------------------------------------------------ relin ModDown + rescale
// acc[item][poly][lv] <- P * d[item][poly][lv] + acc[item][poly][lv] (NTT form):
// the q_l limb of x = P d + acc, next to the special limbs in acc.
__global__ void k_mdr_prep(DevCtx c, const u64 *d, long long dis, long long dps, u64 *acc, int lv) {
    const int nt = lv + 1 + c.np_special;
    const int kp = blockIdx.y;  // item*2 + poly
    const int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= c.n) return;
    const int item = kp >> 1, poly = kp & 1;
    const u64 q = c.q[lv], qi = c.qinv_neg[lv], r2 = c.r2[lv], pm = c.pmod[lv];
    const ulonglong2 dv = ld2(d + item * dis + poly * dps + (long long)lv * c.n + e);
    u64 *ap = acc + ((long long)kp * nt + lv) * c.n + e;
    ulonglong2 av = ld2(ap);
    av.x = add_mod(av.x, mul_mod(dv.x, pm, q, qi, r2), q);
    av.y = add_mod(av.y, mul_mod(dv.y, pm, q, qi, r2), q);
    st2(ap, av);
}

// generic path: sources = acc limbs lv..lv+k (coefficient form) of (item, poly);
// conv[item][poly][i] = FastBConv([x + h]_M -> q_i) - h, i < lv
__global__ void k_mdr_bconv(DevCtx c, const u64 *acc, u64 *conv, int lv) {
    const int nt = lv + 1 + c.np_special, ks = c.np_special + 1;
    const int kp = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= c.n) return;
    u64 y[9];
    for (int j = 0; j < ks; j++) {
        const int sp = j == 0 ? lv : c.nq + j - 1;
        const u64 q = c.q[sp];
        u64 v = acc[((long long)kp * nt + lv + j) * c.n + e];
        v = add_mod(v, c.mdr_pre[(size_t)lv * ks + j], q);
        const ulonglong2 w = c.mdr_inv[(size_t)lv * ks + j];
        y[j] = mul_shoup(v, w.x, w.y, q);
    }
    for (int i = 0; i < lv; i++) {
        acc128 s = {0, 0};
        for (int j = 0; j < ks; j++) mac(s, y[j], c.mdr_hat[((size_t)lv * ks + j) * c.nq + i]);
        const u64 q = c.q[i];
        const u64 r = redc(s.hi, s.lo, q, c.qinv_neg[i]);
        conv[((long long)kp * lv + i) * c.n + e] = sub_mod(r, c.mdr_post[(size_t)lv * c.nq + i], q);
    }
}

// out_i = (acc_i - conv_i) * M^-1 + d_i * q_l^-1, i < lv
__global__ void k_mdr_fin(DevCtx c, const u64 *acc, const u64 *conv, const u64 *d, long long dis, long long dps,
                          u64 *o, long long os, int cap_o, int lv) {
    const int nt = lv + 1 + c.np_special;
    const int li = blockIdx.y;
    const int i = li % lv, kp = li / lv, item = kp >> 1, poly = kp & 1;
    const int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= c.n) return;
    const u64 q = c.q[i];
    const ulonglong2 w = c.mdr_w[(size_t)lv * c.nq + i], w2 = c.rs_qinv[(size_t)lv * c.nq + i];
    const ulonglong2 a = ld2(acc + ((long long)kp * nt + i) * c.n + e);
    const ulonglong2 b = ld2(conv + ((long long)kp * lv + i) * c.n + e);
    const ulonglong2 dv = ld2(d + item * dis + poly * dps + (long long)i * c.n + e);
    ulonglong2 r;
    r.x = add_mod(mul_shoup(sub_mod(a.x, b.x, q), w.x, w.y, q), mul_shoup(dv.x, w2.x, w2.y, q), q);
    r.y = add_mod(mul_shoup(sub_mod(a.y, b.y, q), w.x, w.y, q), mul_shoup(dv.y, w2.x, w2.y, q), q);
    st2(o + item * os + ((long long)poly * cap_o + i) * c.n + e, r);
}

}  // namespace

// ======================================================================
// host launchers
// ======================================================================
static dim3 limb_grid(int n, int per_thread, long long nlimbs) {
    return dim3((unsigned)((n / per_thread + 255) / 256), (unsigned)nlimbs);
}

int launch_addsub(secpe_ctx *ctx, const CtB &a, const CtB &b, const CtB &o, int nl, bool sub, int npoly) {
    if (nl <= 0 || a.B == 0) return SECPE_OK;
    KprofScope kp(ctx, "ew_addsub", 24.0 * ctx->n * a.B * npoly * nl);
    SECPE_LAUNCH(ctx, k_addsub, limb_grid(ctx->n, 2, (long long)a.B * npoly * nl), 256, 0, ctx->dev, a.data,
                 a.stride, b.data, b.stride, o.data, o.stride, a.cap, b.cap, o.cap, nl, sub ? 1 : 0, npoly);
    return SECPE_OK;
}

int launch_sum_cts(secpe_ctx *ctx, const std::vector<const u64 *> &src, const std::vector<int> &cap,
                   const std::vector<int> &qoff, const CtB &dst, int nl) {
    const int nq = (int)qoff.size() - 1;
    if (nq < 1 || nq > dst.B || nl < 1 || nl > dst.cap || src.size() != cap.size() || qoff[0] != 0 ||
        qoff[nq] != (int)src.size())
        return SECPE_EINVAL;
    int q0 = 0;
    while (q0 < nq) {
        // as many queries as the pointer table holds
        int q1 = q0;
        while (q1 < nq && q1 - q0 < SECPE_MAX_BATCH_CONST && qoff[q1 + 1] - qoff[q0] <= SUM_MAXP) q1++;
        if (q1 == q0) return SECPE_EINVAL;  // one query with more inputs than the table
        SumArgs sa;
        const int base = qoff[q0];
        for (int p = base; p < qoff[q1]; p++) {
            if (!src[p] || cap[p] < nl) return SECPE_EINVAL;
            sa.src[p - base] = src[p];
            sa.cap[p - base] = cap[p];
        }
        for (int qq = q0; qq <= q1; qq++) {
            if (qq < q1 && qoff[qq + 1] <= qoff[qq]) return SECPE_EINVAL;
            sa.qoff[qq - q0] = qoff[qq] - base;
        }
        sa.dst = dst.data + (long long)q0 * dst.stride;
        sa.dstride = dst.stride;
        sa.dcap = dst.cap;
        sa.nl = nl;
        const dim3 grid((unsigned)((ctx->n + 2047) / 2048), (unsigned)(2 * nl), (unsigned)(q1 - q0));
        KprofScope kp(ctx, "ew_sum", 16.0 * ctx->n * nl * (qoff[q1] - base + (q1 - q0)));
        SECPE_LAUNCH(ctx, k_sum_cts, grid, 256, 0, ctx->dev, sa);
        q0 = q1;
    }
    return SECPE_OK;
}

int launch_tensor(secpe_ctx *ctx, const CtB &a, const CtB &b, u64 *d, int nl) {
    KprofScope kp(ctx, "ew_tensor", 56.0 * ctx->n * a.B * nl);
    const dim3 grid((unsigned)((ctx->n + 2047) / 2048), (unsigned)((long long)a.B * nl));
    SECPE_LAUNCH(ctx, k_tensor, grid, 256, 0, ctx->dev, a.data, a.stride, a.cap, b.data, b.stride, b.cap, d, nl);
    return SECPE_OK;
}

int launch_tensor2(secpe_ctx *ctx, const CtB &a, const CtB &b, const CtB &c, const CtB &e, u64 *d, int nl) {
    if (a.B != b.B || a.B != c.B || a.B != e.B) return SECPE_EINVAL;
    KprofScope kp(ctx, "ew_tensor2", 88.0 * ctx->n * a.B * nl);
    Tensor2Args t;
    const CtB *src[4] = {&a, &b, &c, &e};
    for (int k = 0; k < 4; k++) {
        t.p[k] = src[k]->data;
        t.s[k] = src[k]->stride;
        t.cap[k] = src[k]->cap;
    }
    t.d = d;
    t.nl = nl;
    const dim3 grid((unsigned)((ctx->n + 2047) / 2048), (unsigned)((long long)a.B * nl));
    SECPE_LAUNCH(ctx, k_tensor2, grid, 256, 0, ctx->dev, t);
    return SECPE_OK;
}

int launch_lincomb(secpe_ctx *ctx, const CtB *xs, const std::vector<long long> *ks, int nt, const CtB &o,
                   int nl) {
    if (nt < 1 || nt > 2 || nl <= 0) return SECPE_EINVAL;
    const int B = o.B;
    if (B < 1 || B > SECPE_MAX_BATCH_CONST) return SECPE_EINVAL;
    LinArgs la;
    la.per_item = 0;
    for (int t = 0; t < nt; t++) {
        if (xs[t].B != B || (ks[t].size() != 1 && (int)ks[t].size() != B)) return SECPE_EINVAL;
        if (ks[t].size() != 1) la.per_item = 1;
    }
    for (int t = 0; t < nt; t++) {
        la.x[t] = xs[t].data;
        la.xs[t] = xs[t].stride;
        la.cap[t] = xs[t].cap;
        for (int b = 0; b < (la.per_item ? B : 1); b++) la.k[t][b] = ks[t][ks[t].size() == 1 ? 0 : b];
    }
    la.o = o.data;
    la.os = o.stride;
    la.cap_o = o.cap;
    la.nl = nl;
    const dim3 grid((unsigned)((ctx->n + 2047) / 2048), (unsigned)((long long)B * 2 * nl));
    KprofScope kp(ctx, "ew_lincomb", 16.0 * ctx->n * B * nl * (nt + 1));
    if (nt == 1)
        SECPE_LAUNCH(ctx, k_lincomb<1>, grid, 256, 0, ctx->dev, la);
    else
        SECPE_LAUNCH(ctx, k_lincomb<2>, grid, 256, 0, ctx->dev, la);
    return SECPE_OK;
}

static int fill_karr(KArr &ka, const std::vector<long long> &k, int B, int &per_item) {
    if ((int)k.size() == 1) {
        per_item = 0;
        ka.k[0] = k[0];
        return SECPE_OK;
    }
    if ((int)k.size() != B || B > SECPE_MAX_BATCH_CONST) return SECPE_EINVAL;
    per_item = 1;
    for (int i = 0; i < B; i++) ka.k[i] = k[i];
    return SECPE_OK;
}

int launch_addconst(secpe_ctx *ctx, const CtB &x, const CtB &o, int nl, const std::vector<long long> &k) {
    KArr ka;
    int per = 0;
    SECPE_CHECK(fill_karr(ka, k, x.B, per));
    SECPE_LAUNCH(ctx, k_addconst, limb_grid(ctx->n, 2, (long long)x.B * 2 * nl), 256, 0, ctx->dev, x.data,
                 x.stride, x.cap, o.data, o.stride, o.cap, nl, ka, per);
    return SECPE_OK;
}

int launch_automorph(secpe_ctx *ctx, const CtB &x, const CtB &o, int nl, unsigned g) {
    SECPE_LAUNCH(ctx, k_automorph, limb_grid(ctx->n, 1, (long long)x.B * 2 * nl), 256, 0, ctx->dev, x.data,
                 x.stride, x.cap, o.data, o.stride, o.cap, nl, g);
    return SECPE_OK;
}

int launch_automorph_flat(secpe_ctx *ctx, const u64 *x, u64 *o, long long nlimbs, unsigned g) {
    if (nlimbs <= 0) return SECPE_OK;
    if (nlimbs > 65535) return SECPE_EINVAL;
    KprofScope kp(ctx, "ew_automorph", 16.0 * ctx->n * nlimbs);
    SECPE_LAUNCH(ctx, k_automorph_flat, limb_grid(ctx->n, 1, nlimbs), 256, 0, ctx->dev, x, o, g);
    return SECPE_OK;
}

int launch_rescale_prep(secpe_ctx *ctx, const u64 *y, u64 *z, int B, int lv) {
    SECPE_LAUNCH(ctx, k_rescale_prep, limb_grid(ctx->n, 2, (long long)B * 2 * lv), 256, 0, ctx->dev, y, z, lv);
    return SECPE_OK;
}

int launch_rescale_fin(secpe_ctx *ctx, const CtB &x, const u64 *z, const CtB &o, int lv) {
    SECPE_LAUNCH(ctx, k_rescale_fin, limb_grid(ctx->n, 2, (long long)x.B * 2 * lv), 256, 0, ctx->dev, x.data,
                 x.stride, x.cap, z, o.data, o.stride, o.cap, lv);
    return SECPE_OK;
}

int launch_modup_bconv(secpe_ctx *ctx, const u64 *x, u64 *ext, long long ext_item_stride, int ext_off,
                       int B, int lv, int j, int lo, int hi, int ntgt) {
    KprofScope kp(ctx, "modup_bconv", 8.0 * ctx->n * B * ((hi - lo) + ntgt));
    const int ngrp = (ntgt + BCONV_TG - 1) / BCONV_TG;
    const dim3 grid = limb_grid(ctx->n, 2, (long long)B * ngrp);
#define MODUP_CASE(ND)                                                                                   \
    case ND:                                                                                             \
        SECPE_LAUNCH(ctx, k_modup_bconv<ND>, grid, 256, 0, ctx->dev, x, ext, ext_item_stride, ext_off, lv, \
                     j, lo, hi, ntgt);                                                                   \
        break;
    switch (hi - lo) {
        MODUP_CASE(1)
        MODUP_CASE(2)
        MODUP_CASE(3)
        MODUP_CASE(4)
        MODUP_CASE(5)
        MODUP_CASE(6)
        MODUP_CASE(7)
        MODUP_CASE(8)
        default:
            SECPE_LAUNCH(ctx, k_modup_bconv<0>, grid, 256, 0, ctx->dev, x, ext, ext_item_stride, ext_off, lv, j,
                         lo, hi, ntgt);
    }
#undef MODUP_CASE
    return SECPE_OK;
}

int launch_ksk_ip(secpe_ctx *ctx, const u64 *d, long long d_item_stride, const u64 *ext,
                  long long ext_item_stride, const KsDigits &dg, const u64 *key, u64 *acc, int B, int lv,
                  unsigned gal) {
    if (ctx->tc_mode) {
        if (gal) return SECPE_EINVAL;
        return launch_ksk_ip_tc(ctx, d, d_item_stride, ext, ext_item_stride, dg, key, acc, B, lv);
    }
    const int nt = lv + 1 + ctx->npsp;
    // inputs (one residue per digit and target), key once, outputs (2 polys)
    KprofScope kp(ctx, "ksk_ip", 8.0 * ctx->n * ((double)B * dg.ndig * nt + 2.0 * dg.ndig * nt + 2.0 * B * nt));
    SECPE_LAUNCH(ctx, k_ksk_ip, limb_grid(ctx->n, 2, (long long)B * nt), 256, 0, ctx->dev, d, d_item_stride,
                 ext, ext_item_stride, dg, key, acc, lv, gal);
    return SECPE_OK;
}

int launch_moddown_bconv(secpe_ctx *ctx, const u64 *acc, u64 *conv, int B, int lv) {
    KprofScope kp(ctx, "moddown_bconv", 8.0 * ctx->n * B * 2.0 * (ctx->npsp + lv + 1));
    const int ngrp = (lv + 1 + BCONV_TG - 1) / BCONV_TG;
    const dim3 grid = limb_grid(ctx->n, 2, (long long)B * 2 * ngrp);
    switch (ctx->npsp) {
        case 1: SECPE_LAUNCH(ctx, k_moddown_bconv<1>, grid, 256, 0, ctx->dev, acc, conv, lv); break;
        case 2: SECPE_LAUNCH(ctx, k_moddown_bconv<2>, grid, 256, 0, ctx->dev, acc, conv, lv); break;
        case 4: SECPE_LAUNCH(ctx, k_moddown_bconv<4>, grid, 256, 0, ctx->dev, acc, conv, lv); break;
        default: SECPE_LAUNCH(ctx, k_moddown_bconv<0>, grid, 256, 0, ctx->dev, acc, conv, lv);
    }
    return SECPE_OK;
}

int launch_moddown_fin(secpe_ctx *ctx, const u64 *acc, const u64 *conv, const CtB &o, int lv, bool acc0,
                       bool acc1) {
    SECPE_LAUNCH(ctx, k_moddown_fin, limb_grid(ctx->n, 2, (long long)o.B * 2 * (lv + 1)), 256, 0, ctx->dev,
                 acc, conv, o.data, o.stride, o.cap, lv, acc0 ? 1 : 0, acc1 ? 1 : 0);
    return SECPE_OK;
}

int launch_sample_uniform(secpe_ctx *ctx, const std::vector<u64> &keys, u64 *out, long long item_stride,
                          const PrimeList &pl) {
    KeyArr ka;
    if ((int)keys.size() > SECPE_MAX_BATCH_CONST) return SECPE_EINVAL;
    for (size_t i = 0; i < keys.size(); i++) ka.k[i] = keys[i];
    SECPE_LAUNCH(ctx, k_sample_uniform, limb_grid(ctx->n, 1, (long long)keys.size() * pl.n), 256, 0, ctx->dev,
                 ka, out, item_stride, pl);
    return SECPE_OK;
}

int launch_sample_small(secpe_ctx *ctx, const std::vector<u64> &keys, long long *out, int kind) {
    KeyArr ka;
    if ((int)keys.size() > SECPE_MAX_BATCH_CONST) return SECPE_EINVAL;
    for (size_t i = 0; i < keys.size(); i++) ka.k[i] = keys[i];
    SECPE_LAUNCH(ctx, k_sample_small, limb_grid(ctx->n, 1, (long long)keys.size()), 256, 0, ctx->dev, ka, out,
                 kind);
    return SECPE_OK;
}

int launch_signed_to_limbs(secpe_ctx *ctx, const long long *m, const long long *e, u64 *out,
                           long long item_stride, int B, const PrimeList &pl) {
    SECPE_LAUNCH(ctx, k_signed_to_limbs, limb_grid(ctx->n, 1, (long long)B * pl.n), 256, 0, ctx->dev, m, e, out,
                 item_stride, pl);
    return SECPE_OK;
}

int launch_enc_finish(secpe_ctx *ctx, const u64 *M, long long ms, const u64 *a, long long as, const u64 *s,
                      const CtB &o, int nl) {
    SECPE_LAUNCH(ctx, k_enc_finish, limb_grid(ctx->n, 1, (long long)o.B * nl), 256, 0, ctx->dev, M, ms, a, as, s,
                 o.data, o.stride, o.cap, nl);
    return SECPE_OK;
}

int launch_dec_dot(secpe_ctx *ctx, const CtB &x, const u64 *s, u64 *m, int nl) {
    SECPE_LAUNCH(ctx, k_dec_dot, limb_grid(ctx->n, 1, (long long)x.B * nl), 256, 0, ctx->dev, x.data, x.stride,
                 x.cap, s, m, nl);
    return SECPE_OK;
}

int launch_crt_double(secpe_ctx *ctx, const u64 *m, int lv, double *out) {
    SECPE_LAUNCH(ctx, k_crt_double, limb_grid(ctx->n, 1, 1), 256, 0, ctx->dev, m, lv, out);
    return SECPE_OK;
}

int launch_crt_lift(secpe_ctx *ctx, const u64 *m, int lv, const long long *e, u64 *out,
                    long long out_item_stride, int ntop, int B) {
    SECPE_LAUNCH(ctx, k_crt_lift, limb_grid(ctx->n, 1, B), 256, 0, ctx->dev, m, lv, e, out, out_item_stride,
                 ntop);
    return SECPE_OK;
}

int launch_ksk_gen(secpe_ctx *ctx, const u64 *a, const u64 *e_ntt, const u64 *s, const u64 *sp,
                   const u64 *pmod, u64 *key, int lo, int hi) {
    SECPE_LAUNCH(ctx, k_ksk_gen, limb_grid(ctx->n, 1, ctx->nprimes), 256, 0, ctx->dev, a, e_ntt, s, sp, pmod,
                 key, lo, hi);
    return SECPE_OK;
}

int launch_from_mont(secpe_ctx *ctx, const u64 *in, u64 *out, int nlimb_total) {
    SECPE_LAUNCH(ctx, k_from_mont, limb_grid(ctx->n, 1, nlimb_total), 256, 0, ctx->dev, in, out, nlimb_total);
    return SECPE_OK;
}

int launch_limb_mul(secpe_ctx *ctx, const u64 *a, const u64 *b, u64 *o) {
    SECPE_LAUNCH(ctx, k_limb_mul, limb_grid(ctx->n, 1, ctx->nprimes), 256, 0, ctx->dev, a, b, o);
    return SECPE_OK;
}

int launch_limb_automorph(secpe_ctx *ctx, const u64 *in, u64 *o, unsigned g) {
    SECPE_LAUNCH(ctx, k_limb_automorph, limb_grid(ctx->n, 1, ctx->nprimes), 256, 0, ctx->dev, in, o, g);
    return SECPE_OK;
}

int launch_mdr_prep(secpe_ctx *ctx, const u64 *d, long long dis, long long dps, u64 *acc, int B, int lv) {
    SECPE_LAUNCH(ctx, k_mdr_prep, limb_grid(ctx->n, 2, (long long)B * 2), 256, 0, ctx->dev, d, dis, dps, acc, lv);
    return SECPE_OK;
}

int launch_mdr_bconv(secpe_ctx *ctx, const u64 *acc, u64 *conv, int B, int lv) {
    if (ctx->npsp + 1 > 9) return SECPE_EINVAL;
    SECPE_LAUNCH(ctx, k_mdr_bconv, limb_grid(ctx->n, 1, (long long)B * 2), 256, 0, ctx->dev, acc, conv, lv);
    return SECPE_OK;
}

int launch_mdr_fin(secpe_ctx *ctx, const u64 *acc, const u64 *conv, const u64 *d, long long dis, long long dps,
                   const CtB &o, int lv) {
    SECPE_LAUNCH(ctx, k_mdr_fin, limb_grid(ctx->n, 2, (long long)o.B * 2 * lv), 256, 0, ctx->dev, acc, conv, d,
                 dis, dps, o.data, o.stride, o.cap, lv);
    return SECPE_OK;
}

// ---------------------------------------------------------------- probe
namespace {
// Four independent multiply-accumulate chains per thread; each round feeds
// the high words back into the multiplicands so no round can be folded.
__global__ void __launch_bounds__(256) k_mul32_probe(int iters, u64 *sink) {
    const u64 t = (u64)blockIdx.x * 256u + threadIdx.x;
    u64 x0 = t * 0x9E3779B97F4A7C15ull + 1, x1 = x0 ^ 0xBF58476D1CE4E5B9ull, x2 = x0 ^ 0x94D049BB133111EBull,
        x3 = x0 ^ 0xD1B54A32D192ED03ull;
    const u64 y = 0xFFFFFFFFFFFFFFC5ull ^ t;
    acc128 a0 = {0, 0}, a1 = {1, 0}, a2 = {2, 0}, a3 = {3, 0};
    for (int i = 0; i < iters; i++) {
        mac(a0, x0, y);
        mac(a1, x1, y);
        mac(a2, x2, y);
        mac(a3, x3, y);
        x0 ^= a0.hi;
        x1 ^= a1.hi;
        x2 ^= a2.hi;
        x3 ^= a3.hi;
    }
    sink[t] = a0.lo ^ a0.hi ^ a1.lo ^ a1.hi ^ a2.lo ^ a2.hi ^ a3.lo ^ a3.hi;
}
}  // namespace

int launch_mul32_probe(secpe_ctx *ctx, unsigned blocks, int iters, u64 *sink) {
    SECPE_LAUNCH(ctx, k_mul32_probe, blocks, 256, 0, iters, sink);
    return SECPE_OK;
}
