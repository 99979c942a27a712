// Fused N = 2^16 NTT passes for key switching and rescale.
//
//  * k_colpass_bconv: forward pass A whose load computes a fast base
//    conversion (FastBConv) of coefficient-form source limbs to the target
//    prime on the fly:  v = sum_j [y_j + pre_j]_{p_j} * hat_{j,t} mod t,
//    minus post_t, where y_j = x_j * inv_j was already applied by the INTT
//    that produced the source (its final N^-1 is replaced by N^-1 inv_j).
//    It serves ModUp (source = one digit of d, inv_j = [Qhat_j^-1]), ModDown
//    (source = the special-prime limbs, inv_j = [Phat_j^-1], rounded by
//    pre_j = [floor(P/2) inv_j], post = floor(P/2)) and the rescale (source
//    = the last limb, inv = hat = 1, pre = post = floor(q_l/2)).  The
//    converted limb is never written before its first NTT pass.
//  * k_rowpass_epi: forward pass B whose store computes
//    out = (X - v) * w (+ out), the last step of ModDown (w = P^-1) and of
//    the rescale (w = q_l^-1).
//  * k_rowpass_ip: forward pass B of every digit's extended limb for one
//    target prime and tile, multiplied by the key-switching key (Montgomery
//    form) and accumulated in registers across digits: the key inner
//    product happens while the tile is on chip, and only the two
//    accumulated limbs are written.
#include "eval.h"
#include "ntt_core.cuh"

namespace {

struct BConvSrc {
    const u64 *base;  // source limb r of (item, poly) at base + item*is + poly*ps + r*N
    long long is, ps;
    int nsrc;
    int src_prime[16];
    u64 pre[16];         // added (mod the source prime) before the multiply-accumulate
    const u64 *hat;      // hat[r * hat_stride + target_prime] (Montgomery form)
    int hat_stride;
    const u64 *post;     // post[target_prime] or null
};

struct BConvArgs {
    DevCtx c;
    LimbSet ls;   // destination limbs (target primes), aux = source group
    int ngroups;
    BConvSrc g[12];
};

template <int NS, int MINB>
__global__ void __launch_bounds__(256, MINB) k_colpass_bconv(const __grid_constant__ BConvArgs a) {
    __shared__ u64 sm[4096];
    const long long lid = blockIdx.x >> 4;
    const int c0 = (blockIdx.x & 15) * 16;
    const int j = (int)(lid % a.ls.nlimb);
    const long long t2 = lid / a.ls.nlimb;
    const int poly = (int)(t2 % a.ls.npoly);
    const long long item = t2 / a.ls.npoly;
    const int li = poly * a.ls.nlimb + j;
    const int tp = a.ls.prime_of[li];
    const BConvSrc &S = a.g[a.ls.aux[li]];
    u64 *__restrict__ g = a.ls.base + item * a.ls.item_stride + poly * a.ls.poly_stride + (long long)j * a.c.n;
    const u64 *__restrict__ src = S.base + item * S.is + poly * S.ps;
    const u64 q = a.c.q[tp], qinv = a.c.qinv_neg[tp];
    const int ns = NS > 0 ? NS : S.nsrc;
    const int col = threadIdx.x & 15, u = threadIdx.x >> 4;
    u64 hat[NS > 0 ? NS : 16];
#pragma unroll
    for (int r = 0; r < ns; r++) hat[r] = S.hat[r * S.hat_stride + tp];
    const u64 post = S.post ? S.post[tp] : 0;
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) {
        const int e = ((k << 4) | u) * 256 + c0 + col;
        acc128 s = {0, 0};
#pragma unroll
        for (int r = 0; r < ns; r++) {
            const u64 pr = a.c.q[S.src_prime[r]];
            const u64 v = add_mod(src[(long long)r * a.c.n + e], S.pre[r], pr);
            mac(s, v, hat[r]);
        }
        x[k] = sub_mod(redc(s.hi, s.lo, q, qinv), post, q);
    }
    const ulonglong2 *tw = a.c.tw_fwd + (size_t)tp * a.c.n;
    fwd_round<8, 4>(x, u, tw, 1, q);
#pragma unroll
    for (int k = 0; k < 16; k++) sm[((k << 4) | u) * 16 + col] = x[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = sm[((u << 4) | k) * 16 + col];
    fwd_round<8, 0>(x, u << 4, tw, 1, q);
#pragma unroll
    for (int k = 0; k < 16; k++) g[((u << 4) | k) * 256 + c0 + col] = x[k];
}

struct EpiArgs {
    DevCtx c;
    LimbSet ls;        // pass-A output (lazy values), limb index = target prime
    const u64 *X;      // X limb i of (item, poly) at X + item*xis + poly*xps + i*N
    long long xis, xps;
    u64 *out;          // out limb i of (item, poly) at out + item*ois + poly*ops + i*N
    long long ois, ops;
    const ulonglong2 *w;  // w[target prime] Shoup pair
    int acc0, acc1;
    const u64 *Y;         // optional: + Y * w2 (Y limb i at Y + item*yis + poly*yps + i*N)
    long long yis, yps;
    const ulonglong2 *w2;
    int has_cadd;         // optional: + cadd[target prime] on polynomial 0 (a constant polynomial)
    u64 cadd[SECPE_MAX_PRIMES];
};

// Dynamic shared memory: the padded transform tile (16 x 272 words), the
// X tile (4096 words, fetched by one bulk copy while the tile is
// transformed) and the copy's mbarrier.
constexpr int EPI_SMEM = (16 * 272 + 4096) * 8 + 16;

__global__ void __launch_bounds__(256, 3) k_rowpass_epi(const __grid_constant__ EpiArgs a) {
    extern __shared__ __align__(16) u64 dsm[];
    u64 *sm = dsm;
    u64 *xs = dsm + 16 * 272;
    uint64_t *bar = reinterpret_cast<uint64_t *>(xs + 4096);
    const long long lid = blockIdx.x >> 4;
    const int r0 = (blockIdx.x & 15) * 16;
    const int j = (int)(lid % a.ls.nlimb);
    const long long t2 = lid / a.ls.nlimb;
    const int poly = (int)(t2 % a.ls.npoly);
    const long long item = t2 / a.ls.npoly;
    const int tp = a.ls.prime_of[poly * a.ls.nlimb + j];
    const u64 *__restrict__ g =
        a.ls.base + item * a.ls.item_stride + poly * a.ls.poly_stride + (long long)j * a.c.n + (size_t)r0 * 256;
    const u64 q = a.c.q[tp];
    const int u = threadIdx.x & 15, row = threadIdx.x >> 4;
    const int base = 256 + r0 + row;
    u64 *__restrict__ srow = sm + row * 272;
    const ulonglong2 *tw = a.c.tw_fwd + (size_t)tp * a.c.n;
    const u64 *__restrict__ X = a.X + item * a.xis + poly * a.xps + (long long)j * a.c.n + (size_t)r0 * 256;
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    // the X tile (32 KiB, contiguous) streams into shared memory while the
    // tile is transformed; the other epilogue operand is fetched to L2
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar, 4096 * 8);
        bulk_g2s(xs, X, 4096 * 8, bar);
    }
    if (a.Y)
        prefetch_tile_l2(a.Y + item * a.yis + poly * a.yps + (long long)j * a.c.n + (size_t)r0 * 256);
    else if (poly == 0 ? a.acc0 : a.acc1)
        prefetch_tile_l2(a.out + item * a.ois + poly * a.ops + (long long)j * a.c.n + (size_t)r0 * 256);
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = g[row * 256 + ((k << 4) | u)];
    fwd_round<8, 4>(x, u, tw, base, q);
#pragma unroll
    for (int k = 0; k < 16; k++) srow[PADR((k << 4) | u)] = x[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = srow[PADR((u << 4) | k)];
    fwd_round<8, 0>(x, u << 4, tw, base, q);
#pragma unroll
    for (int k = 0; k < 16; k++) srow[PADR((u << 4) | k)] = reduce4(x[k], q);
    __syncthreads();
    if (!mbar_wait(bar, 0)) {
        if (threadIdx.x == 0) atomicCAS(a.c.status, 0, SECPE_ETIMEOUT);
        mbar_wait(bar, 0);  // the copy may still be landing in this CTA's shared memory
        return;
    }
    u64 *__restrict__ O = a.out + item * a.ois + poly * a.ops + (long long)j * a.c.n + (size_t)r0 * 256;
    const ulonglong2 w = a.w[tp];
    const bool acc = poly == 0 ? a.acc0 : a.acc1;
    const u64 cadd = (a.has_cadd && poly == 0) ? a.cadd[tp] : 0;
    if (a.Y) {
        const u64 *__restrict__ Y = a.Y + item * a.yis + poly * a.yps + (long long)j * a.c.n + (size_t)r0 * 256;
        const ulonglong2 w2 = a.w2[tp];
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const int e = threadIdx.x + 256 * i;
            const int r = e >> 8, p = e & 255;
            const u64 v = sm[r * 272 + PADR(p)];
            u64 res = add_mod(mul_shoup(sub_mod(xs[e], v, q), w.x, w.y, q), mul_shoup(Y[e], w2.x, w2.y, q), q);
            if (cadd) res = add_mod(res, cadd, q);
            O[e] = res;
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const int e = threadIdx.x + 256 * i;
        const int r = e >> 8, p = e & 255;
        const u64 v = sm[r * 272 + PADR(p)];
        u64 res = mul_shoup(sub_mod(xs[e], v, q), w.x, w.y, q);
        if (acc) res = add_mod(res, O[e], q);
        if (cadd) res = add_mod(res, cadd, q);
        O[e] = res;
    }
}

struct IpArgs {
    DevCtx c;
    const u64 *d;      // d limb t of item at d + item*dis + t*N (NTT form)
    long long dis;
    const u64 *ext;    // pass-A output: item stride eis, digit j target tt at (off_j + tt)*N
    long long eis;
    KsDigits dg;
    const u64 *key;    // [dnum][2][nprimes][N] Montgomery form
    u64 *acc;          // [item][2][nt][N]
    int lv, nitem;
};

// grid: ((t * 16 + tile) * nitem + item): the items sharing a key tile run back to back.
// The two accumulators live in the output tile itself (the first digit
// writes it, later digits read, add and write it back): the CTA touches its
// 64 KiB of output repeatedly within its lifetime, so it stays in L2, and the
// registers stay free for the transform (3 CTAs per SM, no spills).
__global__ void __launch_bounds__(256, 3) k_rowpass_ip(const __grid_constant__ IpArgs a) {
    __shared__ u64 sm[16 * 272];
    const int nt = a.lv + 1 + a.c.np_special;
    const int item = blockIdx.x % a.nitem;
    const int tt16 = blockIdx.x / a.nitem;
    const int tile = tt16 & 15, t = tt16 >> 4;
    const int r0 = tile * 16;
    const int pt = t <= a.lv ? t : a.c.nq + (t - a.lv - 1);
    const u64 q = a.c.q[pt], qinv = a.c.qinv_neg[pt];
    const int u = threadIdx.x & 15, row = threadIdx.x >> 4;
    const int base = 256 + r0 + row;
    u64 *__restrict__ srow = sm + row * 272;
    const ulonglong2 *tw = a.c.tw_fwd + (size_t)pt * a.c.n;
    const long long kpoly = (long long)a.c.nprimes * a.c.n;
    const long long tile_off = (long long)r0 * 256;
    u64 *__restrict__ o0 = a.acc + (long long)item * 2 * nt * a.c.n + (long long)t * a.c.n + tile_off;
    u64 *__restrict__ o1 = o0 + (long long)nt * a.c.n;
    for (int jd = 0; jd < a.dg.ndig; jd++) {
        const int lo = a.dg.lo[jd], hi = a.dg.hi[jd];
        const u64 *kb = a.key + (long long)jd * 2 * kpoly + (long long)pt * a.c.n + tile_off;
        prefetch_tile_l2(kb);
        prefetch_tile_l2(kb + kpoly);
        const bool own = t >= lo && t < hi;
        if (!own) {
            const int ti = t < lo ? t : t - (hi - lo);
            const u64 *g = a.ext + item * a.eis + (long long)(a.dg.off[jd] + ti) * a.c.n + tile_off;
            u64 x[16];
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] = g[row * 256 + ((k << 4) | u)];
            fwd_round<8, 4>(x, u, tw, base, q);
#pragma unroll
            for (int k = 0; k < 16; k++) srow[PADR((k << 4) | u)] = x[k];
            __syncthreads();
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] = srow[PADR((u << 4) | k)];
            fwd_round<8, 0>(x, u << 4, tw, base, q);
#pragma unroll
            for (int k = 0; k < 16; k++) srow[PADR((u << 4) | k)] = reduce4(x[k], q);
            __syncthreads();
        }
        const u64 *src = a.d + item * a.dis + (long long)t * a.c.n + tile_off;
        // four elements at a time: every load of the group is issued before
        // the first product, so up to 20 loads per thread are in flight
#pragma unroll
        for (int i0 = 0; i0 < 16; i0 += 4) {
            u64 v[4], k0[4], k1[4], a0[4], a1[4];
#pragma unroll
            for (int b = 0; b < 4; b++) {
                const int e = threadIdx.x + 256 * (i0 + b);
                v[b] = own ? src[e] : sm[(e >> 8) * 272 + PADR(e & 255)];
                k0[b] = kb[e];
                k1[b] = kb[kpoly + e];
                a0[b] = jd ? o0[e] : 0;
                a1[b] = jd ? o1[e] : 0;
            }
#pragma unroll
            for (int b = 0; b < 4; b++) {
                const int e = threadIdx.x + 256 * (i0 + b);
                u64 p0 = mont_mul(v[b], k0[b], q, qinv);
                u64 p1 = mont_mul(v[b], k1[b], q, qinv);
                if (jd) {
                    p0 = add_mod(p0, a0[b], q);
                    p1 = add_mod(p1, a1[b], q);
                }
                o0[e] = p0;
                o1[e] = p1;
            }
        }
        if (!own) __syncthreads();
    }
}

template <int MINB>
int launch_bconv_ns(secpe_ctx *ctx, const BConvArgs &a, int ns, unsigned grid) {
    static const char *const names[10] = {"k_colpass_bconv<0>", "k_colpass_bconv<1>", "k_colpass_bconv<2>",
                                          "k_colpass_bconv<3>", "k_colpass_bconv<4>", "k_colpass_bconv<5>",
                                          "k_colpass_bconv<6>", "k_colpass_bconv<7>", "k_colpass_bconv<8>",
                                          "k_colpass_bconv<9>"};
    void (*kf)(BConvArgs) = nullptr;
    switch (ns) {
        case 1: kf = k_colpass_bconv<1, MINB>; break;
        case 2: kf = k_colpass_bconv<2, MINB>; break;
        case 3: kf = k_colpass_bconv<3, MINB>; break;
        case 4: kf = k_colpass_bconv<4, MINB>; break;
        case 5: kf = k_colpass_bconv<5, MINB>; break;
        case 6: kf = k_colpass_bconv<6, MINB>; break;
        case 7: kf = k_colpass_bconv<7, MINB>; break;
        case 8: kf = k_colpass_bconv<8, MINB>; break;
        case 9: kf = k_colpass_bconv<9, MINB>; break;
        default: kf = k_colpass_bconv<0, MINB>; ns = 0;
    }
    SECPE_LAUNCH_AS(ctx, names[ns], kf, grid, 256, 0, a);
    return SECPE_OK;
}

int launch_colpass_bconv(secpe_ctx *ctx, const BConvArgs &a) {
    const long long nl = (long long)a.ls.nitem * a.ls.npoly * a.ls.nlimb;
    if (nl == 0) return SECPE_OK;
    int ns = a.g[0].nsrc;
    for (int i = 1; i < a.ngroups; i++)
        if (a.g[i].nsrc != ns) ns = 0;
    const unsigned grid = (unsigned)(nl * 16);
    // reads and writes intermediates of its operation only (algorithmic 0);
    // per residue: one multiply-accumulate per source, a reduction, a pass
    double mul = 0.0;
    for (int li = 0; li < a.ls.npoly * a.ls.nlimb; li++)
        mul += MUL32_MAC * a.g[a.ls.aux[li]].nsrc + MUL32_REDC + MUL32_PASS;
    mul *= (double)ctx->n * a.ls.nitem;
    KprofScope kp(ctx, "ntt16_colpass_bconv", 0.0, 16.0 * ctx->n * nl, mul);
    if (ctx->tune.ctas[TUNE_BCONV] == 4) return launch_bconv_ns<4>(ctx, a, ns, grid);
    return launch_bconv_ns<3>(ctx, a, ns, grid);
}

// Self-test of the bounded device wait used by the bulk-copy kernels: one
// CTA arms an mbarrier for one arrival and, when `arrive`, performs it; every
// thread then waits with the same bounded wait (at most `polls` polls).  A
// wait that runs out records SECPE_ETIMEOUT in the status word and the kernel
// returns; nothing is in flight.
__global__ void k_wait_selftest(const __grid_constant__ DevCtx c, int arrive, long polls) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (arrive && threadIdx.x == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar)) : "memory");
    const bool ok = mbar_wait(&bar, 0, polls);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicCAS(c.status, 0, SECPE_ETIMEOUT);
}

}  // namespace

// ---------------------------------------------------------------- host side
bool fused_path(const secpe_ctx *ctx) { return ctx->log_n == 16 && !ctx->tc_mode; }

int wait_selftest(secpe_ctx *ctx, int arrive, long polls) {
    if (polls < 1 || polls > SECPE_WAIT_LIMIT) return SECPE_EINVAL;
    SECPE_LAUNCH(ctx, k_wait_selftest, 1, 128, 0, ctx->dev, arrive ? 1 : 0, polls);
    return SECPE_OK;
}

// One base-conversion pass of the ModUp shape (alpha sources) over `nitem`
// items of [alpha + ntgt] limbs at buf, for timing candidate launch
// configurations (the data may be anything below the primes).
int bconv_pass_probe(secpe_ctx *ctx, u64 *buf, int nitem, int ntgt) {
    const int n = ctx->n, ns = ctx->alpha;
    if (ns < 1 || ns > 16 || ntgt < 1 || ntgt > SECPE_MAX_LIMBSET) return SECPE_EINVAL;
    BConvArgs a;
    a.c = ctx->dev;
    a.ngroups = 1;
    BConvSrc &S = a.g[0];
    S.base = buf;
    S.is = (long long)(ns + ntgt) * n;
    S.ps = 0;
    S.nsrc = ns;
    for (int r = 0; r < ns; r++) {
        S.src_prime[r] = r;
        S.pre[r] = 0;
    }
    S.hat = ctx->dev.mu_hat;
    S.hat_stride = ctx->nprimes;
    S.post = nullptr;
    a.ls = make_limbset(buf + (size_t)ns * n, nitem, S.is, 1, 0, ntgt, 0);
    for (int j = 0; j < ntgt; j++) a.ls.prime_of[j] = (int8_t)((ns + j) % ctx->nprimes);
    return launch_colpass_bconv(ctx, a);
}

// ModUp + inner product for N = 2^16: pass A with the digit's base
// conversion as prologue into ext, then pass B of every digit fused with the
// key inner product into acc [B][2][nt][N].
int modup_ip_fused(secpe_ctx *ctx, const u64 *d, long long d_item_stride, const u64 *dcoef, int B, int lv,
                   const KsDigits &dg, int tot, const u64 *key, u64 *ext, u64 *acc) {
    const int n = ctx->n, nt = lv + 1 + ctx->npsp;
    if (dg.ndig > 12) return SECPE_EINVAL;
    BConvArgs a;
    a.c = ctx->dev;
    a.ngroups = dg.ndig;
    a.ls.base = ext;
    a.ls.nitem = B;
    a.ls.item_stride = (long long)tot * n;
    a.ls.npoly = 1;
    a.ls.poly_stride = 0;
    a.ls.nlimb = tot;
    int e = 0;
    for (int j = 0; j < dg.ndig; j++) {
        BConvSrc &S = a.g[j];
        const int lo = dg.lo[j], hi = dg.hi[j];
        S.base = dcoef + (size_t)lo * n;
        S.is = (long long)(lv + 1) * n;
        S.ps = 0;
        S.nsrc = hi - lo;
        const size_t tb = ((size_t)lv * ctx->dnum + j) * ctx->alpha;
        for (int r = 0; r < S.nsrc; r++) {
            S.src_prime[r] = lo + r;
            S.pre[r] = 0;
        }
        S.hat = ctx->dev.mu_hat + tb * ctx->nprimes;
        S.hat_stride = ctx->nprimes;
        S.post = nullptr;
        for (int t = 0; t < nt; t++) {
            if (t >= lo && t < hi) continue;
            a.ls.prime_of[e] = (int8_t)(t <= lv ? t : ctx->nq + (t - lv - 1));
            a.ls.aux[e] = (int8_t)j;
            e++;
        }
    }
    const int last = dg.ndig - 1;
    if (dg.ndig > 1 && a.g[last].nsrc != a.g[0].nsrc) {
        // the partial last digit gets its own launch so both use a
        // compile-time source count
        BConvArgs b = a;
        b.ngroups = 1;
        b.g[0] = a.g[last];
        b.ls.base = ext + (size_t)dg.off[last] * n;
        b.ls.nlimb = tot - dg.off[last];
        for (int i = 0; i < b.ls.nlimb; i++) {
            b.ls.prime_of[i] = a.ls.prime_of[dg.off[last] + i];
            b.ls.aux[i] = 0;
        }
        a.ngroups = last;
        a.ls.nlimb = dg.off[last];
        SECPE_CHECK(launch_colpass_bconv(ctx, a));
        SECPE_CHECK(launch_colpass_bconv(ctx, b));
    } else {
        SECPE_CHECK(launch_colpass_bconv(ctx, a));
    }
    IpArgs ip;
    ip.c = ctx->dev;
    ip.d = d;
    ip.dis = d_item_stride;
    ip.ext = ext;
    ip.eis = (long long)tot * n;
    ip.dg = dg;
    ip.key = key;
    ip.acc = acc;
    ip.lv = lv;
    ip.nitem = B;
    // algorithmic: the key-switching key, read once for the batch (d and
    // the accumulators are the operation's input, charged to its INTT, and
    // intermediates); per target residue: a pass B per digit not holding
    // the target prime, two Montgomery products per digit
    const int k = ctx->npsp;
    const double ip_mul = (double)n * B *
                          (MUL32_PASS * ((double)(lv + 1) * (dg.ndig - 1) + (double)k * dg.ndig) +
                           2.0 * MUL32_MONT * dg.ndig * nt);
    KprofScope kp(ctx, "ntt16_rowpass_ip", 8.0 * n * 2.0 * dg.ndig * nt,
                  8.0 * n * ((double)B * (tot + lv + 1) + 2.0 * dg.ndig * nt + 2.0 * B * nt), ip_mul);
    SECPE_LAUNCH(ctx, k_rowpass_ip, (unsigned)((long long)nt * 16 * B), 256, 0, ip);
    return SECPE_OK;
}

// out (+)= (X - NTT(FastBConv(src))) * w [+ Y * w2] over limbs 0..nl-1 of B items x 2 polys.
// x_input: X is an input of the operation (rescale), not an intermediate
// (the profiler charges it as algorithmic bytes only then).
int bconv_ntt_epi(secpe_ctx *ctx, const BConvSrc &S, int B, int nl, u64 *tmp, const u64 *X, long long xis,
                  long long xps, const CtB &out, const ulonglong2 *w, bool acc0, bool acc1, bool x_input,
                  const u64 *Y = nullptr, long long yis = 0, long long yps = 0, const ulonglong2 *w2 = nullptr,
                  const long long *add_k = nullptr) {
    const int n = ctx->n;
    BConvArgs a;
    a.c = ctx->dev;
    a.ngroups = 1;
    a.g[0] = S;
    a.ls = make_limbset(tmp, B, 2ll * nl * n, 2, (long long)nl * n, nl, 0);
    SECPE_CHECK(launch_colpass_bconv(ctx, a));
    EpiArgs ep;
    ep.c = ctx->dev;
    ep.ls = a.ls;
    ep.X = X;
    ep.xis = xis;
    ep.xps = xps;
    ep.out = out.data;
    ep.ois = out.stride;
    ep.ops = out.pstride();
    ep.w = w;
    ep.acc0 = acc0 ? 1 : 0;
    ep.acc1 = acc1 ? 1 : 0;
    ep.Y = Y;
    ep.yis = yis;
    ep.yps = yps;
    ep.w2 = w2;
    ep.has_cadd = add_k ? 1 : 0;
    if (add_k) {
        // the constant k as a residue of every output prime (output limb j is prime j)
        if (nl > SECPE_MAX_PRIMES) return SECPE_EINVAL;
        for (int j = 0; j < nl; j++) {
            const u64 q = ctx->primes[j];
            const u64 m = (u64)(*add_k < 0 ? -(*add_k) : *add_k) % q;
            ep.cadd[j] = (*add_k < 0 && m) ? q - m : m;
        }
    }
    const long long nlimbs = (long long)B * 2 * nl;
    // algorithmic per item: the output (2 nl limbs), X when it is an input,
    // the accumulated output polynomials' old values, and Y with the two
    // top limbs of its polynomials that the preceding steps consumed
    const double alg = 8.0 * n * B *
                       (2.0 * nl + (x_input ? 2.0 * nl : 0.0) + (acc0 ? nl : 0) + (acc1 ? nl : 0) +
                        (Y ? 2.0 * (nl + 1) : 0.0));
    const double epi_mul = (double)n * nlimbs * (MUL32_PASS + MUL32_SHOUP * (Y ? 2.0 : 1.0));
    KprofScope kp(ctx, "ntt16_rowpass_epi", alg, 8.0 * n * nlimbs * (acc0 || acc1 ? 4.0 : 3.0), epi_mul);
    // the bulk copy of the X tile needs 16-byte aligned tiles
    if (((uintptr_t)X & 15) || (xis & 1) || (xps & 1)) return SECPE_EINVAL;
    static bool attr_set[64];
    int dev = 0;
    SECPE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SECPE_ECUDA;
    if (!attr_set[dev]) {
        SECPE_CUDA(cudaFuncSetAttribute(k_rowpass_epi, cudaFuncAttributeMaxDynamicSharedMemorySize, EPI_SMEM));
        attr_set[dev] = true;
    }
    SECPE_LAUNCH(ctx, k_rowpass_epi, (unsigned)(nlimbs * 16), 256, EPI_SMEM, ep);
    return SECPE_OK;
}

// ModDown of acc [B][2][nt][N] (special limbs already INTT'd) into out.
int moddown_fused(secpe_ctx *ctx, const u64 *acc, int B, int lv, const CtB &out, bool acc0, bool acc1, u64 *tmp) {
    const int n = ctx->n, nt = lv + 1 + ctx->npsp, k = ctx->npsp;
    BConvSrc S;
    S.base = acc + (size_t)(lv + 1) * n;
    S.is = 2ll * nt * n;
    S.ps = (long long)nt * n;
    S.nsrc = k;
    for (int j = 0; j < k; j++) {
        const u64 pj = ctx->primes[ctx->nq + j];
        u64 prod = 1;
        for (int j2 = 0; j2 < k; j2++)
            if (j2 != j) prod = hm::mulmod(prod, ctx->primes[ctx->nq + j2] % pj, pj);
        const u64 inv = hm::invmod(prod, pj);
        S.src_prime[j] = ctx->nq + j;
        // [floor(P/2) * inv]_{p_j}: the source limbs already carry the factor inv
        u64 pm = 1;
        for (int j2 = 0; j2 < k; j2++) pm = hm::mulmod(pm, ctx->primes[ctx->nq + j2] % pj, pj);
        S.pre[j] = hm::mulmod(hm::mulmod((pm + pj - 1) % pj, hm::invmod(2, pj), pj), inv, pj);
    }
    S.hat = ctx->dev.md_hat;
    S.hat_stride = ctx->nq;
    S.post = ctx->dev.md_hP;
    return bconv_ntt_epi(ctx, S, B, lv + 1, tmp, acc, 2ll * nt * n, (long long)nt * n, out, ctx->dev.md_pinv, acc0,
                         acc1, false);
}

// Rescale of `in` by q_l into out, y = INTT of the last limb [B][2][N].
int rescale_fused(secpe_ctx *ctx, const CtB &in, const u64 *y, const CtB &out, u64 *tmp, const long long *add_k) {
    const int n = ctx->n, lv = in.level;
    BConvSrc S;
    S.base = y;
    S.is = 2ll * n;
    S.ps = n;
    S.nsrc = 1;
    S.src_prime[0] = lv;
    S.pre[0] = ctx->primes[lv] / 2;
    S.hat = ctx->dev.mont_one;
    S.hat_stride = 0;
    S.post = ctx->dev.rs_hmod + (size_t)lv * ctx->nq;
    return bconv_ntt_epi(ctx, S, in.B, lv, tmp, in.data, in.stride, in.pstride(), out,
                         ctx->dev.rs_qinv + (size_t)lv * ctx->nq, false, false, true, nullptr, 0, 0, nullptr, add_k);
}

// Relinearisation's ModDown fused with the rescale: acc [B][2][nt][N] from
// the key inner product, d = the 3-component tensor [B][3][lv+1][N]; acc's
// limbs lv..lv+k are the sources (q_l limb replaced by P d_l + acc_l, the
// INTT applies the FastBConv pre-multipliers); out at level lv-1.
int moddown_rescale_fused(secpe_ctx *ctx, u64 *acc, const u64 *d, int B, int lv, const CtB &out, u64 *tmp) {
    const int n = ctx->n, nt = lv + 1 + ctx->npsp, k = ctx->npsp, ks = k + 1;
    const long long dis = 3ll * (lv + 1) * n, dps = (long long)(lv + 1) * n;
    SECPE_CHECK(launch_mdr_prep(ctx, d, dis, dps, acc, B, lv));
    LimbSet src = make_limbset(acc + (size_t)lv * n, B, 2ll * nt * n, 2, (long long)nt * n, ks, 0);
    for (int p = 0; p < 2; p++)
        for (int j = 0; j < ks; j++) src.prime_of[p * ks + j] = (int8_t)(j == 0 ? lv : ctx->nq + j - 1);
    SECPE_CHECK(ntt_limbset(ctx, src, true, nullptr, ctx->dev.mdr_ninv, lv * ks, 0.0));  // intermediate
    BConvSrc S;
    S.base = acc + (size_t)lv * n;
    S.is = 2ll * nt * n;
    S.ps = (long long)nt * n;
    S.nsrc = ks;
    for (int j = 0; j < ks; j++) {
        S.src_prime[j] = j == 0 ? lv : ctx->nq + j - 1;
        S.pre[j] = ctx->h_mdr_pre_scaled[(size_t)lv * ks + j];
    }
    S.hat = ctx->dev.mdr_hat + (size_t)lv * ks * ctx->nq;
    S.hat_stride = ctx->nq;
    S.post = ctx->dev.mdr_post + (size_t)lv * ctx->nq;
    return bconv_ntt_epi(ctx, S, B, lv, tmp, acc, 2ll * nt * n, (long long)nt * n, out,
                         ctx->dev.mdr_w + (size_t)lv * ctx->nq, false, false, false, d, dis, dps,
                         ctx->dev.rs_qinv + (size_t)lv * ctx->nq);
}
