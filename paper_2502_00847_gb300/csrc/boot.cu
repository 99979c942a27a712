// CKKS bootstrapping (SecPE Sec. 2.2 and Sec. 4.1 rely on it to restore a
// ciphertext's levels; the paper does not describe it).  Reading: the
// sparse-slot bootstrapping of Cheon, Han, Kim, Kim and Song (2018) with
// the sub-sum of Chen, Chillotti and Song (2019), for a sparse secret and a
// block of n slots (2n <= N/2), on the batched evaluator:
//
//  1. ModRaise: limb 0 of (c0, c1) to coefficient form, centred lift mod
//     q0, residues modulo q_0..q_L, NTT: decrypts to t = m + q0 I; the label
//     becomes q0 (N/2) / n.
//  2. SubSum: y <- y + RotL(y, s), s = n, 2n, .., N/4 (the n-periodic block
//     sum; the polynomial (N/2n) Pi(t) on the subring in X^(N/2n)).
//  3. CoeffToSlot: u = p / q0 of the 2n subring coefficients p into slots
//     [0, n) and [n, 2n) of every 2n-block, from w and its conjugate, as a
//     baby-step giant-step sum of plaintext diagonals (A for w, B for its
//     conjugate; (p_lo + i p_hi)/q0 = V^H w / n, V[j][a] = omega^(a 5^j),
//     omega = exp(i pi / 2n)).
//  4. EvalMod: sin(2 pi u) as cos(2 pi (u - 1/4) / 2^8) by its degree-12
//     Taylor polynomial in y = x^2 (P0(y) + y^3 P1(y)) and 8 double angles.
//  5. SlotToCoeff: slots (q0 / 2 pi) V (f_lo + i f_hi) / label, the block
//     average of the input's slots, with the input's label: an n-periodic
//     input comes back unchanged.
//
// Levels: the top 16 primes (CoeffToSlot 1, EvalMod 14, SlotToCoeff 1);
// the output is at level L - 16.  Every operation is the batched evaluator's
// (one launch per kernel for the whole batch), in the order the CPU oracle
// takes them, so results are bit-identical given the same plaintexts.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

#include "eval.h"

namespace enc {
bool encode_complex_fft(int n, const double *re, const double *im, int nv, double scale, std::vector<long long> &m);
}  // namespace enc

namespace {
constexpr int kDoublings = 8;      // double angles after the Taylor polynomial
constexpr int kTaylorTerms = 7;    // cos(x) = sum_{k < 7} (-1)^k x^(2k) / (2k)!
constexpr int kBootLevels = 16;    // CoeffToSlot 1 + EvalMod 14 + SlotToCoeff 1
using cplx = std::complex<double>;

void bsgs_split(int n_diag, int &bs, int &gs) {
    int lg = 0;
    while ((1 << (lg + 1)) <= n_diag) lg++;
    bs = 1 << ((lg + 1) / 2);
    gs = n_diag / bs;
}
}  // namespace

struct secpe_boot {
    secpe_ctx *ctx = nullptr;
    int n = 0, S = 0, bs1 = 0, gs1 = 0, bs2 = 0, gs2 = 0, L = 0, lf = 0;
    double lambda_u = 0.0, lambda_f = 0.0;
    u64 *c2s = nullptr;  // [2][n][L+1][N]  (A then B), diagonal g bs + b shifted by g bs, Montgomery NTT form
    u64 *s2c = nullptr;  // [2n][lf+1][N]
};

namespace {

// The labels of the EvalMod input (the CoeffToSlot output) and output, by
// the evaluator's own scale arithmetic (the same double operations as the
// run: products multiply labels and rescales divide by the prime, linear
// combinations land on their target exactly).
void predict_labels(const secpe_ctx *ctx, int n, double &lambda_u, double &lambda_f, int &lf) {
    const int L = ctx->L;
    auto q = [&](int l) { return (double)ctx->primes[l]; };
    lambda_u = (double)ctx->primes[0] * (double)(ctx->n / 2) / (double)n;
    const double wl = q(L);
    int lv = L - 1;                      // u
    double x = wl;                       // x at lv - 1
    lv -= 1;
    double y = x * x / q(lv);            // y at lv - 1
    lv -= 1;
    double y2 = y * y / q(lv);
    lv -= 1;
    double y3 = y2 * y / q(lv);
    lv -= 1;                             // y3 at L - 5
    const int lp1 = lv - 1;
    const double t1 = wl * q(lp1) / y3;
    double c = y3 * t1 / q(lp1);         // the product, at lp1 - 1
    lv = lp1 - 1;
    for (int i = 0; i < kDoublings; i++) {
        c = c * c / q(lv);
        lv -= 1;
    }
    lambda_f = c;
    lf = lv;
}

// The CoeffToSlot and SlotToCoeff diagonals (complex slot vectors over N/2
// slots), in the order the plan stores them.
void boot_diagonals(const secpe_ctx *ctx, int n, std::vector<std::vector<cplx>> &c2s,
                    std::vector<std::vector<cplx>> &s2c) {
    const int S = ctx->n / 2;
    const double pi = 3.14159265358979323846;
    std::vector<cplx> V((size_t)n * n);
    for (int j = 0; j < n; j++) {
        long long e = 1;
        for (int t = 0; t < j; t++) e = e * 5 % (4ll * n);
        for (int a = 0; a < n; a++) {
            const double th = pi * (double)((e * a) % (4ll * n)) / (2.0 * n);
            V[(size_t)j * n + a] = cplx(std::cos(th), std::sin(th));
        }
    }
    // A (2n x n) for w, B (2n x n) for its conjugate; G = V^H / n
    std::vector<cplx> A((size_t)2 * n * n), B((size_t)2 * n * n);
    const cplx two(2.0, 0.0), two_i(0.0, 2.0);
    for (int j = 0; j < n; j++)
        for (int a = 0; a < n; a++) {
            const cplx g = std::conj(V[(size_t)a * n + j]) / (double)n;
            A[(size_t)j * n + a] = g / two;
            A[(size_t)(j + n) * n + a] = g / two_i;
            B[(size_t)j * n + a] = std::conj(g) / two;
            B[(size_t)(j + n) * n + a] = -std::conj(g) / two_i;
        }
    int bs, gs;
    bsgs_split(n, bs, gs);
    c2s.assign(2 * (size_t)n, std::vector<cplx>(S));
    for (int t = 0; t < 2; t++)
        for (int k = 0; k < n; k++) {
            const int sh = (k / bs) * bs;
            const std::vector<cplx> &Mx = t == 0 ? A : B;
            for (int j = 0; j < S; j++) {
                const int src = ((j - sh) % S + S) % S;  // RotR by g bs
                c2s[(size_t)t * n + k][j] = Mx[(size_t)(src % (2 * n)) * n + (src + k) % n];
            }
        }
    // SlotToCoeff: M (n x 2n) = [H, i H], H = (q0 / 2 pi) V
    const double h = (double)ctx->primes[0] / (2.0 * pi);
    bsgs_split(2 * n, bs, gs);
    s2c.assign(2 * (size_t)n, std::vector<cplx>(S));
    for (int k = 0; k < 2 * n; k++) {
        const int sh = (k / bs) * bs;
        for (int j = 0; j < S; j++) {
            const int src = ((j - sh) % S + S) % S;
            const int r = src % n, a = (src + k) % (2 * n);
            const cplx v = h * V[(size_t)r * n + (a % n)];
            s2c[k][j] = a < n ? v : cplx(0.0, 1.0) * v;
        }
    }
}

}  // namespace

namespace {

// ModRaise: coefficient-form limb 0 (mod q0) of both polynomials of B items,
// lo [B][2][N], centred and reduced modulo q_0..q_(nl-1) into out
// [B][2][nl][N] (coefficient form).
__global__ void k_mod_raise(DevCtx c, const u64 *lo, u64 *out, int nl) {
    const int li = blockIdx.y;
    const int p = li % nl, kk = (li / nl) & 1, item = li / (2 * nl);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= c.n) return;
    const u64 q0 = c.q[0], q = c.q[p];
    const u64 x = lo[((long long)item * 2 + kk) * c.n + e];
    u64 r;
    if (x > q0 / 2) {
        const u64 m = q0 - x;  // |centred value|
        const u64 mr = m % q;
        r = mr ? q - mr : 0;
    } else {
        r = x % q;
    }
    out[(((long long)item * 2 + kk) * nl + p) * c.n + e] = r;
}

// sum_k diag_k (.) RotL(x_t, k) over the inputs x_t, as
// sum_g RotL(sum_{t,b} P_{t, g bs + b} (.) RotL(x_t, b), g bs), every inner
// sum rescaled once; plaintexts pts [t][ndiag][lv+1][N] at pt_scale; the
// output label is out_scale when > 0.
int bsgs(Eval &E, const std::vector<Ct> &xs, const u64 *pts, int ndiag, int bs, int gs, double pt_scale,
         double out_scale, Ct &out) {
    secpe_ctx *ctx = E.ctx;
    const int lv = xs[0].level(), B = xs[0].B();
    const size_t plane = (size_t)(lv + 1) * ctx->n;
    std::vector<std::vector<Ct>> baby(xs.size());
    for (size_t t = 0; t < xs.size(); t++) {
        // the baby steps of one input share one ModUp (hoisting)
        std::vector<int> steps;
        for (int b = 1; b < bs; b++) steps.push_back(b);
        std::vector<Ct> r;
        SECPE_CHECK(E.rotate_hoisted(xs[t], steps, r));
        baby[t].push_back(xs[t]);
        for (Ct &c : r) baby[t].push_back(c);
    }
    // the inner sums over every input and baby step: with at most
    // kMaxPlainTerms terms, kMaxGiant giant steps per pass (each baby step
    // read once per pass); otherwise one pass per giant step and term chunk
    std::vector<CtB> terms;
    for (size_t t = 0; t < xs.size(); t++)
        for (int b = 0; b < bs; b++) terms.push_back(baby[t][b].v);
    auto pt_of = [&](size_t k, int g) {
        const size_t t = k / bs, b = k % bs;
        return (const u64 *)(pts + ((size_t)t * ndiag + (size_t)g * bs + b) * plane);
    };
    std::vector<Ct> accs(gs);
    for (int g = 0; g < gs; g++) SECPE_CHECK(ct_alloc(ctx, B, lv, xs[0].scale() * pt_scale, accs[g]));
    if ((int)terms.size() <= kMaxPlainTerms) {
        for (int g0 = 0; g0 < gs; g0 += kMaxGiant) {
            const int g1 = std::min(gs, g0 + kMaxGiant);
            std::vector<std::vector<const u64 *>> ps(terms.size());
            std::vector<CtB> os;
            for (size_t k = 0; k < terms.size(); k++)
                for (int g = g0; g < g1; g++) ps[k].push_back(pt_of(k, g));
            for (int g = g0; g < g1; g++) os.push_back(accs[g].v);
            SECPE_CHECK(launch_bsgs_inner(ctx, terms, ps, os, lv + 1));
        }
    } else {
        for (int g = 0; g < gs; g++)
            for (size_t t0 = 0; t0 < terms.size(); t0 += kMaxPlainTerms) {
                const size_t t1 = std::min(terms.size(), t0 + kMaxPlainTerms);
                std::vector<const u64 *> tps;
                for (size_t k = t0; k < t1; k++) tps.push_back(pt_of(k, g));
                SECPE_CHECK(launch_mul_plain_sum(ctx, std::vector<CtB>(terms.begin() + t0, terms.begin() + t1), tps,
                                                 accs[g].v, lv + 1, t0 > 0));
            }
    }
    baby.clear();
    Ct total;
    for (int g = 0; g < gs; g++) {
        Ct acc = accs[g];
        accs[g] = Ct();
        Ct inner;
        SECPE_CHECK(E.rescale(acc, inner));
        acc = Ct();
        if (out_scale > 0.0) inner.v.scale = out_scale;
        if (g) {
            Ct r;
            SECPE_CHECK(E.rotate(inner, g * bs, r));
            inner = r;
        }
        if (!total.buf) {
            total = inner;
        } else {
            Ct s;
            SECPE_CHECK(E.add(total, inner, s));
            total = s;
        }
    }
    out = total;
    return SECPE_OK;
}

int check_boot(const secpe_ctx *ctx) {
    if (ctx->p.boot_primes < kBootLevels || ctx->p.secret_hw < 1 || ctx->p.secret_hw > 32) return SECPE_EINVAL;
    if (ctx->L - kBootLevels < 1 + ctx->p.reserve) return SECPE_ELEVEL;
    return SECPE_OK;
}

}  // namespace

int boot_block(const secpe_boot *bt) { return bt->n; }

int boot_out_level(const secpe_ctx *ctx) { return ctx->L - kBootLevels; }

// Bootstrapping of a batch (labels kept, output at level L - 16).
int boot_batch(secpe_ctx *ctx, const secpe_keys *keys, const secpe_boot *bt, const Ct &in, Ct &out) {
    const int L = ctx->L, n = ctx->n, B = in.B();
    Eval E{ctx, keys, {}, 0};
    // 1. ModRaise
    DevBuf lo;
    SECPE_CHECK(lo.alloc(ctx, sizeof(u64) * (size_t)B * 2 * n));
    LimbSet src = make_limbset(in.v.data, B, in.v.stride, 2, in.v.pstride(), 1, 0);
    LimbSet dst = make_limbset(lo.u(), B, 2ll * n, 2, n, 1, 0);
    SECPE_CHECK(ntt_limbset(ctx, dst, true, &src));
    Ct x;
    SECPE_CHECK(ct_alloc(ctx, B, L, bt->lambda_u, x));
    SECPE_LAUNCH(ctx, k_mod_raise, dim3((unsigned)((n + 255) / 256), (unsigned)(B * 2 * (L + 1))), 256, 0, ctx->dev,
                 lo.u(), x.v.data, L + 1);
    lo.release();
    LimbSet xl = make_limbset(x.v.data, B, x.v.stride, 2, x.v.pstride(), L + 1, 0);
    SECPE_CHECK(ntt_limbset(ctx, xl, false));
    // 2. SubSum
    for (int s = bt->n; s < bt->S; s <<= 1) {
        Ct r, a;
        SECPE_CHECK(E.rotate(x, s, r));
        SECPE_CHECK(E.add(x, r, a));
        x = a;
    }
    // 3. CoeffToSlot
    Ct wc, u;
    SECPE_CHECK(E.rotate(x, SECPE_STEP_CONJ, wc));
    SECPE_CHECK(bsgs(E, {x, wc}, bt->c2s, bt->n, bt->bs1, bt->gs1, (double)ctx->primes[L], 0.0, u));
    x = Ct();
    wc = Ct();
    // 4. EvalMod
    const double pi = 3.14159265358979323846;
    const double wl = (double)ctx->primes[L];
    const double a = 2.0 * pi / (double)(1 << kDoublings);
    double c[kTaylorTerms];
    double fact = 1.0;
    for (int k = 0; k < kTaylorTerms; k++) {
        if (k) fact *= (double)(2 * k - 1) * (double)(2 * k);
        c[k] = (k % 2 ? -1.0 : 1.0) / fact;
    }
    Ct x0, xx, y, y2, y3;
    SECPE_CHECK(E.mul_const(u, {a}, wl, u.level() - 1, x0));
    u = Ct();
    SECPE_CHECK(E.add_const(x0, -a / 4.0, xx));
    x0 = Ct();
    SECPE_CHECK(E.mul(xx, xx, y));
    xx = Ct();
    SECPE_CHECK(E.mul(y, y, y2));
    SECPE_CHECK(E.mul(y2, y, y3));
    const int lp1 = y3.level() - 1;
    const double t1 = wl * (double)ctx->primes[lp1] / y3.scale();
    Ct l1, l2, l12, p1, t3, prod, l0, p0, cs;
    SECPE_CHECK(E.lincomb({&y, &y2}, {{c[4]}, {c[5]}}, t1, lp1, l1));
    SECPE_CHECK(E.lincomb({&y3}, {{c[6]}}, t1, lp1, l2));
    SECPE_CHECK(E.add(l1, l2, l12));
    SECPE_CHECK(E.add_const(l12, c[3], p1));
    l1 = l2 = l12 = Ct();
    SECPE_CHECK(E.tensor(y3, p1, t3));
    SECPE_CHECK(E.relin_rescale(t3, prod));
    t3 = p1 = y3 = Ct();
    SECPE_CHECK(E.lincomb({&y, &y2}, {{c[1]}, {c[2]}}, prod.scale(), prod.level(), l0));
    SECPE_CHECK(E.add_const(l0, c[0], p0));
    y = y2 = l0 = Ct();
    SECPE_CHECK(E.add(prod, p0, cs));
    for (int i = 0; i < kDoublings; i++) {
        Ct d, dd, e2;
        SECPE_CHECK(E.mul(cs, cs, d));
        SECPE_CHECK(E.add(d, d, dd));
        SECPE_CHECK(E.add_const(dd, -1.0, e2));
        cs = e2;
    }
    // 5. SlotToCoeff, with the input's label
    const double pt_scale = (double)ctx->primes[cs.level()] / cs.scale();
    return bsgs(E, {cs}, bt->s2c, 2 * bt->n, bt->bs2, bt->gs2, pt_scale, in.scale(), out);
}

namespace {

secpe_boot *new_plan(secpe_ctx *ctx, int n) {
    secpe_boot *bt = new secpe_boot();
    bt->ctx = ctx;
    bt->n = n;
    bt->S = ctx->n / 2;
    bt->L = ctx->L;
    bsgs_split(n, bt->bs1, bt->gs1);
    bsgs_split(2 * n, bt->bs2, bt->gs2);
    predict_labels(ctx, n, bt->lambda_u, bt->lambda_f, bt->lf);
    return bt;
}

// 2n <= N/2, written as n <= N/4 so that no n near 2^30 overflows
bool block_ok(const secpe_ctx *ctx, int n) { return n >= 2 && (n & (n - 1)) == 0 && n <= ctx->n / 4; }

}  // namespace

extern "C" int secpe_boot_rotation_steps(const secpe_ctx *ctx, int n, int32_t *steps, int capacity, int *count) {
    if (!ctx || !count || !block_ok(ctx, n)) return SECPE_EINVAL;
    std::vector<int32_t> v;
    v.push_back(SECPE_STEP_CONJ);
    for (int s = n; s < ctx->n / 2; s <<= 1) v.push_back(s);
    for (int nd : {n, 2 * n}) {
        int bs, gs;
        bsgs_split(nd, bs, gs);
        for (int b = 1; b < bs; b++) v.push_back(b);
        for (int g = 1; g < gs; g++) v.push_back(g * bs);
    }
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    *count = (int)v.size();
    if (steps) {
        if (capacity < (int)v.size()) return SECPE_EINVAL;
        std::memcpy(steps, v.data(), sizeof(int32_t) * v.size());
    }
    return SECPE_OK;
}

extern "C" int secpe_boot_create_coeffs(secpe_ctx *ctx, int n, const int64_t *c2s_m, const int64_t *s2c_m,
                                        secpe_boot **out) {
    if (!ctx || !c2s_m || !s2c_m || !out || !block_ok(ctx, n)) return SECPE_EINVAL;
    SECPE_CHECK(check_boot(ctx));
    secpe_boot *bt = new_plan(ctx, n);
    const size_t N = ctx->n;
    int st = SECPE_OK;
    if (cudaMalloc(&bt->c2s, sizeof(u64) * 2 * (size_t)n * (bt->L + 1) * N) != cudaSuccess ||
        cudaMalloc(&bt->s2c, sizeof(u64) * 2 * (size_t)n * (bt->lf + 1) * N) != cudaSuccess) {
        cudaGetLastError();
        st = SECPE_ENOMEM;
    }
    ctx->stream = 0;
    if (st == SECPE_OK) st = upload_plain(ctx, c2s_m, 2 * n, bt->L + 1, true, bt->c2s);
    if (st == SECPE_OK) st = upload_plain(ctx, s2c_m, 2 * n, bt->lf + 1, true, bt->s2c);
    if (st != SECPE_OK) {
        secpe_boot_destroy(bt);
        return st;
    }
    *out = bt;
    return SECPE_OK;
}

extern "C" int secpe_boot_create(secpe_ctx *ctx, int n, secpe_boot **out) {
    if (!ctx || !out || !block_ok(ctx, n)) return SECPE_EINVAL;
    SECPE_CHECK(check_boot(ctx));
    double lu, lf_scale;
    int lf;
    predict_labels(ctx, n, lu, lf_scale, lf);
    std::vector<std::vector<cplx>> c2s, s2c;
    boot_diagonals(ctx, n, c2s, s2c);
    const int N = ctx->n, S = N / 2;
    std::vector<int64_t> c2s_m((size_t)2 * n * N), s2c_m((size_t)2 * n * N);
    std::vector<double> re(S), im(S);
    std::vector<long long> m;
    auto enc = [&](const std::vector<cplx> &z, double scale, int64_t *dst) {
        for (int j = 0; j < S; j++) {
            re[j] = z[j].real();
            im[j] = z[j].imag();
        }
        if (!enc::encode_complex_fft(N, re.data(), im.data(), S, scale, m)) return false;
        std::memcpy(dst, m.data(), sizeof(int64_t) * N);
        return true;
    };
    for (size_t k = 0; k < c2s.size(); k++)
        if (!enc(c2s[k], (double)ctx->primes[ctx->L], c2s_m.data() + k * N)) return SECPE_EINVAL;
    const double s2c_scale = (double)ctx->primes[lf] / lf_scale;
    for (size_t k = 0; k < s2c.size(); k++)
        if (!enc(s2c[k], s2c_scale, s2c_m.data() + k * N)) return SECPE_EINVAL;
    return secpe_boot_create_coeffs(ctx, n, c2s_m.data(), s2c_m.data(), out);
}

extern "C" void secpe_boot_destroy(secpe_boot *bt) {
    if (!bt) return;
    cudaDeviceSynchronize();
    if (bt->c2s) cudaFree(bt->c2s);
    if (bt->s2c) cudaFree(bt->s2c);
    delete bt;
}

extern "C" int secpe_bootstrap_batch(secpe_ctx *ctx, const secpe_keys *keys, const secpe_boot *bt,
                                     const secpe_ctbatch *in, secpe_ctbatch *out, void *stream) {
    if (!ctx || !keys || !bt || bt->ctx != ctx || !in || !out || !in->data || !out->data) return SECPE_EINVAL;
    const int n = ctx->n, L = ctx->L, lo = L - kBootLevels;
    if (in->batch < 1 || in->batch > SECPE_MAX_BATCH_CONST || in->level < 0 || in->level > L ||
        in->cap < in->level + 1 || in->stride < 2ull * in->cap * n || !(in->scale > 0.0) || !aligned16(in->data) ||
        (in->stride & 1))
        return SECPE_EINVAL;
    if (out->cap < lo + 1 || out->stride < 2ull * out->cap * n || !aligned16(out->data) || (out->stride & 1))
        return SECPE_EINVAL;
    ctx->stream = (cudaStream_t)stream;
    Ct x;
    x.v.data = (u64 *)in->data;
    x.v.B = in->batch;
    x.v.cap = in->cap;
    x.v.stride = (long long)in->stride;
    x.v.level = in->level;
    x.v.scale = in->scale;
    x.v.n = n;
    Ct r;
    SECPE_CHECK(boot_batch(ctx, keys, bt, x, r));
    CtB o;
    o.data = (u64 *)out->data;
    o.B = in->batch;
    o.cap = out->cap;
    o.stride = (long long)out->stride;
    o.level = r.level();
    o.scale = r.scale();
    o.n = n;
    for (int b = 0; b < in->batch; b++)
        SECPE_CUDA(cudaMemcpy2DAsync(o.data + (size_t)b * o.stride, sizeof(u64) * o.cap * n,
                                     r.v.data + (size_t)b * r.v.stride, sizeof(u64) * r.v.cap * n,
                                     sizeof(u64) * (r.level() + 1) * n, 2, cudaMemcpyDeviceToDevice, ctx->stream));
    out->batch = in->batch;
    out->level = r.level();
    out->scale = r.scale();
    return cudaGetLastError() == cudaSuccess ? SECPE_OK : SECPE_ECUDA;
}

extern "C" int secpe_bootstrap(secpe_ctx *ctx, const secpe_keys *keys, const secpe_boot *bt, const secpe_ct *in,
                               secpe_ct *out, void *stream) {
    if (!in || !out) return SECPE_EINVAL;
    secpe_ctbatch bi = {in->data, 1, in->cap, in->level, in->scale, 2ull * in->cap * (uint64_t)(ctx ? ctx->n : 0)};
    secpe_ctbatch bo = {out->data, 1, out->cap, 0, 0.0, 2ull * out->cap * (uint64_t)(ctx ? ctx->n : 0)};
    SECPE_CHECK(secpe_bootstrap_batch(ctx, keys, bt, &bi, &bo, stream));
    out->level = bo.level;
    out->scale = bo.scale;
    return SECPE_OK;
}
