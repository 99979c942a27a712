// The encrypted linear step ahead of the ensemble aggregation: CLIP-style
// prompt ensembling (SecPE Sec. 2.3) scores an encrypted image embedding
// x = I(x_in) (d values) against the plaintext text embeddings of every
// prompt template i and class c, y_i[c] = <T_i[c], x>, and aggregates the K
// logit vectors y_i before the Argmax (Sec. 3.1 step 3).
//
// Layout (a reading: the paper gives the formula, not the packing).  The
// user encrypts x with x[j] repeated in the C' slots [j C', (j+1) C')
// (d C' <= N/2, d a power of two).  For prompt i the server multiplies by
// the plaintext W_i with T_i[c][j] at slot j C' + c, then adds log2(d)
// rotations by C' 2^t (t = 0..log2 d - 1), after which slot c < C' holds
// sum_j T_i[c][j] x[j]; a plaintext mask keeps slots [0, C) and a plaintext
// pad puts d_min in [C, C'): the result is the layout secpe_encrypt_logits
// produces, ready for secpe_argmax_batch.  Two levels (the two plaintext
// products, each rescaled with exact scale bookkeeping: W_i is encoded at
// scale q_l, the mask at scale q_(l-1), so the output keeps the input's
// scale), log2(d) rotations per prompt, batched over the K prompts.
#include <cmath>
#include <cstring>

#include "eval.h"
#include "modarith.cuh"

namespace enc {
bool encode_real_fft(int n, const double *v, int nv, double scale, std::vector<long long> &m);
}  // namespace enc

struct secpe_linear {
    secpe_ctx *ctx = nullptr;
    int K = 0, C = 0, cp = 0, d = 0, level = 0;
    u64 *W = nullptr;     // [K][level+1][N] Montgomery NTT form (scale q_level)
    u64 *mask = nullptr;  // [level][N]      Montgomery NTT form (scale q_(level-1))
    u64 *pad = nullptr;   // [level-1][N]    NTT form (scale Delta)
};

namespace {

// o = x (.) p per residue; x item b at x + b*xs (xs may be 0: one input for
// every item), plaintext limb i of item b at p + b*ps + i*N in Montgomery
// form (ps may be 0: one plaintext for every item).
__global__ void k_mul_plain(DevCtx c, const u64 *x, long long xs, int cap_x, const u64 *p, long long ps, u64 *o,
                            long long os, int cap_o, int nl, int acc) {
    const int li = blockIdx.y;
    const int i = li % nl, kk = (li / nl) & 1, item = li / (2 * nl);
    const int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= c.n) return;
    const u64 q = c.q[i], qi = c.qinv_neg[i];
    const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(x + item * xs + ((long long)kk * cap_x + i) * c.n + e);
    const ulonglong2 w = *reinterpret_cast<const ulonglong2 *>(p + item * ps + (long long)i * c.n + e);
    ulonglong2 r;
    r.x = mont_mul(v.x, w.x, q, qi);
    r.y = mont_mul(v.y, w.y, q, qi);
    ulonglong2 *op = reinterpret_cast<ulonglong2 *>(o + item * os + ((long long)kk * cap_o + i) * c.n + e);
    if (acc) {
        const ulonglong2 prev = *op;
        r.x = add_mod(r.x, prev.x, q);
        r.y = add_mod(r.y, prev.y, q);
    }
    *op = r;
}

// o (+)= sum_t x_t (.) p_t per residue (the inner sums of a baby-step
// giant-step linear transform): plaintext p_t limb i at p_t + i*N in
// Montgomery form, one for every item.  The products are summed in 128 bits
// and reduced every 15 of them (15 q^2 < q 2^64 for q < 2^60), the partial
// results added mod q, so the result equals the sequence of k_mul_plain
// accumulations residue for residue.
struct PlainSumArgs {
    const u64 *x[kMaxPlainTerms];
    long long xs[kMaxPlainTerms];
    int cap[kMaxPlainTerms];
    const u64 *p[kMaxPlainTerms];
    int nt;
};

__global__ void k_mul_plain_sum(DevCtx c, const __grid_constant__ PlainSumArgs a, u64 *o, long long os, int cap_o,
                                int nl, int acc) {
    const int li = blockIdx.y;
    const int i = li % nl, kk = (li / nl) & 1, item = li / (2 * nl);
    const int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= c.n) return;
    const u64 q = c.q[i], qi = c.qinv_neg[i];
    ulonglong2 *op = reinterpret_cast<ulonglong2 *>(o + item * os + ((long long)kk * cap_o + i) * c.n + e);
    ulonglong2 r = acc ? *op : make_ulonglong2(0, 0);
    acc128 s0 = {0, 0}, s1 = {0, 0};
    int cnt = 0;
#pragma unroll 4
    for (int t = 0; t < a.nt; t++) {
        const ulonglong2 v =
            *reinterpret_cast<const ulonglong2 *>(a.x[t] + item * a.xs[t] + ((long long)kk * a.cap[t] + i) * c.n + e);
        const ulonglong2 w = *reinterpret_cast<const ulonglong2 *>(a.p[t] + (long long)i * c.n + e);
        mac(s0, v.x, w.x);
        mac(s1, v.y, w.y);
        if (++cnt == 15) {
            r.x = add_mod(r.x, redc(s0.hi, s0.lo, q, qi), q);
            r.y = add_mod(r.y, redc(s1.hi, s1.lo, q, qi), q);
            s0 = s1 = acc128{0, 0};
            cnt = 0;
        }
    }
    if (cnt) {
        r.x = add_mod(r.x, redc(s0.hi, s0.lo, q, qi), q);
        r.y = add_mod(r.y, redc(s1.hi, s1.lo, q, qi), q);
    }
    *op = r;
}

// The inner sums of up to kMaxGiant giant steps in one pass:
// o_g = sum_k x_k (.) p_{k,g}, every baby-step ciphertext x_k read once for
// all of them.  One residue per thread; rows ordered limb-major, so the rows
// that share one limb's plaintexts run back to back and find them in L2.
// Products summed in 128 bits, reduced every 15 (as k_mul_plain_sum).
struct BsgsInnerArgs {
    const u64 *x[kMaxPlainTerms];
    long long xs[kMaxPlainTerms];
    int cap[kMaxPlainTerms];
    const u64 *p[kMaxPlainTerms][kMaxGiant];
    u64 *o[kMaxGiant];
    long long os;
    int cap_o, nt, ng, B;
};

__global__ void k_bsgs_inner(DevCtx c, const __grid_constant__ BsgsInnerArgs a) {
    const int li = blockIdx.y;
    const int i = li / (2 * a.B), rem = li % (2 * a.B);
    const int item = rem >> 1, kk = rem & 1;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= c.n) return;
    const u64 q = c.q[i], qi = c.qinv_neg[i];
    const long long off = (long long)i * c.n + e;
    acc128 sm[kMaxGiant];
    u64 r[kMaxGiant];
#pragma unroll
    for (int g = 0; g < kMaxGiant; g++) {
        sm[g] = acc128{0, 0};
        r[g] = 0;
    }
    int cnt = 0;
    for (int k = 0; k < a.nt; k++) {
        const u64 v = a.x[k][item * a.xs[k] + ((long long)kk * a.cap[k] + i) * c.n + e];
#pragma unroll
        for (int g = 0; g < kMaxGiant; g++)
            if (g < a.ng) mac(sm[g], v, a.p[k][g][off]);
        if (++cnt == 15) {
#pragma unroll
            for (int g = 0; g < kMaxGiant; g++) {
                r[g] = add_mod(r[g], redc(sm[g].hi, sm[g].lo, q, qi), q);
                sm[g] = acc128{0, 0};
            }
            cnt = 0;
        }
    }
#pragma unroll
    for (int g = 0; g < kMaxGiant; g++) {
        if (g >= a.ng) break;
        if (cnt) r[g] = add_mod(r[g], redc(sm[g].hi, sm[g].lo, q, qi), q);
        a.o[g][item * a.os + ((long long)kk * a.cap_o + i) * c.n + e] = r[g];
    }
}

// o = x + (p, 0): plaintext limbs (NTT form) added to c0 of every item.
__global__ void k_add_plain(DevCtx c, const u64 *x, long long xs, int cap_x, const u64 *p, u64 *o, long long os,
                            int cap_o, int nl) {
    const int li = blockIdx.y;
    const int i = li % nl, kk = (li / nl) & 1, item = li / (2 * nl);
    const int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= c.n) return;
    const u64 q = c.q[i];
    ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(x + item * xs + ((long long)kk * cap_x + i) * c.n + e);
    if (kk == 0) {
        const ulonglong2 w = *reinterpret_cast<const ulonglong2 *>(p + (long long)i * c.n + e);
        v.x = add_mod(v.x, w.x, q);
        v.y = add_mod(v.y, w.y, q);
    }
    *reinterpret_cast<ulonglong2 *>(o + item * os + ((long long)kk * cap_o + i) * c.n + e) = v;
}

// p <- p 2^64 mod q (Montgomery form), nl limbs of each of B plaintexts
__global__ void k_to_mont(DevCtx c, u64 *p, long long ps, int nl) {
    const int li = blockIdx.y;
    const int i = li % nl, item = li / nl;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= c.n) return;
    u64 *a = p + item * ps + (long long)i * c.n + e;
    *a = mont_mul(*a, c.r2[i], c.q[i], c.qinv_neg[i]);
}

dim3 grid_of(int n, int per_thread, long long rows) {
    return dim3((unsigned)((n / per_thread + 255) / 256), (unsigned)rows);
}

}  // namespace

// B plaintexts from int64 coefficients m[B][N] (host): residues of limbs
// 0..nl-1 in NTT form, optionally in Montgomery form, at dst [B][nl][N].
int upload_plain(secpe_ctx *ctx, const int64_t *m, int B, int nl, bool mont, u64 *dst) {
    const int n = ctx->n;
    DevBuf dm;
    SECPE_CHECK(dm.alloc(ctx, sizeof(int64_t) * (size_t)B * n));
    SECPE_CUDA(cudaMemcpyAsync(dm.p, m, sizeof(int64_t) * (size_t)B * n, cudaMemcpyHostToDevice, ctx->stream));
    PrimeList pl;
    pl.n = nl;
    for (int i = 0; i < nl; i++) pl.p[i] = i;
    for (int b = 0; b < B; b++)
        SECPE_CHECK(launch_signed_to_limbs(ctx, (const long long *)dm.p + (size_t)b * n, nullptr,
                                           dst + (size_t)b * nl * n, 0, 1, pl));
    LimbSet ls = make_limbset(dst, B, (long long)nl * n, 1, 0, nl, 0);
    SECPE_CHECK(ntt_limbset(ctx, ls, false));
    if (mont) SECPE_LAUNCH(ctx, k_to_mont, grid_of(n, 1, (long long)B * nl), 256, 0, ctx->dev, dst, (long long)nl * n, nl);
    // the host buffer may be released when the call returns
    SECPE_CUDA(cudaStreamSynchronize(ctx->stream));
    return SECPE_OK;
}

namespace {

int pow2_ceil(int C) {
    int cp = 1;
    while (cp < C) cp <<= 1;
    return cp;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

int launch_mul_plain(secpe_ctx *ctx, const CtB &x, long long xs, const u64 *p, long long ps, const CtB &o, int nl,
                     bool acc) {
    KprofScope kp(ctx, "ew_mul_plain", 8.0 * ctx->n * o.B * ((acc ? 6.0 : 4.0) * nl + (ps ? (double)nl : 0.0)));
    SECPE_LAUNCH(ctx, k_mul_plain, grid_of(ctx->n, 2, (long long)o.B * 2 * nl), 256, 0, ctx->dev, x.data, xs, x.cap,
                 p, ps, o.data, o.stride, o.cap, nl, acc ? 1 : 0);
    return SECPE_OK;
}

int launch_mul_plain_sum(secpe_ctx *ctx, const std::vector<CtB> &xs, const std::vector<const u64 *> &ps,
                         const CtB &o, int nl, bool acc) {
    const int nt = (int)xs.size();
    if (nt < 1 || nt > kMaxPlainTerms || (int)ps.size() != nt) return SECPE_EINVAL;
    PlainSumArgs a;
    for (int t = 0; t < nt; t++) {
        if (xs[t].B != o.B || xs[t].cap < nl) return SECPE_EINVAL;
        a.x[t] = xs[t].data;
        a.xs[t] = xs[t].stride;
        a.cap[t] = xs[t].cap;
        a.p[t] = ps[t];
    }
    a.nt = nt;
    KprofScope kp(ctx, "ew_mul_plain_sum",
                  8.0 * ctx->n * nl * ((double)o.B * (2.0 * nt + (acc ? 4.0 : 2.0)) + (double)nt));
    SECPE_LAUNCH(ctx, k_mul_plain_sum, grid_of(ctx->n, 2, (long long)o.B * 2 * nl), 256, 0, ctx->dev, a, o.data,
                 o.stride, o.cap, nl, acc ? 1 : 0);
    return SECPE_OK;
}

int launch_bsgs_inner(secpe_ctx *ctx, const std::vector<CtB> &xs, const std::vector<std::vector<const u64 *>> &ps,
                      const std::vector<CtB> &os, int nl) {
    const int nt = (int)xs.size(), ng = (int)os.size();
    if (nt < 1 || nt > kMaxPlainTerms || ng < 1 || ng > kMaxGiant || (int)ps.size() != nt) return SECPE_EINVAL;
    BsgsInnerArgs a;
    const int B = os[0].B;
    for (int k = 0; k < nt; k++) {
        if (xs[k].B != B || xs[k].cap < nl || (int)ps[k].size() != ng) return SECPE_EINVAL;
        a.x[k] = xs[k].data;
        a.xs[k] = xs[k].stride;
        a.cap[k] = xs[k].cap;
        for (int g = 0; g < ng; g++) a.p[k][g] = ps[k][g];
    }
    for (int g = 0; g < ng; g++) {
        if (os[g].B != B || os[g].stride != os[0].stride || os[g].cap != os[0].cap || os[g].cap < nl)
            return SECPE_EINVAL;
        a.o[g] = os[g].data;
    }
    a.os = os[0].stride;
    a.cap_o = os[0].cap;
    a.nt = nt;
    a.ng = ng;
    a.B = B;
    KprofScope kp(ctx, "ew_bsgs_inner", 8.0 * ctx->n * nl * ((double)B * 2.0 * (nt + ng) + (double)nt * ng));
    SECPE_LAUNCH(ctx, k_bsgs_inner, grid_of(ctx->n, 1, (long long)B * 2 * nl), 256, 0, ctx->dev, a);
    return SECPE_OK;
}

int launch_add_plain(secpe_ctx *ctx, const CtB &x, const u64 *p, const CtB &o, int nl) {
    SECPE_LAUNCH(ctx, k_add_plain, grid_of(ctx->n, 2, (long long)o.B * 2 * nl), 256, 0, ctx->dev, x.data, x.stride,
                 x.cap, p, o.data, o.stride, o.cap, nl);
    return SECPE_OK;
}

namespace {

CtB view_ct(const secpe_ctx *ctx, const secpe_ct *c) {
    CtB v;
    v.data = (u64 *)c->data;
    v.B = 1;
    v.cap = c->cap;
    v.stride = 2ll * c->cap * ctx->n;
    v.level = c->level;
    v.scale = c->scale;
    v.n = ctx->n;
    return v;
}

bool ct_ok(const secpe_ctx *ctx, const secpe_ct *c) {
    return c && c->data && aligned16(c->data) && c->level >= 0 && c->level <= ctx->L && c->cap >= c->level + 1 &&
           c->scale > 0.0;
}

}  // namespace

extern "C" int secpe_linear_create_coeffs(secpe_ctx *ctx, const int64_t *W_m, const int64_t *mask_m,
                                          const int64_t *pad_m, int K, int C, int d, secpe_linear **out) {
    if (!ctx || !W_m || !mask_m || !pad_m || !out || K < 1 || K > SECPE_MAX_BATCH_CONST || C < 1 || !is_pow2(d) ||
        C > ctx->n / 2)
        return SECPE_EINVAL;
    const int cp = pow2_ceil(C), L = ctx->L, n = ctx->n;
    if ((long long)d * cp > n / 2) return SECPE_EINVAL;
    if (L < 2 + ctx->p.reserve + 1) return SECPE_ELEVEL;
    secpe_linear *lin = new secpe_linear();
    lin->ctx = ctx;
    lin->K = K;
    lin->C = C;
    lin->cp = cp;
    lin->d = d;
    lin->level = L;
    int st = SECPE_OK;
    if (cudaMalloc(&lin->W, sizeof(u64) * (size_t)K * (L + 1) * n) != cudaSuccess ||
        cudaMalloc(&lin->mask, sizeof(u64) * (size_t)L * n) != cudaSuccess ||
        cudaMalloc(&lin->pad, sizeof(u64) * (size_t)(L - 1) * n) != cudaSuccess) {
        cudaGetLastError();
        st = SECPE_ENOMEM;
    }
    ctx->stream = 0;
    if (st == SECPE_OK) st = upload_plain(ctx, W_m, K, L + 1, true, lin->W);
    if (st == SECPE_OK) st = upload_plain(ctx, mask_m, 1, L, true, lin->mask);
    if (st == SECPE_OK) st = upload_plain(ctx, pad_m, 1, L - 1, false, lin->pad);
    if (st != SECPE_OK) {
        secpe_linear_destroy(lin);
        return st;
    }
    *out = lin;
    return SECPE_OK;
}

extern "C" int secpe_linear_create(secpe_ctx *ctx, const double *T, int K, int C, int d, double d_min,
                                   secpe_linear **out) {
    if (!ctx || !T || !out || K < 1 || C < 1 || !is_pow2(d) || C > ctx->n / 2) return SECPE_EINVAL;
    const int cp = pow2_ceil(C), L = ctx->L, n = ctx->n;
    if ((long long)d * cp > n / 2 || L < 2) return SECPE_EINVAL;
    const int nv = d * cp;
    std::vector<double> v(nv);
    std::vector<long long> m;
    std::vector<int64_t> Wm((size_t)K * n), mask(n), pad(n);
    for (int i = 0; i < K; i++) {
        for (int j = 0; j < d; j++)
            for (int c = 0; c < cp; c++) v[(size_t)j * cp + c] = c < C ? T[((size_t)i * C + c) * d + j] : 0.0;
        if (!enc::encode_real_fft(n, v.data(), nv, (double)ctx->primes[L], m)) return SECPE_EINVAL;
        std::memcpy(Wm.data() + (size_t)i * n, m.data(), sizeof(int64_t) * n);
    }
    std::vector<double> mv(cp, 0.0), pv(cp, 0.0);  // mask: 1 on the C logits; pad: d_min above them
    for (int c = 0; c < cp; c++) {
        if (c < C)
            mv[c] = 1.0;
        else
            pv[c] = d_min;
    }
    if (!enc::encode_real_fft(n, mv.data(), cp, (double)ctx->primes[L - 1], m)) return SECPE_EINVAL;
    std::memcpy(mask.data(), m.data(), sizeof(int64_t) * n);
    if (!enc::encode_real_fft(n, pv.data(), cp, ctx->scale, m)) return SECPE_EINVAL;
    std::memcpy(pad.data(), m.data(), sizeof(int64_t) * n);
    return secpe_linear_create_coeffs(ctx, Wm.data(), mask.data(), pad.data(), K, C, d, out);
}

extern "C" void secpe_linear_destroy(secpe_linear *lin) {
    if (!lin) return;
    cudaDeviceSynchronize();
    if (lin->W) cudaFree(lin->W);
    if (lin->mask) cudaFree(lin->mask);
    if (lin->pad) cudaFree(lin->pad);
    delete lin;
}

extern "C" int secpe_linear_apply(secpe_ctx *ctx, const secpe_keys *keys, const secpe_linear *lin,
                                  const secpe_ct *x, secpe_ct *outs, void *stream) {
    if (!ctx || !keys || !lin || lin->ctx != ctx || !outs || !ct_ok(ctx, x)) return SECPE_EINVAL;
    const int K = lin->K, L = lin->level, n = ctx->n;
    if (x->level != L) return SECPE_ELEVEL;
    if (std::fabs(x->scale - ctx->scale) > ctx->scale * std::ldexp(1.0, -40)) return SECPE_ESCALE;
    for (int i = 0; i < K; i++)
        if (!outs[i].data || !aligned16(outs[i].data) || outs[i].cap < L - 1) return SECPE_EINVAL;
    ctx->stream = (cudaStream_t)stream;
    Eval E{ctx, keys, {}, 0};
    // W_i (.) x for every prompt, rescaled: level L - 1, x's scale
    Ct T, P;
    SECPE_CHECK(ct_alloc(ctx, K, L, x->scale * (double)ctx->primes[L], T));
    SECPE_CHECK(launch_mul_plain(ctx, view_ct(ctx, x), 0, lin->W, (long long)(L + 1) * n, T.v, L + 1));
    SECPE_CHECK(E.rescale(T, P));
    T = Ct();
    // sum over j: log2(d) rotations by C' 2^t
    for (int s = lin->cp; s < lin->cp * lin->d; s <<= 1) {
        Ct R, S;
        SECPE_CHECK(E.rotate(P, s, R));
        SECPE_CHECK(E.add(P, R, S));
        P = S;
    }
    // mask to the C logit slots, rescaled: level L - 2
    Ct T2, M;
    SECPE_CHECK(ct_alloc(ctx, K, L - 1, P.scale() * (double)ctx->primes[L - 1], T2));
    SECPE_CHECK(launch_mul_plain(ctx, P.v, P.v.stride, lin->mask, 0, T2.v, L));
    P = Ct();
    SECPE_CHECK(E.rescale(T2, M));
    T2 = Ct();
    // d_min in the padding slots [C, C')
    for (int i = 0; i < K; i++) {
        CtB o = view_ct(ctx, &outs[i]);
        SECPE_CHECK(launch_add_plain(ctx, ct_slice(M, i, i + 1).v, lin->pad, o, L - 1));
        outs[i].level = L - 2;
        outs[i].scale = M.scale();
    }
    return cudaGetLastError() == cudaSuccess ? SECPE_OK : SECPE_ECUDA;
}

extern "C" int secpe_encrypt_replicated(secpe_ctx *ctx, const secpe_keys *keys, const double *x, int d, int C,
                                        uint64_t seed, secpe_ct *out, void *stream) {
    if (!ctx || !x || C < 1 || !is_pow2(d) || C > ctx->n / 2) return SECPE_EINVAL;
    const int cp = pow2_ceil(C), n = ctx->n;
    if ((long long)d * cp > n / 2) return SECPE_EINVAL;
    std::vector<double> v((size_t)d * cp);
    for (int j = 0; j < d; j++)
        for (int c = 0; c < cp; c++) v[(size_t)j * cp + c] = x[j];
    std::vector<long long> m;
    if (!enc::encode_real_fft(n, v.data(), d * cp, ctx->scale, m)) return SECPE_EINVAL;
    return secpe_encrypt_coeffs(ctx, keys, (const int64_t *)m.data(), ctx->L, ctx->scale, seed, out, stream);
}
