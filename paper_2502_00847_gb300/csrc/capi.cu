// extern "C" entry points declared in include/secpe.h.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <map>
#include <string>

#include "eval.h"

namespace enc {
bool encode_real(int n, const double *v, int nv, double scale, std::vector<long long> &m);
void decode_real(int n, const double *coeffs, double scale, int nslots, double *out);
bool encode_real_fft(int n, const double *v, int nv, double scale, std::vector<long long> &m);
void decode_real_fft(int n, const double *coeffs, double scale, int nslots, double *out);
}  // namespace enc

int argmax_batch_impl(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q, int nq_);
int phoenix_batch_impl(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q, int nq_);

namespace {

// Per-call guard: sets the stream, and turns a sticky CUDA error into ECUDA.
struct CallScope {
    secpe_ctx *ctx;
    CallScope(secpe_ctx *c, void *stream) : ctx(c) { c->stream = (cudaStream_t)stream; }
};

Ct view(secpe_ctx *ctx, const secpe_ct *c) {
    Ct r;
    r.v.data = (u64 *)c->data;
    r.v.B = 1;
    r.v.cap = c->cap;
    r.v.stride = 2ll * c->cap * ctx->n;
    r.v.level = c->level;
    r.v.scale = c->scale;
    r.v.n = ctx->n;
    return r;
}

int check_ct(const secpe_ctx *ctx, const secpe_ct *c) {
    if (!c || !c->data || !aligned16(c->data) || c->level < 0 || c->level > ctx->L || c->cap < c->level + 1)
        return SECPE_EINVAL;
    if (!(c->scale > 0.0)) return SECPE_EINVAL;
    return SECPE_OK;
}

int copy_out(secpe_ctx *ctx, const Ct &src, secpe_ct *dst) {
    if (!dst || !dst->data || !aligned16(dst->data) || dst->cap < src.level() + 1) return SECPE_EINVAL;
    const size_t n = ctx->n;
    if ((u64 *)dst->data != src.v.data)
        SECPE_CUDA(cudaMemcpy2DAsync(dst->data, sizeof(u64) * dst->cap * n, src.v.data, sizeof(u64) * src.v.cap * n,
                                     sizeof(u64) * (src.level() + 1) * n, 2, cudaMemcpyDeviceToDevice, ctx->stream));
    dst->level = src.level();
    dst->scale = src.scale();
    return SECPE_OK;
}

int finish(secpe_ctx *ctx, int st) {
    if (st != SECPE_OK) return st;
    return cudaGetLastError() == cudaSuccess ? SECPE_OK : SECPE_ECUDA;
}

int make_ksk(secpe_ctx *ctx, secpe_keys *keys, const u64 *s_new, uint64_t kid, u64 **out) {
    const int n = ctx->n, np = ctx->nprimes, L = ctx->L, alpha = ctx->alpha;
    const int ndig = (L + 1 + alpha - 1) / alpha;
    u64 *key = nullptr;
    SECPE_CUDA(cudaMalloc(&key, sizeof(u64) * (size_t)ndig * 2 * np * n));
    *out = key;
    DevBuf a, e, en, pm;
    SECPE_CHECK(a.alloc(ctx, sizeof(u64) * (size_t)np * n));
    SECPE_CHECK(e.alloc(ctx, sizeof(long long) * (size_t)n));
    SECPE_CHECK(en.alloc(ctx, sizeof(u64) * (size_t)np * n));
    // [P]_{q_t}
    std::vector<u64> pmod(np);
    for (int t = 0; t < np; t++) {
        u64 x = 1;
        for (int j = 0; j < ctx->npsp; j++) x = hm::mulmod(x, ctx->primes[ctx->nq + j] % ctx->primes[t], ctx->primes[t]);
        pmod[t] = x;
    }
    SECPE_CHECK(pm.alloc(ctx, sizeof(u64) * np));
    SECPE_CUDA(cudaMemcpyAsync(pm.p, pmod.data(), sizeof(u64) * np, cudaMemcpyHostToDevice, ctx->stream));
    PrimeList pl;
    pl.n = np;
    for (int t = 0; t < np; t++) pl.p[t] = t;
    LimbSet ls = make_limbset(en.u(), 1, 0, 1, 0, np, 0);
    for (int j = 0; j < ndig; j++) {
        const int lo = j * alpha, hi = std::min((j + 1) * alpha, L + 1);
        std::vector<u64> ka(1, hm::sm_stream(keys->seed, DOM_KSK_A, kid * 64 + j));
        std::vector<u64> ke(1, hm::sm_stream(keys->seed, DOM_KSK_E, kid * 64 + j));
        SECPE_CHECK(launch_sample_uniform(ctx, ka, a.u(), 0, pl));
        SECPE_CHECK(launch_sample_small(ctx, ke, (long long *)e.p, 1));
        SECPE_CHECK(launch_signed_to_limbs(ctx, (const long long *)e.p, nullptr, en.u(), 0, 1, pl));
        SECPE_CHECK(ntt_limbset(ctx, ls, false));
        SECPE_CHECK(launch_ksk_gen(ctx, a.u(), en.u(), keys->s_ntt, s_new, pm.u(),
                                   key + (size_t)j * 2 * np * n, lo, hi));
    }
    return SECPE_OK;
}

}  // namespace

extern "C" const char *secpe_strerror(int code) {
    switch (code) {
        case SECPE_OK: return "ok";
        case SECPE_EINVAL: return "invalid argument";
        case SECPE_ENOMEM: return "device allocation failed";
        case SECPE_ELEVEL: return "not enough levels";
        case SECPE_ESCALE: return "scale mismatch";
        case SECPE_EKEY: return "missing key";
        case SECPE_ECUDA: return "CUDA error";
        case SECPE_ETIMEOUT: return "device wait timed out";
        case SECPE_EADMIT: return "admission budget exceeded";
        default: return "unknown error";
    }
}

extern "C" int secpe_device_wait_selftest(secpe_ctx *ctx, int arrive, int64_t polls, void *stream) {
    if (!ctx || polls < 1 || polls > (1 << 22)) return SECPE_EINVAL;
    CallScope cs(ctx, stream);
    return finish(ctx, wait_selftest(ctx, arrive, (long)polls));
}

extern "C" int secpe_stream_status(secpe_ctx *ctx, void *stream, int *device_status) {
    if (!ctx || !device_status) return SECPE_EINVAL;
    SECPE_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int v = 0;
    SECPE_CUDA(cudaMemcpy(&v, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    int z = 0;
    SECPE_CUDA(cudaMemcpy(ctx->d_status, &z, sizeof(int), cudaMemcpyHostToDevice));
    *device_status = v;
    return SECPE_OK;
}

extern "C" int secpe_get_counters(const secpe_ctx *ctx, secpe_counters *out) {
    if (!ctx || !out) return SECPE_EINVAL;
    *out = ctx->counters;
    return SECPE_OK;
}

extern "C" int secpe_reset_counters(secpe_ctx *ctx) {
    if (!ctx) return SECPE_EINVAL;
    std::memset(&ctx->counters, 0, sizeof(ctx->counters));
    return SECPE_OK;
}

// ---------------------------------------------------------------- keys
extern "C" int secpe_keygen(secpe_ctx *ctx, uint64_t seed, const int32_t *rot_steps, int n_rot,
                            secpe_keys **out) {
    if (!ctx || !out || n_rot < 0 || (n_rot > 0 && !rot_steps)) return SECPE_EINVAL;
    *out = nullptr;
    CallScope cs(ctx, nullptr);
    const int n = ctx->n, np = ctx->nprimes;
    secpe_keys *k = new secpe_keys();
    k->seed = seed;
    k->seed_set = 1;
    k->s_ntt = nullptr;
    k->rlk = nullptr;
    int st = SECPE_OK;
    do {
        if (cudaMalloc(&k->s_ntt, sizeof(u64) * (size_t)np * n) != cudaSuccess) {
            st = SECPE_ENOMEM;
            break;
        }
        DevBuf s, s2;
        if ((st = s.alloc(ctx, sizeof(long long) * n)) != SECPE_OK) break;
        std::vector<u64> ks(1, hm::sm_stream(seed, DOM_SECRET, 0));
        if (ctx->p.secret_hw > 0) {
            std::vector<long long> sh;
            hm::sample_sparse_secret(ks[0], n, ctx->p.secret_hw, sh);
            if (cudaMemcpy(s.p, sh.data(), sizeof(long long) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
                st = SECPE_ECUDA;
                break;
            }
        } else if ((st = launch_sample_small(ctx, ks, (long long *)s.p, 0)) != SECPE_OK) {
            break;
        }
        PrimeList pl;
        pl.n = np;
        for (int t = 0; t < np; t++) pl.p[t] = t;
        if ((st = launch_signed_to_limbs(ctx, (const long long *)s.p, nullptr, k->s_ntt, 0, 1, pl)) != SECPE_OK) break;
        LimbSet ls = make_limbset(k->s_ntt, 1, 0, 1, 0, np, 0);
        if ((st = ntt_limbset(ctx, ls, false)) != SECPE_OK) break;
        if ((st = s2.alloc(ctx, sizeof(u64) * (size_t)np * n)) != SECPE_OK) break;
        if ((st = launch_limb_mul(ctx, k->s_ntt, k->s_ntt, s2.u())) != SECPE_OK) break;
        if ((st = make_ksk(ctx, k, s2.u(), 0, &k->rlk)) != SECPE_OK) break;
        for (int r = 0; r < n_rot && st == SECPE_OK; r++) {
            const unsigned g = galois_elt(ctx, rot_steps[r]);
            if (k->gks.count(g)) continue;
            DevBuf sg;
            if ((st = sg.alloc(ctx, sizeof(u64) * (size_t)np * n)) != SECPE_OK) break;
            if ((st = launch_limb_automorph(ctx, k->s_ntt, sg.u(), g)) != SECPE_OK) break;
            u64 *key = nullptr;
            st = make_ksk(ctx, k, sg.u(), g, &key);
            if (key) k->gks[g] = key;
        }
    } while (0);
    if (st == SECPE_OK && cudaStreamSynchronize(0) != cudaSuccess) st = SECPE_ECUDA;
    if (st != SECPE_OK) {
        secpe_keys_destroy(k);
        return st;
    }
    *out = k;
    return SECPE_OK;
}

extern "C" void secpe_keys_destroy(secpe_keys *keys) {
    if (!keys) return;
    cudaDeviceSynchronize();
    if (keys->s_ntt) cudaFree(keys->s_ntt);
    if (keys->rlk) cudaFree(keys->rlk);
    for (auto &kv : keys->gks) cudaFree(kv.second);
    delete keys;
}

extern "C" int secpe_keys_export(const secpe_ctx *cctx, const secpe_keys *keys, int which, int32_t step,
                                 uint64_t *host_out, size_t words) {
    secpe_ctx *ctx = const_cast<secpe_ctx *>(cctx);
    if (!ctx || !keys || !host_out) return SECPE_EINVAL;
    CallScope cs(ctx, nullptr);
    const size_t n = ctx->n, np = ctx->nprimes;
    const int ndig = (ctx->L + 1 + ctx->alpha - 1) / ctx->alpha;
    if (which == 0) {
        if (words < np * n) return SECPE_EINVAL;
        SECPE_CUDA(cudaMemcpy(host_out, keys->s_ntt, sizeof(u64) * np * n, cudaMemcpyDeviceToHost));
        return SECPE_OK;
    }
    const u64 *src = nullptr;
    if (which == 1) src = keys->rlk;
    else if (which == 2) src = galois_key(keys, galois_elt(ctx, step));
    if (!src) return SECPE_EKEY;
    const size_t total = (size_t)ndig * 2 * np * n;
    if (words < total) return SECPE_EINVAL;
    DevBuf tmp;
    SECPE_CHECK(tmp.alloc(ctx, sizeof(u64) * total));
    SECPE_CHECK(launch_from_mont(ctx, src, tmp.u(), ndig * 2 * (int)np));
    SECPE_CUDA(cudaMemcpyAsync(host_out, tmp.p, sizeof(u64) * total, cudaMemcpyDeviceToHost, ctx->stream));
    SECPE_CUDA(cudaStreamSynchronize(ctx->stream));
    return SECPE_OK;
}

// ---------------------------------------------------------------- client
extern "C" int secpe_encrypt_coeffs(secpe_ctx *ctx, const secpe_keys *keys, const int64_t *m, int level,
                                    double scale, uint64_t seed, secpe_ct *out, void *stream) {
    if (!ctx || !keys || !m || !out || !out->data || !aligned16(out->data) || level < 0 || level > ctx->L || out->cap < level + 1 ||
        !(scale > 0))
        return SECPE_EINVAL;
    CallScope cs(ctx, stream);
    const int n = ctx->n;
    DevBuf dm, e, M, a;
    SECPE_CHECK(dm.alloc(ctx, sizeof(long long) * n));
    SECPE_CUDA(cudaMemcpyAsync(dm.p, m, sizeof(long long) * n, cudaMemcpyHostToDevice, ctx->stream));
    SECPE_CHECK(e.alloc(ctx, sizeof(long long) * n));
    std::vector<u64> ke(1, hm::sm_stream(seed, DOM_ENC_E, 0)), ka(1, hm::sm_stream(seed, DOM_ENC_A, 0));
    SECPE_CHECK(launch_sample_small(ctx, ke, (long long *)e.p, 1));
    PrimeList pl;
    pl.n = level + 1;
    for (int i = 0; i <= level; i++) pl.p[i] = i;
    SECPE_CHECK(M.alloc(ctx, sizeof(u64) * (size_t)(level + 1) * n));
    SECPE_CHECK(launch_signed_to_limbs(ctx, (const long long *)dm.p, (const long long *)e.p, M.u(), 0, 1, pl));
    LimbSet ls = make_limbset(M.u(), 1, 0, 1, 0, level + 1, 0);
    SECPE_CHECK(ntt_limbset(ctx, ls, false));
    SECPE_CHECK(a.alloc(ctx, sizeof(u64) * (size_t)(level + 1) * n));
    SECPE_CHECK(launch_sample_uniform(ctx, ka, a.u(), 0, pl));
    Ct o = view(ctx, out);
    o.v.level = level;
    SECPE_CHECK(launch_enc_finish(ctx, M.u(), 0, a.u(), 0, keys->s_ntt, o.v, level + 1));
    out->level = level;
    out->scale = scale;
    return finish(ctx, SECPE_OK);
}

extern "C" int secpe_encrypt(secpe_ctx *ctx, const secpe_keys *keys, const double *v, int n, uint64_t seed,
                             secpe_ct *out, void *stream) {
    if (!ctx || (!v && n > 0) || n < 0 || n > ctx->n / 2) return SECPE_EINVAL;
    std::vector<long long> m;
    if (!enc::encode_real(ctx->n, v, n, ctx->scale, m)) return SECPE_EINVAL;
    return secpe_encrypt_coeffs(ctx, keys, (const int64_t *)m.data(), ctx->L, ctx->scale, seed, out, stream);
}

extern "C" int secpe_encrypt_logits(secpe_ctx *ctx, const secpe_keys *keys, const double *v, int C, double d_min,
                                    uint64_t seed, secpe_ct *out, void *stream) {
    if (!ctx || !v || C < 1 || C > ctx->n / 2) return SECPE_EINVAL;
    int cp = 1;
    while (cp < C) cp <<= 1;
    if (cp > ctx->n / 2) return SECPE_EINVAL;
    std::vector<double> full(cp, d_min);
    for (int i = 0; i < C; i++) full[i] = v[i];
    return secpe_encrypt(ctx, keys, full.data(), cp, seed, out, stream);
}

// ---- slot packing: P inputs of C classes per ciphertext, block b at slots
// [2 C' b, 2 C' (b + 1)): v_b in the first C slots, d_min up to C', zeros in
// the upper half (room for Alg. 1's duplication within the block).
static int pow2_at_least(int C) {
    int cp = 1;
    while (cp < C) cp <<= 1;
    return cp;
}

extern "C" int secpe_packed_capacity(int log_n, int C) {
    if (log_n < 4 || log_n > 17 || C < 1) return SECPE_EINVAL;
    const long long slots = 1ll << (log_n - 1);
    if (C > slots / 2) return 0;  // 2 C' > slots; also keeps C' far from int overflow
    const long long cp = pow2_at_least(C);
    return 2 * cp > slots ? 0 : (int)(slots / (2 * cp));
}

extern "C" int secpe_encode_packed(int log_n, double scale, const double *v, int P, int C, double d_min,
                                   int64_t *m_out) {
    const int cap = secpe_packed_capacity(log_n, C);
    if (cap < 0 || !v || !m_out || P < 1 || P > cap || !(scale > 0.0)) return SECPE_EINVAL;
    const int n = 1 << log_n, cp = pow2_at_least(C);
    std::vector<double> slots((size_t)P * 2 * cp, 0.0);
    for (int b = 0; b < P; b++)
        for (int j = 0; j < cp; j++) slots[(size_t)b * 2 * cp + j] = j < C ? v[(size_t)b * C + j] : d_min;
    std::vector<long long> m;
    if (!enc::encode_real_fft(n, slots.data(), (int)slots.size(), scale, m)) return SECPE_EINVAL;
    std::memcpy(m_out, m.data(), sizeof(int64_t) * n);
    return SECPE_OK;
}

extern "C" int secpe_decode_packed(int log_n, double scale, const double *coeffs, int P, int C, double *out) {
    const int cap = secpe_packed_capacity(log_n, C);
    if (cap < 0 || !coeffs || !out || P < 1 || P > cap || !(scale > 0.0)) return SECPE_EINVAL;
    const int n = 1 << log_n, cp = pow2_at_least(C);
    std::vector<double> slots((size_t)P * 2 * cp);
    enc::decode_real_fft(n, coeffs, scale, (int)slots.size(), slots.data());
    for (int b = 0; b < P; b++)
        for (int j = 0; j < C; j++) out[(size_t)b * C + j] = slots[(size_t)b * 2 * cp + j];
    return SECPE_OK;
}

extern "C" int secpe_encrypt_logits_packed(secpe_ctx *ctx, const secpe_keys *keys, const double *v, int P, int C,
                                           double d_min, uint64_t seed, secpe_ct *out, void *stream) {
    if (!ctx) return SECPE_EINVAL;
    std::vector<int64_t> m(ctx->n);
    SECPE_CHECK(secpe_encode_packed(ctx->log_n, ctx->scale, v, P, C, d_min, m.data()));
    return secpe_encrypt_coeffs(ctx, keys, m.data(), ctx->L, ctx->scale, seed, out, stream);
}

static int decrypt_to_host_coeffs(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ct *ct,
                                  std::vector<double> &coeffs) {
    const int n = ctx->n, lv = ct->level;
    DevBuf m, dbl;
    SECPE_CHECK(m.alloc(ctx, sizeof(u64) * (size_t)(lv + 1) * n));
    Ct x = view(ctx, ct);
    SECPE_CHECK(launch_dec_dot(ctx, x.v, keys->s_ntt, m.u(), lv + 1));
    LimbSet ls = make_limbset(m.u(), 1, 0, 1, 0, lv + 1, 0);
    SECPE_CHECK(ntt_limbset(ctx, ls, true));
    SECPE_CHECK(dbl.alloc(ctx, sizeof(double) * n));
    SECPE_CHECK(launch_crt_double(ctx, m.u(), lv, (double *)dbl.p));
    coeffs.resize(n);
    SECPE_CUDA(cudaMemcpyAsync(coeffs.data(), dbl.p, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    SECPE_CUDA(cudaStreamSynchronize(ctx->stream));
    return SECPE_OK;
}

extern "C" int secpe_decrypt_coeffs(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ct *ct,
                                    double *coeffs_out, void *stream) {
    if (!ctx || !keys || !coeffs_out) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, ct));
    CallScope cs(ctx, stream);
    std::vector<double> c;
    SECPE_CHECK(decrypt_to_host_coeffs(ctx, keys, ct, c));
    std::memcpy(coeffs_out, c.data(), sizeof(double) * ctx->n);
    return SECPE_OK;
}

extern "C" int secpe_decrypt_packed(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ct *ct, int P, int C,
                                    double *out, void *stream) {
    if (!ctx || !keys || !out) return SECPE_EINVAL;
    const int cap = secpe_packed_capacity(ctx->log_n, C);
    if (cap < 0 || P < 1 || P > cap) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, ct));
    CallScope cs(ctx, stream);
    std::vector<double> c;
    SECPE_CHECK(decrypt_to_host_coeffs(ctx, keys, ct, c));
    return secpe_decode_packed(ctx->log_n, ct->scale, c.data(), P, C, out);
}

extern "C" int secpe_decrypt(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ct *ct, double *v_out, int n,
                             void *stream) {
    if (!ctx || !keys || !v_out || n < 0 || n > ctx->n / 2) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, ct));
    CallScope cs(ctx, stream);
    std::vector<double> c;
    SECPE_CHECK(decrypt_to_host_coeffs(ctx, keys, ct, c));
    enc::decode_real(ctx->n, c.data(), ct->scale, n, v_out);
    return SECPE_OK;
}

// ---------------------------------------------------------------- primitives
extern "C" int secpe_ntt(secpe_ctx *ctx, uint64_t *limbs, const int32_t *prime_idx, int count, int inverse,
                         void *stream) {
    if (!ctx || !limbs || !aligned16(limbs) || !prime_idx || count < 0) return SECPE_EINVAL;
    CallScope cs(ctx, stream);
    for (int s = 0; s < count; s += SECPE_MAX_LIMBSET) {
        const int c = std::min(SECPE_MAX_LIMBSET, count - s);
        LimbSet ls = make_limbset((u64 *)limbs + (size_t)s * ctx->n, 1, 0, 1, 0, c, 0);
        for (int j = 0; j < c; j++) {
            if (prime_idx[s + j] < 0 || prime_idx[s + j] >= ctx->nprimes) return SECPE_EINVAL;
            ls.prime_of[j] = (int8_t)prime_idx[s + j];
        }
        SECPE_CHECK(ntt_limbset(ctx, ls, inverse != 0));
    }
    return finish(ctx, SECPE_OK);
}

extern "C" int secpe_ntt_cts(secpe_ctx *ctx, uint64_t *base, int batch, size_t ct_stride, int cap, int level,
                             int inverse, void *stream) {
    if (!ctx || !base || !aligned16(base) || (ct_stride & 1) || batch < 0 || level < 0 || level >= cap ||
        level > ctx->L || ct_stride < 2ull * cap * ctx->n)
        return SECPE_EINVAL;
    CallScope cs(ctx, stream);
    LimbSet ls = make_limbset((u64 *)base, batch, (long long)ct_stride, 2, (long long)cap * ctx->n, level + 1, 0);
    return finish(ctx, ntt_limbset(ctx, ls, inverse != 0));
}

#define EVAL_PROLOGUE(ctx, stream) \
    CallScope cs(ctx, stream);     \
    Eval E{ctx, keys_, {}, 0};

extern "C" int secpe_add(secpe_ctx *ctx, const secpe_ct *a, const secpe_ct *b, secpe_ct *out, void *stream) {
    if (!ctx) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, a));
    SECPE_CHECK(check_ct(ctx, b));
    const secpe_keys *keys_ = nullptr;
    EVAL_PROLOGUE(ctx, stream);
    Ct r;
    SECPE_CHECK(E.add(view(ctx, a), view(ctx, b), r));
    return finish(ctx, copy_out(ctx, r, out));
}

extern "C" int secpe_sub(secpe_ctx *ctx, const secpe_ct *a, const secpe_ct *b, secpe_ct *out, void *stream) {
    if (!ctx) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, a));
    SECPE_CHECK(check_ct(ctx, b));
    const secpe_keys *keys_ = nullptr;
    EVAL_PROLOGUE(ctx, stream);
    Ct r;
    SECPE_CHECK(E.sub(view(ctx, a), view(ctx, b), r));
    return finish(ctx, copy_out(ctx, r, out));
}

extern "C" int secpe_mul_const(secpe_ctx *ctx, const secpe_ct *a, double c, double target_scale, int out_level,
                               secpe_ct *out, void *stream) {
    if (!ctx || !(target_scale > 0)) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, a));
    const secpe_keys *keys_ = nullptr;
    EVAL_PROLOGUE(ctx, stream);
    Ct r;
    SECPE_CHECK(E.mul_const(view(ctx, a), {c}, target_scale, out_level, r));
    return finish(ctx, copy_out(ctx, r, out));
}

extern "C" int secpe_add_const(secpe_ctx *ctx, const secpe_ct *a, double c, secpe_ct *out, void *stream) {
    if (!ctx) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, a));
    const secpe_keys *keys_ = nullptr;
    EVAL_PROLOGUE(ctx, stream);
    Ct r;
    SECPE_CHECK(E.add_const(view(ctx, a), c, r));
    return finish(ctx, copy_out(ctx, r, out));
}

extern "C" int secpe_mul_relin(secpe_ctx *ctx, const secpe_keys *keys_, const secpe_ct *a, const secpe_ct *b,
                               secpe_ct *out, void *stream) {
    if (!ctx || !keys_) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, a));
    SECPE_CHECK(check_ct(ctx, b));
    EVAL_PROLOGUE(ctx, stream);
    Ct r;
    SECPE_CHECK(E.mul(view(ctx, a), view(ctx, b), r));
    return finish(ctx, copy_out(ctx, r, out));
}

extern "C" int secpe_rescale(secpe_ctx *ctx, const secpe_ct *in, secpe_ct *out, void *stream) {
    if (!ctx) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, in));
    const secpe_keys *keys_ = nullptr;
    EVAL_PROLOGUE(ctx, stream);
    Ct r;
    SECPE_CHECK(E.rescale(view(ctx, in), r));
    return finish(ctx, copy_out(ctx, r, out));
}

extern "C" int secpe_rotate(secpe_ctx *ctx, const secpe_keys *keys_, const secpe_ct *in, int steps, secpe_ct *out,
                            void *stream) {
    if (!ctx || !keys_) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, in));
    EVAL_PROLOGUE(ctx, stream);
    Ct r;
    SECPE_CHECK(E.rotate(view(ctx, in), steps, r));
    return finish(ctx, copy_out(ctx, r, out));
}

extern "C" int secpe_rotate_hoisted(secpe_ctx *ctx, const secpe_keys *keys_, const secpe_ct *in, const int32_t *steps,
                                    int count, secpe_ct *outs, void *stream) {
    if (!ctx || !keys_ || !steps || !outs || count < 1 || count > 64) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, in));
    for (int i = 0; i < count; i++) {
        if (!outs[i].data || !aligned16(outs[i].data) || outs[i].cap < in->level + 1) return SECPE_EINVAL;
        if (outs[i].data == in->data) return SECPE_EINVAL;
    }
    EVAL_PROLOGUE(ctx, stream);
    std::vector<Ct> r;
    SECPE_CHECK(E.rotate_hoisted(view(ctx, in), std::vector<int>(steps, steps + count), r));
    for (int i = 0; i < count; i++) SECPE_CHECK(copy_out(ctx, r[i], &outs[i]));
    return finish(ctx, SECPE_OK);
}

extern "C" int secpe_keyswitch(secpe_ctx *ctx, const secpe_keys *keys, int galois_step, const uint64_t *d,
                               int level, int cap, uint64_t *ks0, uint64_t *ks1, void *stream) {
    if (!ctx || !keys || !d || !ks0 || !ks1 || !aligned16(d) || !aligned16(ks0) || !aligned16(ks1) || level < 0 ||
        level > ctx->L || cap < level + 1)
        return SECPE_EINVAL;
    CallScope cs(ctx, stream);
    const u64 *key = galois_step == 0 ? keys->rlk : galois_key(keys, galois_elt(ctx, galois_step));
    if (!key) return SECPE_EKEY;
    const int n = ctx->n;
    // result polys are written into a temporary [2][level+1][N] and copied
    Ct o;
    SECPE_CHECK(ct_alloc(ctx, 1, level, 1.0, o));
    SECPE_CHECK(keyswitch(ctx, (const u64 *)d, 0, 1, level, key, o.v, false, false));
    SECPE_CUDA(cudaMemcpyAsync(ks0, o.v.data, sizeof(u64) * (level + 1) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    SECPE_CUDA(cudaMemcpyAsync(ks1, o.v.data + o.v.pstride(), sizeof(u64) * (level + 1) * n,
                               cudaMemcpyDeviceToDevice, ctx->stream));
    return finish(ctx, SECPE_OK);
}

extern "C" int secpe_refresh_testonly(secpe_ctx *ctx, const secpe_keys *keys_, const secpe_ct *in, uint64_t qseed,
                                      uint64_t refresh_index, secpe_ct *out, void *stream) {
    if (!ctx || !keys_) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, in));
    EVAL_PROLOGUE(ctx, stream);
    E.qseeds.assign(1, qseed);
    E.ridx = refresh_index;
    Ct r;
    SECPE_CHECK(E.refresh(view(ctx, in), r));
    return finish(ctx, copy_out(ctx, r, out));
}

extern "C" int secpe_sign(secpe_ctx *ctx, const secpe_keys *keys_, const secpe_ct *x, int out_levels, uint64_t qseed,
                          uint64_t *refresh_index, secpe_ct *out, void *stream) {
    if (!ctx || !keys_ || !refresh_index || out_levels < 0) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, x));
    EVAL_PROLOGUE(ctx, stream);
    E.qseeds.assign(1, qseed);
    E.ridx = *refresh_index;
    Ct r;
    SECPE_CHECK(E.sign(view(ctx, x), out_levels, r));
    *refresh_index = E.ridx;
    return finish(ctx, copy_out(ctx, r, out));
}

extern "C" int secpe_max(secpe_ctx *ctx, const secpe_keys *keys_, const secpe_ct *a, const secpe_ct *y,
                         uint64_t qseed, uint64_t *refresh_index, secpe_ct *out, void *stream) {
    if (!ctx || !keys_ || !refresh_index) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, a));
    SECPE_CHECK(check_ct(ctx, y));
    EVAL_PROLOGUE(ctx, stream);
    E.qseeds.assign(1, qseed);
    E.ridx = *refresh_index;
    Ct r;
    SECPE_CHECK(E.max(view(ctx, a), view(ctx, y), r));
    *refresh_index = E.ridx;
    return finish(ctx, copy_out(ctx, r, out));
}

extern "C" int secpe_ensemble_aggregate(secpe_ctx *ctx, const secpe_ct *cts, int K, double d_min, double d_max,
                                        secpe_ct *out, void *stream) {
    if (!ctx || !cts || K < 1 || !(d_max > d_min)) return SECPE_EINVAL;
    for (int i = 0; i < K; i++) SECPE_CHECK(check_ct(ctx, &cts[i]));
    const secpe_keys *keys_ = nullptr;
    EVAL_PROLOGUE(ctx, stream);
    Ct y = view(ctx, &cts[0]);
    for (int i = 1; i < K; i++) {
        Ct t;
        SECPE_CHECK(E.add(y, view(ctx, &cts[i]), t));
        y = t;
    }
    const double w = 1.0 / (K * (d_max - d_min));
    Ct r;
    SECPE_CHECK(E.mul_const(y, {w}, ctx->scale, y.level() - 1, r));
    return finish(ctx, copy_out(ctx, r, out));
}

extern "C" int secpe_encrypted_argmax(secpe_ctx *ctx, const secpe_keys *keys_, const secpe_ct *y, int C,
                                      uint64_t qseed, secpe_ct *z_out, void *stream) {
    if (!ctx || !keys_) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, y));
    EVAL_PROLOGUE(ctx, stream);
    E.qseeds.assign(1, qseed);
    Ct r;
    SECPE_CHECK(E.argmax(view(ctx, y), C, r));
    return finish(ctx, copy_out(ctx, r, z_out));
}

extern "C" int secpe_level_plan(const secpe_params *p, int C, int entry_level, int refresh_level, int32_t *targets,
                                int capacity, int *count) {
    if (!p || !count || C < 2 || p->reserve < 1 || p->sign_dg < 0 || p->sign_df < 0 || p->sign_dg + p->sign_df < 1 ||
        entry_level < 0 || entry_level >= p->n_q || refresh_level < 1 || refresh_level >= p->n_q)
        return SECPE_EINVAL;
    // 2 C' slots must fit in the N/2 of the ring: C <= N/4 (N <= 2^17)
    if (p->log_n < 4 || p->log_n > 17 || C > (1 << (p->log_n - 2))) return SECPE_EINVAL;
    int r = 0;
    while ((1 << r) < C) r++;
    LevelPlan lp;
    SECPE_CHECK(make_level_plan(p->reserve, p->sign_dg + p->sign_df, refresh_level, r, entry_level, lp));
    *count = (int)lp.target.size();
    if (!targets) return SECPE_OK;
    if (capacity < *count) return SECPE_EINVAL;
    for (int j = 0; j < *count; j++) targets[j] = lp.target[j];
    return SECPE_OK;
}

extern "C" int secpe_argmax_batch(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q, int n_queries,
                                  void *stream) {
    if (!ctx || !q || n_queries < 0) return SECPE_EINVAL;
    if (n_queries == 0) return SECPE_OK;
    CallScope cs(ctx, stream);
    return finish(ctx, argmax_batch_impl(ctx, keys, q, n_queries));
}

extern "C" int secpe_phoenix_argmax(secpe_ctx *ctx, const secpe_keys *keys_, const secpe_ct *y, int C,
                                    uint64_t qseed, secpe_ct *z_out, void *stream) {
    if (!ctx || !keys_) return SECPE_EINVAL;
    SECPE_CHECK(check_ct(ctx, y));
    EVAL_PROLOGUE(ctx, stream);
    E.qseeds.assign(1, qseed);
    Ct r;
    SECPE_CHECK(E.phoenix(view(ctx, y), C, r));
    return finish(ctx, copy_out(ctx, r, z_out));
}

extern "C" int secpe_phoenix_argmax_batch(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q,
                                          int n_queries, void *stream) {
    if (!ctx || !q || n_queries < 0) return SECPE_EINVAL;
    if (n_queries == 0) return SECPE_OK;
    CallScope cs(ctx, stream);
    return finish(ctx, phoenix_batch_impl(ctx, keys, q, n_queries));
}

extern "C" int secpe_argmax_batch_boot(secpe_ctx *ctx, const secpe_keys *keys, const secpe_boot *bt,
                                       const secpe_query *q, int n_queries, void *stream) {
    if (!ctx || !bt || !q || n_queries < 0) return SECPE_EINVAL;
    for (int i = 0; i < n_queries; i++) {
        if (q[i].C > boot_block(bt)) return SECPE_EINVAL;
        int cp = 1;
        while (cp < q[i].C) cp <<= 1;
        if (2 * cp > boot_block(bt)) return SECPE_EINVAL;
    }
    if (n_queries == 0) return SECPE_OK;
    CallScope cs(ctx, stream);
    ctx->boot = bt;
    const int st = argmax_batch_impl(ctx, keys, q, n_queries);
    ctx->boot = nullptr;
    return finish(ctx, st);
}

// ---------------------------------------------------------------- autotuning
static const char *const kTuneNames[TUNE_NSLOTS] = {"ntt16_colpass", "ntt16_rowpass", "intt16_colpass",
                                                     "intt16_rowpass", "colpass_bconv"};

extern "C" int secpe_tuning_set(secpe_ctx *ctx, int kernel, int ctas_per_sm) {
    if (!ctx || kernel < 0 || kernel >= TUNE_NSLOTS || (ctas_per_sm != 3 && ctas_per_sm != 4)) return SECPE_EINVAL;
    ctx->tune.ctas[kernel] = ctas_per_sm;
    return SECPE_OK;
}

extern "C" int secpe_autotune(secpe_ctx *ctx, secpe_tuning *out, void *stream) {
    if (!ctx) return SECPE_EINVAL;
    if (out) std::memset(out, 0, sizeof(*out));
    if (ctx->log_n != 16) return SECPE_OK;
    CallScope cs(ctx, stream);
    // 64 items of 32 limbs (1 GiB): larger than L2, like the batched workload
    const int n = ctx->n, nitem = 64, nlimb = 32, reps = 5;
    DevBuf buf;
    SECPE_CHECK(buf.alloc(ctx, sizeof(u64) * (size_t)nitem * nlimb * n));
    SECPE_CUDA(cudaMemsetAsync(buf.p, 0, buf.bytes, ctx->stream));
    LimbSet ls = make_limbset(buf.u(), nitem, (long long)nlimb * n, 1, 0, nlimb, 0);
    for (int j = 0; j < nlimb; j++) ls.prime_of[j] = (int8_t)(j % ctx->nprimes);
    cudaEvent_t e0, e1;
    SECPE_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SECPE_ECUDA;
    }
    const secpe_counters saved = ctx->counters;
    int st = SECPE_OK;
    float ms[TUNE_NSLOTS][2] = {};
    auto run = [&](int slot) {
        return slot == TUNE_BCONV ? bconv_pass_probe(ctx, buf.u(), nitem, nlimb - ctx->alpha)
                                  : ntt16_pass(ctx, slot, ls);
    };
    for (int slot = 0; slot < TUNE_NSLOTS && st == SECPE_OK; slot++) {
        // the candidates alternate, so that clock and thermal drift hit both;
        // each keeps the median of its launch times
        std::vector<float> t[2];
        for (int r = 0; r < 2 * reps + 2 && st == SECPE_OK; r++) {
            const int v = r & 1;
            ctx->tune.ctas[slot] = 3 + v;
            float m = 0.f;
            if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) st = SECPE_ECUDA;
            if (st == SECPE_OK) st = run(slot);
            if (st == SECPE_OK && (cudaEventRecord(e1, ctx->stream) != cudaSuccess ||
                                   cudaEventSynchronize(e1) != cudaSuccess ||
                                   cudaEventElapsedTime(&m, e0, e1) != cudaSuccess))
                st = SECPE_ECUDA;
            if (r >= 2) t[v].push_back(m);  // the first round of each is a warm-up
        }
        for (int v = 0; v < 2 && st == SECPE_OK; v++) {
            std::sort(t[v].begin(), t[v].end());
            ms[slot][v] = t[v][t[v].size() / 2];
        }
        // 4 CTAs per SM only for a clear win (it caps registers at 64)
        ctx->tune.ctas[slot] = ms[slot][1] < 0.97f * ms[slot][0] ? 4 : 3;
    }
    ctx->counters = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SECPE_OK) {
        for (int slot = 0; slot < TUNE_NSLOTS; slot++) ctx->tune.ctas[slot] = 3;
        return st;
    }
    ctx->tune.tuned = true;
    if (out) {
        out->n_kernels = TUNE_NSLOTS;
        for (int slot = 0; slot < TUNE_NSLOTS; slot++) {
            std::snprintf(out->name[slot], sizeof out->name[slot], "%s", kTuneNames[slot]);
            out->ctas_per_sm[slot] = ctx->tune.ctas[slot];
            out->ms[slot][0] = ms[slot][0];
            out->ms[slot][1] = ms[slot][1];
        }
    }
    return finish(ctx, SECPE_OK);
}

struct secpe_graph {
    secpe_ctx *ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    secpe_counters counts{};  // operation and kernel counts of one replay
};

extern "C" int secpe_argmax_batch_capture(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q,
                                          int n_queries, secpe_graph **out, int64_t *n_nodes) {
    if (!ctx || !q || n_queries < 1 || !out) return SECPE_EINVAL;
    *out = nullptr;
    cudaStream_t cs = nullptr;
    SECPE_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const secpe_counters saved = ctx->counters;
    const cudaStream_t saved_stream = ctx->stream;
    std::memset(&ctx->counters, 0, sizeof(ctx->counters));
    cudaGraph_t g = nullptr;
    int st = SECPE_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        st = SECPE_ECUDA;
    } else {
        ctx->stream = cs;
        st = argmax_batch_impl(ctx, keys, q, n_queries);
        if (cudaStreamEndCapture(cs, &g) != cudaSuccess && st == SECPE_OK) st = SECPE_ECUDA;
    }
    const secpe_counters captured = ctx->counters;
    ctx->counters = saved;
    ctx->stream = saved_stream;
    cudaGraphExec_t e = nullptr;
    if (st == SECPE_OK && (!g || cudaGraphInstantiate(&e, g, 0) != cudaSuccess)) st = SECPE_ECUDA;
    if (st == SECPE_OK && n_nodes) {
        size_t nn = 0;
        if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess) st = SECPE_ECUDA;
        *n_nodes = (int64_t)nn;
    }
    cudaStreamDestroy(cs);
    if (st != SECPE_OK) {
        if (e) cudaGraphExecDestroy(e);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st;
    }
    secpe_graph *r = new secpe_graph;
    r->ctx = ctx;
    r->graph = g;
    r->exec = e;
    r->counts = captured;
    *out = r;
    return SECPE_OK;
}

extern "C" int secpe_graph_launch(secpe_graph *g, void *stream) {
    if (!g || !g->exec) return SECPE_EINVAL;
    SECPE_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    secpe_counters &c = g->ctx->counters;
    c.rotations += g->counts.rotations;
    c.signs += g->counts.signs;
    c.relins += g->counts.relins;
    c.refreshes += g->counts.refreshes;
    c.keyswitches += g->counts.keyswitches;
    c.launches += g->counts.launches;
    return SECPE_OK;
}

extern "C" void secpe_graph_destroy(secpe_graph *g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    // hand the graph's allocations back to the device
    int dev = 0;
    if (cudaDeviceSynchronize() == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGraphMemTrim(dev);
}

extern "C" int secpe_pool_usage(int trim, uint64_t *used, uint64_t *reserved) {
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) {
        cudaGetLastError();
        return SECPE_ECUDA;
    }
    if (trim) {
        SECPE_CUDA(cudaDeviceSynchronize());
        SECPE_CUDA(cudaMemPoolTrimTo(pool, 0));
    }
    unsigned long long u = 0, r = 0;  // the attributes are 64-bit values
    SECPE_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u));
    SECPE_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r));
    if (used) *used = (uint64_t)u;
    if (reserved) *reserved = (uint64_t)r;
    return SECPE_OK;
}

extern "C" int secpe_kprof_begin(secpe_ctx *ctx, const char *name_filter, int max_launches) {
    if (!ctx || !name_filter || max_launches < 1 || max_launches > (1 << 20)) return SECPE_EINVAL;
    KProf &k = ctx->kprof;
    while ((int)k.ev.size() < 2 * max_launches) {
        cudaEvent_t e;
        SECPE_CUDA(cudaEventCreate(&e));
        k.ev.push_back(e);
    }
    k.filter = name_filter;
    k.all = k.filter == "*";
    k.used = 0;
    k.launches = 0;
    k.bytes = 0.0;
    k.model_bytes = 0.0;
    k.mul32 = 0.0;
    k.active = true;
    return SECPE_OK;
}

extern "C" int secpe_kprof_end(secpe_ctx *ctx, secpe_kprof *out) {
    if (!ctx || !out) return SECPE_EINVAL;
    KProf &k = ctx->kprof;
    k.active = false;
    SECPE_CUDA(cudaDeviceSynchronize());
    double ms = 0.0;
    k.ms.assign(k.used, 0.f);
    for (int i = 0; i < k.used; i++) {
        float t = 0.f;
        SECPE_CUDA(cudaEventElapsedTime(&t, k.ev[2 * i], k.ev[2 * i + 1]));
        k.ms[i] = t;
        ms += t;
    }
    out->launches = k.used;
    out->total_ms = ms;
    out->bytes = k.bytes;
    out->model_bytes = k.model_bytes;
    out->mul32 = k.mul32;
    return SECPE_OK;
}

extern "C" int secpe_mul32_probe(secpe_ctx *ctx, int ctas_per_sm, int iters, double *mul32_per_s, void *stream) {
    if (!ctx || !mul32_per_s || iters < 1 || iters > (1 << 20) || ctas_per_sm < 1 || ctas_per_sm > 32)
        return SECPE_EINVAL;
    CallScope cs(ctx, stream);
    int dev = 0, sms = 0;
    SECPE_CUDA(cudaGetDevice(&dev));
    SECPE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long blocks = (long long)sms * ctas_per_sm, threads = blocks * 256;
    DevBuf sink;
    SECPE_CHECK(sink.alloc(ctx, sizeof(u64) * (size_t)threads));
    cudaEvent_t e0, e1;
    SECPE_CUDA(cudaEventCreate(&e0));
    SECPE_CUDA(cudaEventCreate(&e1));
    int st = launch_mul32_probe(ctx, (unsigned)blocks, iters, sink.u());
    if (st == SECPE_OK && cudaEventRecord(e0, ctx->stream) != cudaSuccess) st = SECPE_ECUDA;
    if (st == SECPE_OK) st = launch_mul32_probe(ctx, (unsigned)blocks, iters, sink.u());
    if (st == SECPE_OK && cudaEventRecord(e1, ctx->stream) != cudaSuccess) st = SECPE_ECUDA;
    float ms = 0.f;
    if (st == SECPE_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        st = SECPE_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SECPE_OK) return st;
    *mul32_per_s = ms > 0.f ? (double)threads * iters * 4.0 * MUL32_MAC / (ms * 1e-3) : 0.0;
    return finish(ctx, SECPE_OK);
}

extern "C" int secpe_kprof_report(const secpe_ctx *ctx, char *buf, size_t len, size_t *needed) {
    if (!ctx || (!buf && len) || !needed) return SECPE_EINVAL;
    const KProf &k = ctx->kprof;
    if (k.active) return SECPE_EINVAL;
    std::map<std::string, std::pair<int64_t, double>> agg;
    for (int i = 0; i < (int)k.ms.size() && i < (int)k.names.size(); i++) {
        if (!k.names[i]) continue;
        auto &a = agg[k.names[i]];
        a.first++;
        a.second += k.ms[i];
    }
    std::vector<std::pair<double, std::string>> rows;
    for (auto &kv : agg) {
        char line[512];
        snprintf(line, sizeof line, "%s\t%lld\t%.6f\n", kv.first.c_str(), (long long)kv.second.first, kv.second.second);
        rows.push_back({kv.second.second, line});
    }
    std::sort(rows.begin(), rows.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    std::string text;
    for (auto &r : rows) text += r.second;
    *needed = text.size() + 1;
    if (len) {
        const size_t m = std::min(len - 1, text.size());
        memcpy(buf, text.data(), m);
        buf[m] = 0;
    }
    return SECPE_OK;
}

// ---------------------------------------------------------------- batched primitives
namespace {
int check_batch(const secpe_ctx *ctx, const secpe_ctbatch *b) {
    if (!b || !b->data || !aligned16(b->data) || (b->stride & 1) || b->batch < 1 || b->batch > SECPE_MAX_BATCH_CONST ||
        b->level < 0 || b->level > ctx->L || b->cap < b->level + 1 || b->stride < 2ull * b->cap * ctx->n ||
        !(b->scale > 0))
        return SECPE_EINVAL;
    return SECPE_OK;
}
Ct bview(secpe_ctx *ctx, const secpe_ctbatch *b) {
    Ct r;
    r.v.data = (u64 *)b->data;
    r.v.B = b->batch;
    r.v.cap = b->cap;
    r.v.stride = (long long)b->stride;
    r.v.level = b->level;
    r.v.scale = b->scale;
    r.v.n = ctx->n;
    return r;
}
// Output batch of a batched call: checked before anything is launched (the
// capacity is checked against the result's level when it is copied).
int check_batch_out(const secpe_ctx *ctx, const secpe_ctbatch *out, int batch) {
    if (!out || !out->data || !aligned16(out->data) || (out->stride & 1) || out->batch != batch || out->cap < 1 ||
        out->stride < 2ull * out->cap * ctx->n)
        return SECPE_EINVAL;
    return SECPE_OK;
}

int copy_batch_out(secpe_ctx *ctx, const Ct &src, secpe_ctbatch *dst) {
    if (dst->cap < src.level() + 1 || dst->batch != src.B()) return SECPE_EINVAL;
    const size_t n = ctx->n;
    for (int b = 0; b < src.B(); b++)
        SECPE_CUDA(cudaMemcpy2DAsync((u64 *)dst->data + b * dst->stride, sizeof(u64) * dst->cap * n,
                                     src.v.data + b * src.v.stride, sizeof(u64) * src.v.cap * n,
                                     sizeof(u64) * (src.level() + 1) * n, 2, cudaMemcpyDeviceToDevice, ctx->stream));
    dst->level = src.level();
    dst->scale = src.scale();
    return SECPE_OK;
}
}  // namespace

extern "C" int secpe_keyswitch_batch(secpe_ctx *ctx, const secpe_keys *keys, int galois_step,
                                     const secpe_ctbatch *d, secpe_ctbatch *out, void *stream) {
    if (!ctx || !keys || !out) return SECPE_EINVAL;
    SECPE_CHECK(check_batch(ctx, d));
    if (!out->data || !aligned16(out->data) || (out->stride & 1) || out->batch != d->batch ||
        out->cap < d->level + 1 || out->stride < 2ull * out->cap * ctx->n)
        return SECPE_EINVAL;
    CallScope cs(ctx, stream);
    const u64 *key = galois_step == 0 ? keys->rlk : galois_key(keys, galois_elt(ctx, galois_step));
    if (!key) return SECPE_EKEY;
    CtB o = {(u64 *)out->data, out->batch, (long long)out->stride, out->cap, d->level, d->scale, ctx->n};
    SECPE_CHECK(keyswitch(ctx, (const u64 *)d->data, (long long)d->stride, d->batch, d->level, key, o, false, false));
    out->level = d->level;
    out->scale = d->scale;
    return finish(ctx, SECPE_OK);
}

extern "C" int secpe_keyswitch_batch_tc(secpe_ctx *ctx, const secpe_keys *keys, int galois_step,
                                        const secpe_ctbatch *d, secpe_ctbatch *out, void *stream) {
    if (!ctx || !keys || !out) return SECPE_EINVAL;
    if (ctx->log_n != 16 || ctx->dnum > 8) return SECPE_EINVAL;
    SECPE_CHECK(check_batch(ctx, d));
    if (!out->data || !aligned16(out->data) || (out->stride & 1) || out->batch != d->batch ||
        out->cap < d->level + 1 || out->stride < 2ull * out->cap * ctx->n)
        return SECPE_EINVAL;
    CallScope cs(ctx, stream);
    const u64 *key = galois_step == 0 ? keys->rlk : galois_key(keys, galois_elt(ctx, galois_step));
    if (!key) return SECPE_EKEY;
    struct TcMode {
        secpe_ctx *c;
        explicit TcMode(secpe_ctx *x) : c(x) { c->tc_mode = 1; }
        ~TcMode() { c->tc_mode = 0; }
    } tm(ctx);
    CtB o = {(u64 *)out->data, out->batch, (long long)out->stride, out->cap, d->level, d->scale, ctx->n};
    SECPE_CHECK(keyswitch(ctx, (const u64 *)d->data, (long long)d->stride, d->batch, d->level, key, o, false, false));
    out->level = d->level;
    out->scale = d->scale;
    return finish(ctx, SECPE_OK);
}

extern "C" int secpe_mul_relin_batch(secpe_ctx *ctx, const secpe_keys *keys_, const secpe_ctbatch *a,
                                     const secpe_ctbatch *b, secpe_ctbatch *out, void *stream) {
    if (!ctx || !keys_ || !out) return SECPE_EINVAL;
    SECPE_CHECK(check_batch(ctx, a));
    SECPE_CHECK(check_batch(ctx, b));
    SECPE_CHECK(check_batch_out(ctx, out, a->batch));
    EVAL_PROLOGUE(ctx, stream);
    Ct r;
    SECPE_CHECK(E.mul(bview(ctx, a), bview(ctx, b), r));
    return finish(ctx, copy_batch_out(ctx, r, out));
}

extern "C" int secpe_rotate_batch(secpe_ctx *ctx, const secpe_keys *keys_, const secpe_ctbatch *in, int steps,
                                  secpe_ctbatch *out, void *stream) {
    if (!ctx || !keys_ || !out) return SECPE_EINVAL;
    SECPE_CHECK(check_batch(ctx, in));
    SECPE_CHECK(check_batch_out(ctx, out, in->batch));
    EVAL_PROLOGUE(ctx, stream);
    Ct r;
    SECPE_CHECK(E.rotate(bview(ctx, in), steps, r));
    return finish(ctx, copy_batch_out(ctx, r, out));
}

extern "C" int secpe_rescale_batch(secpe_ctx *ctx, const secpe_ctbatch *in, secpe_ctbatch *out, void *stream) {
    if (!ctx || !out) return SECPE_EINVAL;
    SECPE_CHECK(check_batch(ctx, in));
    SECPE_CHECK(check_batch_out(ctx, out, in->batch));
    const secpe_keys *keys_ = nullptr;
    EVAL_PROLOGUE(ctx, stream);
    Ct r;
    SECPE_CHECK(E.rescale(bview(ctx, in), r));
    return finish(ctx, copy_batch_out(ctx, r, out));
}

// ---------------------------------------------------------------- precision variant
extern "C" int secpe_ntt_tc(secpe_ctx *ctx, uint64_t *limbs, const int32_t *prime_idx, int count, int inverse,
                            void *stream) {
    if (!ctx || !limbs || !aligned16(limbs) || !prime_idx || count < 0 || ctx->log_n != 16) return SECPE_EINVAL;
    CallScope cs(ctx, stream);
    for (int s = 0; s < count; s += SECPE_MAX_LIMBSET) {
        const int c = std::min(SECPE_MAX_LIMBSET, count - s);
        LimbSet ls = make_limbset((u64 *)limbs + (size_t)s * ctx->n, 1, 0, 1, 0, c, 0);
        for (int j = 0; j < c; j++) {
            if (prime_idx[s + j] < 0 || prime_idx[s + j] >= ctx->nprimes) return SECPE_EINVAL;
            ls.prime_of[j] = (int8_t)prime_idx[s + j];
        }
        SECPE_CHECK(ntt_limbset_tc(ctx, ls, inverse != 0));
    }
    return finish(ctx, SECPE_OK);
}

extern "C" int secpe_ntt_cts_tc(secpe_ctx *ctx, uint64_t *base, int batch, size_t ct_stride, int cap, int level,
                                int inverse, void *stream) {
    if (!ctx || !base || !aligned16(base) || (ct_stride & 1) || batch < 0 || level < 0 || level >= cap ||
        level > ctx->L || ctx->log_n != 16 || ct_stride < 2ull * cap * ctx->n)
        return SECPE_EINVAL;
    CallScope cs(ctx, stream);
    LimbSet ls = make_limbset((u64 *)base, batch, (long long)ct_stride, 2, (long long)cap * ctx->n, level + 1, 0);
    return finish(ctx, ntt_limbset_tc(ctx, ls, inverse != 0));
}

extern "C" int secpe_expand_seeded(secpe_ctx *ctx, uint64_t *base, int batch, size_t ct_stride, int cap, int level,
                                   const uint64_t *seeds, void *stream) {
    if (!ctx || !base || !aligned16(base) || (ct_stride & 1) || !seeds || batch < 0 || level < 0 || level > ctx->L ||
        cap < level + 1 || ct_stride < 2ull * cap * ctx->n)
        return SECPE_EINVAL;
    CallScope cs(ctx, stream);
    PrimeList pl;
    pl.n = level + 1;
    for (int i = 0; i <= level; i++) pl.p[i] = i;
    for (int s0 = 0; s0 < batch; s0 += SECPE_MAX_BATCH_CONST) {
        const int c = std::min(SECPE_MAX_BATCH_CONST, batch - s0);
        std::vector<u64> keys(c);
        for (int i = 0; i < c; i++) keys[i] = hm::sm_stream(seeds[s0 + i], DOM_ENC_A, 0);
        u64 *c1 = (u64 *)base + (size_t)s0 * ct_stride + (size_t)cap * ctx->n;
        SECPE_CHECK(launch_sample_uniform(ctx, keys, c1, (long long)ct_stride, pl));
    }
    return finish(ctx, SECPE_OK);
}
