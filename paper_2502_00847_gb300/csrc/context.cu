// Context creation: primes, NTT twiddles and every base-conversion / rescale
// / CRT constant, computed on the host and uploaded once to the device.
#include <cstring>

#include "internal.h"
#include "launch.h"

namespace {

template <typename T>
T *upload(secpe_ctx *ctx, const std::vector<T> &v) {
    void *d = nullptr;
    size_t bytes = sizeof(T) * (v.empty() ? 1 : v.size());
    if (cudaMalloc(&d, bytes) != cudaSuccess) return nullptr;
    if (!v.empty() && cudaMemcpy(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) !=
                          cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    ctx->allocations.push_back(d);
    return (T *)d;
}

ulonglong2 sh(u64 w, u64 q) { return make_ulonglong2(w, hm::shoup(w, q)); }

u64 mont(u64 x, u64 q) {  // x * 2^64 mod q
    return (u64)((((u128)(x % q)) << 64) % q);
}

}  // namespace

extern "C" int secpe_ctx_create(const secpe_params *p, secpe_ctx **out) {
    if (!p || !out) return SECPE_EINVAL;
    *out = nullptr;
    if (p->dnum < 1 || p->dnum > p->n_q || p->log_scale < 10 || p->log_scale > 58 ||
        p->reserve < 1 || p->sign_dg < 0 || p->sign_df < 0 || p->sign_dg + p->sign_df < 1 || p->secret_hw < 0 ||
        (p->log_n >= 4 && p->log_n <= 17 && p->secret_hw > (1 << p->log_n)))
        return SECPE_EINVAL;
    std::vector<u64> qs, sp;
    if (!hm::select_primes(*p, qs, sp)) return SECPE_EINVAL;
    int alpha = (p->n_q + p->dnum - 1) / p->dnum;
    if (alpha > 15 || p->dnum > 15) return SECPE_EINVAL;
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) return SECPE_ECUDA;

    secpe_ctx *ctx = new secpe_ctx();
    ctx->p = *p;
    ctx->log_n = p->log_n;
    ctx->n = 1 << p->log_n;
    ctx->nq = p->n_q;
    ctx->npsp = p->n_p;
    ctx->nprimes = p->n_q + p->n_p;
    ctx->L = p->n_q - 1;
    ctx->dnum = p->dnum;
    ctx->alpha = alpha;
    ctx->primes = qs;
    ctx->primes.insert(ctx->primes.end(), sp.begin(), sp.end());
    ctx->scale = std::ldexp(1.0, p->log_scale);
    ctx->stream = 0;
    std::memset(&ctx->counters, 0, sizeof(ctx->counters));

    const int n = ctx->n, np = ctx->nprimes, nq = ctx->nq, L = ctx->L, k = ctx->npsp;
    const std::vector<u64> &P = ctx->primes;

    std::vector<u64> qinv(np), r2(np), mu(np), mone(np);
    std::vector<ulonglong2> twf((size_t)np * n), twi((size_t)np * n), ninv(np), ninvw1(np);
    for (int t = 0; t < np; t++) {
        u64 q = P[t];
        qinv[t] = hm::neg_inv64(q);
        u64 r = (u64)((((u128)1) << 64) % q);
        r2[t] = hm::mulmod(r, r, q);
        mone[t] = r;
        mu[t] = (u64)((((u128)1) << 64) / q);
        u64 psi = hm::find_psi(q, n);
        ctx->psi.push_back(psi);
        u64 psi_inv = hm::invmod(psi, q);
        std::vector<u64> pw(n), ipw(n);
        pw[0] = ipw[0] = 1;
        for (int i = 1; i < n; i++) {
            pw[i] = hm::mulmod(pw[i - 1], psi, q);
            ipw[i] = hm::mulmod(ipw[i - 1], psi_inv, q);
        }
        for (int i = 0; i < n; i++) {
            uint32_t b = hm::bitrev(i, ctx->log_n);
            twf[(size_t)t * n + i] = sh(pw[b], q);
            twi[(size_t)t * n + i] = sh(ipw[b], q);
        }
        u64 ni = hm::invmod((u64)n, q);
        ninv[t] = sh(ni, q);
        ninvw1[t] = sh(hm::mulmod(ni, ipw[hm::bitrev(1, ctx->log_n)], q), q);
    }
    ctx->h_qinv_neg = qinv;
    ctx->h_r2 = r2;
    ctx->h_mu = mu;

    // ModUp tables per (level, digit)
    std::vector<ulonglong2> mu_inv((size_t)(L + 1) * ctx->dnum * alpha, make_ulonglong2(0, 0));
    std::vector<u64> mu_hat((size_t)(L + 1) * ctx->dnum * alpha * np, 0);
    for (int lv = 0; lv <= L; lv++) {
        for (int j = 0; j < ctx->dnum; j++) {
            int lo = j * alpha, hi = std::min((j + 1) * alpha, lv + 1);
            if (lo > lv) break;
            for (int i = lo; i < hi; i++) {
                // Qhat_i = prod_{i' in digit, i' != i} q_i'
                u64 prod = 1;
                for (int i2 = lo; i2 < hi; i2++)
                    if (i2 != i) prod = hm::mulmod(prod, P[i2] % P[i], P[i]);
                size_t base = ((size_t)lv * ctx->dnum + j) * alpha + (i - lo);
                mu_inv[base] = sh(hm::invmod(prod, P[i]), P[i]);
                for (int t = 0; t < np; t++) {
                    u64 h = 1 % P[t];
                    for (int i2 = lo; i2 < hi; i2++)
                        if (i2 != i) h = hm::mulmod(h, P[i2] % P[t], P[t]);
                    mu_hat[base * np + t] = mont(h, P[t]);
                }
            }
        }
    }

    ctx->h_mu_inv = mu_inv;
    std::vector<ulonglong2> ninv_modup((size_t)2 * nq * nq, make_ulonglong2(0, 0));
    for (int lv = 0; lv <= L; lv++)
        for (int i = 0; i <= lv; i++) {
            const int j = i / alpha;
            const size_t base = ((size_t)lv * ctx->dnum + j) * alpha + (i - j * alpha);
            const u64 q = P[i];
            const u64 ni = hm::invmod((u64)n, q);
            const u64 s0 = hm::mulmod(ni, mu_inv[base].x, q);
            const u64 w1 = hm::invmod(hm::powmod(ctx->psi[i], hm::bitrev(1, ctx->log_n), q), q);
            ninv_modup[2 * ((size_t)lv * nq + i)] = sh(s0, q);
            ninv_modup[2 * ((size_t)lv * nq + i) + 1] = sh(hm::mulmod(s0, w1, q), q);
        }

    // ModDown tables
    std::vector<ulonglong2> md_inv(k), md_pinv(nq);
    std::vector<u64> md_hat((size_t)k * nq), md_hP(np);
    for (int j = 0; j < k; j++) {
        u64 pj = P[nq + j];
        u64 prod = 1;
        for (int j2 = 0; j2 < k; j2++)
            if (j2 != j) prod = hm::mulmod(prod, P[nq + j2] % pj, pj);
        md_inv[j] = sh(hm::invmod(prod, pj), pj);
        for (int i = 0; i < nq; i++) {
            u64 h = 1 % P[i];
            for (int j2 = 0; j2 < k; j2++)
                if (j2 != j) h = hm::mulmod(h, P[nq + j2] % P[i], P[i]);
            md_hat[(size_t)j * nq + i] = mont(h, P[i]);
        }
    }
    for (int i = 0; i < nq; i++) {
        u64 pm = 1;
        for (int j = 0; j < k; j++) pm = hm::mulmod(pm, P[nq + j] % P[i], P[i]);
        md_pinv[i] = sh(hm::invmod(pm, P[i]), P[i]);
    }
    std::vector<ulonglong2> ninv_moddown((size_t)2 * k);
    for (int j = 0; j < k; j++) {
        const u64 q = P[nq + j];
        const u64 ni = hm::invmod((u64)n, q);
        const u64 s0 = hm::mulmod(ni, md_inv[j].x, q);
        const u64 w1 = hm::invmod(hm::powmod(ctx->psi[nq + j], hm::bitrev(1, ctx->log_n), q), q);
        ninv_moddown[2 * j] = sh(s0, q);
        ninv_moddown[2 * j + 1] = sh(hm::mulmod(s0, w1, q), q);
    }
    // floor(P/2) mod t: P is odd, so floor(P/2) = (P - 1)/2 = (P - 1) * 2^-1 mod t
    for (int t = 0; t < np; t++) {
        u64 pm = 1;
        for (int j = 0; j < k; j++) pm = hm::mulmod(pm, P[nq + j] % P[t], P[t]);
        u64 pm1 = (pm + P[t] - 1) % P[t];
        md_hP[t] = hm::mulmod(pm1, hm::invmod(2, P[t]), P[t]);
    }

    // Relinearisation ModDown + rescale tables (per level l >= 1)
    const int ks = k + 1;
    std::vector<ulonglong2> mdr_ninv((size_t)2 * nq * ks, make_ulonglong2(0, 0)), mdr_inv((size_t)nq * ks,
                                                                                         make_ulonglong2(0, 0));
    std::vector<ulonglong2> mdr_w((size_t)nq * nq, make_ulonglong2(0, 0));
    std::vector<u64> mdr_pre((size_t)nq * ks, 0), mdr_hat((size_t)nq * ks * nq, 0), mdr_post((size_t)nq * nq, 0);
    std::vector<u64> mdr_pre_scaled((size_t)nq * ks, 0), pmod(np);
    for (int t = 0; t < np; t++) {
        u64 pm = 1;
        for (int j = 0; j < k; j++) pm = hm::mulmod(pm, P[nq + j] % P[t], P[t]);
        pmod[t] = pm;
    }
    for (int lv = 1; lv < nq; lv++) {
        std::vector<int> src(ks);
        src[0] = lv;
        for (int j = 0; j < k; j++) src[1 + j] = nq + j;
        for (int j = 0; j < ks; j++) {
            const u64 s_ = P[src[j]];
            u64 mh = 1;  // M / s_j mod s_j
            for (int j2 = 0; j2 < ks; j2++)
                if (j2 != j) mh = hm::mulmod(mh, P[src[j2]] % s_, s_);
            const u64 inv = hm::invmod(mh, s_);
            mdr_inv[(size_t)lv * ks + j] = sh(inv, s_);
            u64 mm = 1;  // M mod s_j
            for (int j2 = 0; j2 < ks; j2++) mm = hm::mulmod(mm, P[src[j2]] % s_, s_);
            const u64 hmod = hm::mulmod((mm + s_ - 1) % s_, hm::invmod(2, s_), s_);
            mdr_pre[(size_t)lv * ks + j] = hmod;
            mdr_pre_scaled[(size_t)lv * ks + j] = hm::mulmod(hmod, inv, s_);
            const u64 ni = hm::invmod((u64)n, s_);
            const u64 s0 = hm::mulmod(ni, inv, s_);
            const u64 w1 = hm::invmod(hm::powmod(ctx->psi[src[j]], hm::bitrev(1, ctx->log_n), s_), s_);
            mdr_ninv[2 * ((size_t)lv * ks + j)] = sh(s0, s_);
            mdr_ninv[2 * ((size_t)lv * ks + j) + 1] = sh(hm::mulmod(s0, w1, s_), s_);
            for (int i = 0; i < nq; i++) {
                u64 hq = 1;
                for (int j2 = 0; j2 < ks; j2++)
                    if (j2 != j) hq = hm::mulmod(hq, P[src[j2]] % P[i], P[i]);
                mdr_hat[((size_t)lv * ks + j) * nq + i] = mont(hq, P[i]);
            }
        }
        for (int i = 0; i < nq; i++) {
            u64 mm = 1;
            for (int j2 = 0; j2 < ks; j2++) mm = hm::mulmod(mm, P[src[j2]] % P[i], P[i]);
            mdr_post[(size_t)lv * nq + i] = hm::mulmod((mm + P[i] - 1) % P[i], hm::invmod(2, P[i]), P[i]);
            if (i < lv) mdr_w[(size_t)lv * nq + i] = sh(hm::invmod(mm, P[i]), P[i]);
        }
    }
    ctx->h_mdr_pre_scaled = mdr_pre_scaled;

    // Rescale tables
    std::vector<ulonglong2> rs_qinv((size_t)nq * nq, make_ulonglong2(0, 0));
    std::vector<u64> rs_hmod((size_t)nq * nq, 0);
    for (int lv = 1; lv < nq; lv++)
        for (int i = 0; i < lv; i++) {
            rs_qinv[(size_t)lv * nq + i] = sh(hm::invmod(P[lv] % P[i], P[i]), P[i]);
            rs_hmod[(size_t)lv * nq + i] = (P[lv] / 2) % P[i];
        }

    // Mixed-radix CRT tables
    std::vector<ulonglong2> mr_inv((size_t)nq * nq, make_ulonglong2(0, 0));
    std::vector<u64> mr_M((size_t)nq * nq), mr_H((size_t)nq * nq, 0), mr_Q((size_t)nq * nq);
    std::vector<double> mr_Mf(nq);
    for (int j = 0; j < nq; j++)
        for (int i = j + 1; i < nq; i++) mr_inv[(size_t)j * nq + i] = sh(hm::invmod(P[j] % P[i], P[i]), P[i]);
    for (int i = 0; i < nq; i++) {
        double mf = 1.0;
        for (int j = 0; j < i; j++) mf *= (double)P[j];
        mr_Mf[i] = mf;
        for (int t = 0; t < nq; t++) {
            u64 m = 1 % P[t];
            for (int j = 0; j < i; j++) m = hm::mulmod(m, P[j] % P[t], P[t]);
            mr_M[(size_t)i * nq + t] = m;
        }
    }
    for (int lv = 0; lv < nq; lv++) {
        // residues of H = (Q_l - 1)/2 are (q_i - 1)/2; convert to mixed radix
        std::vector<u64> v(lv + 1);
        for (int i = 0; i <= lv; i++) {
            u64 x = (P[i] - 1) / 2;
            for (int j = 0; j < i; j++) x = hm::mulmod((x + P[i] - v[j] % P[i]) % P[i], hm::invmod(P[j] % P[i], P[i]), P[i]);
            v[i] = x;
            mr_H[(size_t)lv * nq + i] = x;
        }
        for (int t = 0; t < nq; t++) {
            u64 m = 1 % P[t];
            for (int j = 0; j <= lv; j++) m = hm::mulmod(m, P[j] % P[t], P[t]);
            mr_Q[(size_t)lv * nq + t] = m;
        }
    }

    DevCtx &d = ctx->dev;
    d.log_n = ctx->log_n;
    d.n = n;
    d.nq = nq;
    d.np_special = k;
    d.nprimes = np;
    d.dnum = ctx->dnum;
    d.alpha = alpha;
    bool ok = true;
#define UP(field, vec)                       \
    do {                                     \
        d.field = upload(ctx, vec);          \
        ok = ok && (d.field != nullptr);     \
    } while (0)
    UP(q, P);
    UP(qinv_neg, qinv);
    UP(r2, r2);
    UP(mu, mu);
    UP(mont_one, mone);
    UP(tw_fwd, twf);
    UP(tw_inv, twi);
    UP(ninv, ninv);
    UP(ninv_w1, ninvw1);
    UP(ninv_modup, ninv_modup);
    UP(ninv_moddown, ninv_moddown);
    UP(mu_inv, mu_inv);
    UP(mu_hat, mu_hat);
    UP(md_inv, md_inv);
    UP(md_hat, md_hat);
    UP(md_pinv, md_pinv);
    UP(md_hP, md_hP);
    UP(mdr_ninv, mdr_ninv);
    UP(mdr_inv, mdr_inv);
    UP(mdr_pre, mdr_pre);
    UP(mdr_hat, mdr_hat);
    UP(mdr_post, mdr_post);
    UP(mdr_w, mdr_w);
    UP(pmod, pmod);
    UP(rs_qinv, rs_qinv);
    UP(rs_hmod, rs_hmod);
    UP(mr_inv, mr_inv);
    UP(mr_M, mr_M);
    UP(mr_H, mr_H);
    UP(mr_Q, mr_Q);
    UP(mr_Mf, mr_Mf);
#undef UP
    std::vector<int> zero(1, 0);
    ctx->d_status = upload(ctx, zero);
    d.status = ctx->d_status;
    if (!ok || !ctx->d_status) {
        secpe_ctx_destroy(ctx);
        return SECPE_ENOMEM;
    }
    // keep freed stream-ordered allocations cached in the pool
    int devid = 0;
    cudaGetDevice(&devid);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, devid) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = ctx;
    return SECPE_OK;
}

extern "C" void secpe_ctx_destroy(secpe_ctx *ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    tc_forget_ctx(ctx);
    for (void *p : ctx->allocations) cudaFree(p);
    delete ctx;
}

extern "C" int secpe_ctx_primes(const secpe_ctx *ctx, uint64_t *out) {
    if (!ctx || !out) return SECPE_EINVAL;
    for (size_t i = 0; i < ctx->primes.size(); i++) out[i] = ctx->primes[i];
    return SECPE_OK;
}

extern "C" int secpe_select_primes(const secpe_params *p, uint64_t *out, int capacity) {
    if (!p || !out) return SECPE_EINVAL;
    std::vector<u64> qs, sp;
    if (!hm::select_primes(*p, qs, sp)) return SECPE_EINVAL;
    if (capacity < (int)(qs.size() + sp.size())) return SECPE_EINVAL;
    for (size_t i = 0; i < qs.size(); i++) out[i] = qs[i];
    for (size_t i = 0; i < sp.size(); i++) out[qs.size() + i] = sp[i];
    return SECPE_OK;
}

extern "C" int secpe_ctx_n(const secpe_ctx *ctx) { return ctx ? ctx->n : 0; }
