// Hybrid key switching (ModUp -> key inner product -> ModDown) and rescale,
// orchestrated over batches of ciphertexts.
//
// Key switching of d (limbs 0..l, NTT form) with key (b_j, a_j), j < dnum:
//  1. INTT of d.
//  2. ModUp, per digit j = primes [j alpha, min((j+1) alpha, l+1)):
//     FastBConv of the digit's limbs to every other prime of Q_l u P
//     (no correction), then NTT of those limbs.  The digit's own limbs are d.
//  3. Inner product over digits with the key, in Montgomery form, one
//     reduction per output residue (lazy accumulation in 128 bits).
//  4. ModDown: INTT of the special-prime limbs, rounded FastBConv to q_i
//     (add floor(P/2) before, subtract it after), NTT, then
//     (x_i - conv_i) * P^-1.
// Rescale: INTT of the last limb, per other prime ([y + h]_{q_l} - h) mod
// q_i, NTT, (x_i - z_i) * q_l^-1.
#include "eval.h"

int keyswitch_acc(secpe_ctx *ctx, const u64 *d, long long d_item_stride, int B, int lv, const u64 *key, DevBuf &acc) {
    const int n = ctx->n, k = ctx->npsp, alpha = ctx->alpha;
    const int nt = lv + 1 + k;
    KsDigits dg;
    dg.ndig = 0;
    int tot = 0;
    LimbSet ext_ls;
    ext_ls.npoly = 1;
    for (int j = 0; j * alpha <= lv; j++) {
        const int lo = j * alpha, hi = std::min((j + 1) * alpha, lv + 1);
        dg.lo[j] = lo;
        dg.hi[j] = hi;
        dg.off[j] = tot;
        for (int t = 0; t < nt; t++) {
            if (t >= lo && t < hi) continue;
            if (tot >= SECPE_MAX_LIMBSET) return SECPE_EINVAL;
            ext_ls.prime_of[tot] = (int8_t)(t <= lv ? t : ctx->nq + (t - lv - 1));
            ext_ls.aux[tot] = 0;
            tot++;
        }
        dg.ndig++;
    }
    ctx->counters.keyswitches++;
    SECPE_CHECK(acc.alloc(ctx, sizeof(u64) * (size_t)B * 2 * nt * n));

    // 1. INTT of d into dcoef [B][lv+1][N] (on the fused path the INTT also
    //    applies the ModUp pre-multiplier [Qhat_i^-1]_{q_i})
    DevBuf dcoef;
    SECPE_CHECK(dcoef.alloc(ctx, sizeof(u64) * (size_t)B * (lv + 1) * n));
    LimbSet dst = make_limbset(dcoef.u(), B, (long long)(lv + 1) * n, 1, 0, lv + 1, 0);
    LimbSet src = make_limbset((u64 *)d, B, d_item_stride, 1, 0, lv + 1, 0);
    const bool fused = fused_path(ctx);
    // (the profiler charges this INTT the key switch's input d, read once)
    SECPE_CHECK(ntt_limbset(ctx, dst, true, &src, fused ? ctx->dev.ninv_modup : nullptr, lv * ctx->nq, 8.0 * n));

    DevBuf ext;
    SECPE_CHECK(ext.alloc(ctx, sizeof(u64) * (size_t)B * tot * n));
    if (fused) return modup_ip_fused(ctx, d, d_item_stride, dcoef.u(), B, lv, dg, tot, key, ext.u(), acc.u());

    // 2. ModUp: FastBConv per digit, NTT of the extended limbs
    const long long ext_stride = (long long)tot * n;
    for (int j = 0; j < dg.ndig; j++) {
        const int ntgt = nt - (dg.hi[j] - dg.lo[j]);
        SECPE_CHECK(launch_modup_bconv(ctx, dcoef.u(), ext.u(), ext_stride, dg.off[j], B, lv, j, dg.lo[j],
                                       dg.hi[j], ntgt));
    }
    dcoef.release();
    ext_ls.base = ext.u();
    ext_ls.nitem = B;
    ext_ls.item_stride = ext_stride;
    ext_ls.poly_stride = 0;
    ext_ls.nlimb = tot;
    SECPE_CHECK(ntt_limbset(ctx, ext_ls, false));
    // 3. inner product -> acc [B][2][nt][N]
    return launch_ksk_ip(ctx, d, d_item_stride, ext.u(), ext_stride, dg, key, acc.u(), B, lv);
}

int keyswitch(secpe_ctx *ctx, const u64 *d, long long d_item_stride, int B, int lv, const u64 *key,
              const CtB &out, bool acc0, bool acc1) {
    if (B == 0) return SECPE_OK;
    const int n = ctx->n, k = ctx->npsp, nt = lv + 1 + k;
    DevBuf acc, tmp;
    SECPE_CHECK(keyswitch_acc(ctx, d, d_item_stride, B, lv, key, acc));
    // 4. ModDown
    LimbSet pls = make_limbset(acc.u() + (size_t)(lv + 1) * n, B, 2ll * nt * n, 2, (long long)nt * n, k, ctx->nq);
    SECPE_CHECK(tmp.alloc(ctx, sizeof(u64) * (size_t)B * 2 * (lv + 1) * n));
    if (fused_path(ctx)) {
        SECPE_CHECK(ntt_limbset(ctx, pls, true, nullptr, ctx->dev.ninv_moddown, 0, 0.0));  // intermediate
        return moddown_fused(ctx, acc.u(), B, lv, out, acc0, acc1, tmp.u());
    }
    SECPE_CHECK(ntt_limbset(ctx, pls, true));
    SECPE_CHECK(launch_moddown_bconv(ctx, acc.u(), tmp.u(), B, lv));
    LimbSet cls = make_limbset(tmp.u(), B, 2ll * (lv + 1) * n, 2, (long long)(lv + 1) * n, lv + 1, 0);
    SECPE_CHECK(ntt_limbset(ctx, cls, false));
    return launch_moddown_fin(ctx, acc.u(), tmp.u(), out, lv, acc0, acc1);
}

// Digits of level lv and the prime of every extended limb, in the order
// keyswitch_acc lays them out.
static int ks_digits(const secpe_ctx *ctx, int lv, KsDigits &dg, LimbSet &ext_ls, int &tot) {
    const int k = ctx->npsp, alpha = ctx->alpha, nt = lv + 1 + k;
    dg.ndig = 0;
    tot = 0;
    ext_ls.npoly = 1;
    for (int j = 0; j * alpha <= lv; j++) {
        const int lo = j * alpha, hi = std::min((j + 1) * alpha, lv + 1);
        dg.lo[j] = lo;
        dg.hi[j] = hi;
        dg.off[j] = tot;
        for (int t = 0; t < nt; t++) {
            if (t >= lo && t < hi) continue;
            if (tot >= SECPE_MAX_LIMBSET) return SECPE_EINVAL;
            ext_ls.prime_of[tot] = (int8_t)(t <= lv ? t : ctx->nq + (t - lv - 1));
            ext_ls.aux[tot] = 0;
            tot++;
        }
        dg.ndig++;
    }
    return SECPE_OK;
}

// Hoisting: the ModUp of x's second polynomial once (INTT, FastBConv per
// digit, NTT: the extended limbs in NTT form), then per Galois element
// gal[i]: the automorphism onto x (into outs[i]) and onto every extended
// limb, the key inner product with keys[i] and ModDown, so that
// outs[i] = (sigma(c0) + ks0, ks1).  The automorphism of an extended limb
// differs from the ModUp of the automorphism only by the permuted multiple
// of the digit modulus that FastBConv leaves.
int rotate_hoisted(secpe_ctx *ctx, const CtB &x, const std::vector<unsigned> &gal, const std::vector<const u64 *> &keys,
                   const std::vector<CtB> &outs) {
    const int n = ctx->n, k = ctx->npsp, B = x.B, lv = x.level, nt = lv + 1 + k;
    if (gal.size() != keys.size() || gal.size() != outs.size() || B < 1) return SECPE_EINVAL;
    if (gal.empty()) return SECPE_OK;
    KsDigits dg;
    LimbSet ext_ls;
    int tot = 0;
    SECPE_CHECK(ks_digits(ctx, lv, dg, ext_ls, tot));
    if ((long long)B * tot > 65535) return SECPE_EINVAL;
    // 1. INTT of c1 (plain coefficients: the ModUp kernel applies [Qhat_i^-1])
    DevBuf dcoef, ext, sext, acc, tmp;
    SECPE_CHECK(dcoef.alloc(ctx, sizeof(u64) * (size_t)B * (lv + 1) * n));
    LimbSet dst = make_limbset(dcoef.u(), B, (long long)(lv + 1) * n, 1, 0, lv + 1, 0);
    LimbSet src = make_limbset(x.data + x.pstride(), B, x.stride, 1, 0, lv + 1, 0);
    SECPE_CHECK(ntt_limbset(ctx, dst, true, &src, nullptr, 0, 8.0 * n));
    // 2. ModUp per digit, then the NTT of every extended limb
    const long long ext_stride = (long long)tot * n;
    SECPE_CHECK(ext.alloc(ctx, sizeof(u64) * (size_t)B * tot * n));
    for (int j = 0; j < dg.ndig; j++) {
        const int ntgt = nt - (dg.hi[j] - dg.lo[j]);
        SECPE_CHECK(launch_modup_bconv(ctx, dcoef.u(), ext.u(), ext_stride, dg.off[j], B, lv, j, dg.lo[j],
                                       dg.hi[j], ntgt));
    }
    dcoef.release();
    ext_ls.base = ext.u();
    ext_ls.nitem = B;
    ext_ls.item_stride = ext_stride;
    ext_ls.poly_stride = 0;
    ext_ls.nlimb = tot;
    SECPE_CHECK(ntt_limbset(ctx, ext_ls, false));
    if (ctx->tc_mode) SECPE_CHECK(sext.alloc(ctx, sizeof(u64) * (size_t)B * tot * n));
    SECPE_CHECK(acc.alloc(ctx, sizeof(u64) * (size_t)B * 2 * nt * n));
    SECPE_CHECK(tmp.alloc(ctx, sizeof(u64) * (size_t)B * 2 * (lv + 1) * n));
    // 3. per rotation: automorphisms, inner product, ModDown
    for (size_t i = 0; i < gal.size(); i++) {
        const CtB &o = outs[i];
        if (o.B != B || o.cap < lv + 1 || !keys[i]) return SECPE_EINVAL;
        SECPE_CHECK(launch_automorph(ctx, x, o, lv + 1, gal[i]));
        ctx->counters.keyswitches++;
        if (ctx->tc_mode) {
            // the precision variant's inner product reads a permuted copy
            SECPE_CHECK(launch_automorph_flat(ctx, ext.u(), sext.u(), (long long)B * tot, gal[i]));
            SECPE_CHECK(launch_ksk_ip(ctx, o.data + o.pstride(), o.stride, sext.u(), ext_stride, dg, keys[i],
                                      acc.u(), B, lv));
        } else {
            // the inner product reads the extended limbs through the automorphism
            SECPE_CHECK(launch_ksk_ip(ctx, o.data + o.pstride(), o.stride, ext.u(), ext_stride, dg, keys[i],
                                      acc.u(), B, lv, gal[i]));
        }
        LimbSet pls =
            make_limbset(acc.u() + (size_t)(lv + 1) * n, B, 2ll * nt * n, 2, (long long)nt * n, k, ctx->nq);
        if (fused_path(ctx)) {
            SECPE_CHECK(ntt_limbset(ctx, pls, true, nullptr, ctx->dev.ninv_moddown, 0, 0.0));
            SECPE_CHECK(moddown_fused(ctx, acc.u(), B, lv, o, true, false, tmp.u()));
        } else {
            SECPE_CHECK(ntt_limbset(ctx, pls, true));
            SECPE_CHECK(launch_moddown_bconv(ctx, acc.u(), tmp.u(), B, lv));
            LimbSet cls = make_limbset(tmp.u(), B, 2ll * (lv + 1) * n, 2, (long long)(lv + 1) * n, lv + 1, 0);
            SECPE_CHECK(ntt_limbset(ctx, cls, false));
            SECPE_CHECK(launch_moddown_fin(ctx, acc.u(), tmp.u(), o, lv, true, false));
        }
    }
    return SECPE_OK;
}

int relin_rescale_batch(secpe_ctx *ctx, const u64 *d, int B, int lv, const u64 *key, const CtB &out) {
    if (B == 0) return SECPE_OK;
    const int n = ctx->n, k = ctx->npsp, nt = lv + 1 + k;
    const long long dis = 3ll * (lv + 1) * n, dps = (long long)(lv + 1) * n;
    DevBuf acc, tmp;
    SECPE_CHECK(keyswitch_acc(ctx, d + 2 * dps, dis, B, lv, key, acc));
    SECPE_CHECK(tmp.alloc(ctx, sizeof(u64) * (size_t)B * 2 * lv * n));
    if (fused_path(ctx)) return moddown_rescale_fused(ctx, acc.u(), d, B, lv, out, tmp.u());
    SECPE_CHECK(launch_mdr_prep(ctx, d, dis, dps, acc.u(), B, lv));
    LimbSet src = make_limbset(acc.u() + (size_t)lv * n, B, 2ll * nt * n, 2, (long long)nt * n, k + 1, 0);
    for (int p = 0; p < 2; p++)
        for (int j = 0; j <= k; j++) src.prime_of[p * (k + 1) + j] = (int8_t)(j == 0 ? lv : ctx->nq + j - 1);
    SECPE_CHECK(ntt_limbset(ctx, src, true));
    SECPE_CHECK(launch_mdr_bconv(ctx, acc.u(), tmp.u(), B, lv));
    LimbSet cls = make_limbset(tmp.u(), B, 2ll * lv * n, 2, (long long)lv * n, lv, 0);
    SECPE_CHECK(ntt_limbset(ctx, cls, false));
    return launch_mdr_fin(ctx, acc.u(), tmp.u(), d, dis, dps, out, lv);
}

int rescale_batch(secpe_ctx *ctx, const CtB &in, const CtB &out, const long long *add_k) {
    const int lv = in.level, n = ctx->n, B = in.B;
    if (lv < 1) return SECPE_ELEVEL;
    DevBuf y, z;
    SECPE_CHECK(y.alloc(ctx, sizeof(u64) * (size_t)B * 2 * n));
    SECPE_CHECK(z.alloc(ctx, sizeof(u64) * (size_t)B * 2 * lv * n));
    LimbSet ysrc = make_limbset(in.data + (size_t)lv * n, B, in.stride, 2, in.pstride(), 1, lv);
    LimbSet ydst = make_limbset(y.u(), B, 2ll * n, 2, n, 1, lv);
    // (charged the input's last limbs, read once)
    SECPE_CHECK(ntt_limbset(ctx, ydst, true, &ysrc, nullptr, 0, 8.0 * n));
    if (fused_path(ctx)) return rescale_fused(ctx, in, y.u(), out, z.u(), add_k);
    SECPE_CHECK(launch_rescale_prep(ctx, y.u(), z.u(), B, lv));
    LimbSet zls = make_limbset(z.u(), B, 2ll * lv * n, 2, (long long)lv * n, lv, 0);
    SECPE_CHECK(ntt_limbset(ctx, zls, false));
    SECPE_CHECK(launch_rescale_fin(ctx, in, z.u(), out, lv));
    if (add_k) SECPE_CHECK(launch_addconst(ctx, out, out, lv, std::vector<long long>(1, *add_k)));
    return SECPE_OK;
}
