// Host launchers of the building-block kernels (kernels.cu).
#pragma once
#include <vector>

#include "internal.h"

#define SECPE_MAX_BATCH_CONST 1024

// digit layout of one key switch at a given level
struct KsDigits {
    int ndig;
    int lo[16], hi[16], off[16];  // prime range of digit j, offset of its targets in ext
};
struct KeyArr {
    u64 k[SECPE_MAX_BATCH_CONST];
};
struct PrimeList {
    int n;
    int p[SECPE_MAX_PRIMES];
};

int launch_addsub(secpe_ctx *ctx, const CtB &a, const CtB &b, const CtB &o, int nl, bool sub, int npoly = 2);
int launch_tensor(secpe_ctx *ctx, const CtB &a, const CtB &b, u64 *d, int nl);
// d = a (x) b + c (x) e in one pass (3-component output, limbs 0..nl-1)
int launch_tensor2(secpe_ctx *ctx, const CtB &a, const CtB &b, const CtB &c, const CtB &e, u64 *d, int nl);
// Item q of dst (limbs 0..nl-1 of both polynomials) = the sum of the
// ciphertexts src[qoff[q] .. qoff[q+1]) (each [2][cap[p]][N]); queries are
// launched in chunks that fit one pointer table.
int launch_sum_cts(secpe_ctx *ctx, const std::vector<const u64 *> &src, const std::vector<int> &cap,
                   const std::vector<int> &qoff, const CtB &dst, int nl);
// o = sum_t xs[t] * ks[t] (one constant per term, or one per item) over
// limbs 0..nl-1 of both polynomials, nt in {1, 2}.
int launch_lincomb(secpe_ctx *ctx, const CtB *xs, const std::vector<long long> *ks, int nt, const CtB &o, int nl);
int launch_addconst(secpe_ctx *ctx, const CtB &x, const CtB &o, int nl, const std::vector<long long> &k);
int launch_automorph(secpe_ctx *ctx, const CtB &x, const CtB &o, int nl, unsigned g);
// the automorphism on nlimbs contiguous limbs [nlimbs][N] (NTT form)
int launch_automorph_flat(secpe_ctx *ctx, const u64 *x, u64 *o, long long nlimbs, unsigned g);
int launch_rescale_prep(secpe_ctx *ctx, const u64 *y, u64 *z, int B, int lv);
int launch_rescale_fin(secpe_ctx *ctx, const CtB &x, const u64 *z, const CtB &o, int lv);
int launch_modup_bconv(secpe_ctx *ctx, const u64 *x, u64 *ext, long long ext_item_stride, int ext_off,
                       int B, int lv, int j, int lo, int hi, int ntgt);
// gal != 0: ext is read through the automorphism X -> X^gal (not with the
// precision variant)
int launch_ksk_ip(secpe_ctx *ctx, const u64 *d, long long d_item_stride, const u64 *ext,
                  long long ext_item_stride, const KsDigits &dg, const u64 *key, u64 *acc, int B, int lv,
                  unsigned gal = 0);
// The same inner product as exact 8-bit-limb contractions on the tensor
// pipe (precision variant, ntt_tc.cu; N = 2^16, at most 8 digits).
int launch_ksk_ip_tc(secpe_ctx *ctx, const u64 *d, long long d_item_stride, const u64 *ext,
                     long long ext_item_stride, const KsDigits &dg, const u64 *key, u64 *acc, int B, int lv);
int launch_moddown_bconv(secpe_ctx *ctx, const u64 *acc, u64 *conv, int B, int lv);
int launch_moddown_fin(secpe_ctx *ctx, const u64 *acc, const u64 *conv, const CtB &o, int lv, bool acc0,
                       bool acc1);
int launch_sample_uniform(secpe_ctx *ctx, const std::vector<u64> &keys, u64 *out, long long item_stride,
                          const PrimeList &pl);
int launch_sample_small(secpe_ctx *ctx, const std::vector<u64> &keys, long long *out, int kind);
int launch_signed_to_limbs(secpe_ctx *ctx, const long long *m, const long long *e, u64 *out,
                           long long item_stride, int B, const PrimeList &pl);
int launch_enc_finish(secpe_ctx *ctx, const u64 *M, long long ms, const u64 *a, long long as, const u64 *s,
                      const CtB &o, int nl);
int launch_dec_dot(secpe_ctx *ctx, const CtB &x, const u64 *s, u64 *m, int nl);
int launch_crt_double(secpe_ctx *ctx, const u64 *m, int lv, double *out);
int launch_crt_lift(secpe_ctx *ctx, const u64 *m, int lv, const long long *e, u64 *out,
                    long long out_item_stride, int ntop, int B);
int launch_ksk_gen(secpe_ctx *ctx, const u64 *a, const u64 *e_ntt, const u64 *s, const u64 *sp,
                   const u64 *pmod, u64 *key, int lo, int hi);
int launch_from_mont(secpe_ctx *ctx, const u64 *in, u64 *out, int nlimb_total);
int launch_limb_mul(secpe_ctx *ctx, const u64 *a, const u64 *b, u64 *o);
int launch_limb_automorph(secpe_ctx *ctx, const u64 *in, u64 *o, unsigned g);
// Integer multiply throughput probe: `blocks` CTAs of 256 threads, 4
// independent 128-bit multiply-accumulate chains per thread, `iters` rounds.
int launch_mul32_probe(secpe_ctx *ctx, unsigned blocks, int iters, u64 *sink);
int launch_mdr_prep(secpe_ctx *ctx, const u64 *d, long long dis, long long dps, u64 *acc, int B, int lv);
int launch_mdr_bconv(secpe_ctx *ctx, const u64 *acc, u64 *conv, int B, int lv);
int launch_mdr_fin(secpe_ctx *ctx, const u64 *acc, const u64 *conv, const u64 *d, long long dis, long long dps,
                   const CtB &o, int lv);
