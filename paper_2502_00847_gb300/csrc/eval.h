// Batched homomorphic evaluator (internal).
#pragma once
#include <memory>
#include <vector>

#include "internal.h"
#include "kernels.h"
#include "launch.h"

// Stream-ordered device buffer (cudaMallocAsync / cudaFreeAsync on the
// stream of the call in progress).
struct DevBuf {
    secpe_ctx *ctx = nullptr;
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    int alloc(secpe_ctx *c, size_t b) {
        ctx = c;
        bytes = b;
        if (b == 0) return SECPE_OK;
        if (cudaMallocAsync(&p, b, c->stream) != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return SECPE_ENOMEM;
        }
        return SECPE_OK;
    }
    void release() {
        if (p) cudaFreeAsync(p, ctx->stream);
        p = nullptr;
    }
    ~DevBuf() { release(); }
    u64 *u() const { return (u64 *)p; }
};

// A batch ciphertext value: a CtB view plus (optionally) the buffer owning it.
struct Ct {
    std::shared_ptr<DevBuf> buf;
    CtB v;
    int level() const { return v.level; }
    double scale() const { return v.scale; }
    int B() const { return v.B; }
};

// allocate a compact batch [B][2][level+1][N]
int ct_alloc(secpe_ctx *ctx, int B, int level, double scale, Ct &out);
// view of items [s, e) of a batch
Ct ct_slice(const Ct &x, int s, int e);
// same data, lower level (modulus drop)
Ct ct_drop(const Ct &x, int level);

// Level plan of one Argmax (level-aware QuickMax; the paper does not
// discuss levels).  Alg. 1 with r QuickMax rounds, evaluated greedily
// (refresh before a step that lacks its levels), falls into ranges: the
// first starts at y after the duplication, each refresh starts the next.
// Range by range, the plan starts each range as low as it can while every
// refresh stays at the same step (and the refreshed step keeps its levels),
// so the refresh count is unchanged and the steps run on fewer limbs.
struct LevelPlan {
    std::vector<int> target;  // [0]: level of y entering round 0; [j]: level after refresh j
    std::vector<int> lv;      // planned level of y when phase k = 0..r starts (k = r: the final Sign)
    std::vector<int> nref;    // refreshes before phase k, k = 0..r+1
    // what two queries must share to run phase k as one batch
    std::vector<int> signature(int k) const;
};
int make_level_plan(const secpe_ctx *ctx, int r, int entry, LevelPlan &plan);
// the same from the reserve, the polynomials per Sign and the refresh's output level
int make_level_plan(int res, int n_poly, int top, int r, int entry, LevelPlan &plan);
int refresh_out_level(const secpe_ctx *ctx);

struct Eval {
    secpe_ctx *ctx;
    const secpe_keys *keys;
    std::vector<u64> qseeds;  // per item, refresh randomness
    u64 ridx = 0;             // refresh counter (shared by the batch)
    const LevelPlan *plan = nullptr;  // set inside an Argmax: drops after each refresh

    int add(const Ct &a, const Ct &b, Ct &out);
    int sub(const Ct &a, const Ct &b, Ct &out);
    int mul(const Ct &a, const Ct &b, Ct &out);
    // 3-component ciphertexts (stride 3 (level+1) N, scale tracked)
    int tensor(const Ct &a, const Ct &b, Ct &out3);
    // a (x) b + c (x) e as one 3-component ciphertext (equal to add3 of the two tensors)
    int tensor2(const Ct &a, const Ct &b, const Ct &c, const Ct &e, Ct &out3);
    int add3(const Ct &a3, const Ct &b3, Ct &out3);
    int relin_rescale(const Ct &d3, Ct &out);
    int mul_const(const Ct &x, const std::vector<double> &c, double target, int out_level, Ct &out);
    // add_c: optional constant added to the result (as add_const, in the rescale's last pass)
    int lincomb(const std::vector<const Ct *> &xs, const std::vector<std::vector<double>> &cs, double target,
                int out_level, Ct &out, const double *add_c = nullptr);
    int add_const(const Ct &x, double c, Ct &out);
    int rescale(const Ct &in, Ct &out, const long long *add_k = nullptr);
    int rotate(const Ct &x, int steps, Ct &out);
    // rotations of x by every step, sharing one ModUp (bootstrapping's baby steps)
    int rotate_hoisted(const Ct &x, const std::vector<int> &steps, std::vector<Ct> &outs);
    int refresh(const Ct &x, Ct &out);
    int ensure(const Ct &x, int k, Ct &out);
    int poly9(const Ct &x, const double *c, double s_out, Ct &out);
    int sign(const Ct &x, int out_levels, Ct &out, double last_factor = 1.0, bool lowest = false);
    int max(const Ct &a, const Ct &y, Ct &out);
    int argmax(const Ct &y, int C, Ct &out);
    // the Phoenix Argmax baseline (m + 1 Signs, m + 1 rotations, m = C' - 1)
    int phoenix(const Ct &y, int C, Ct &out);
};

// Per-slot plaintext products (linear.cu): o (+)= x (.) p with p in
// Montgomery NTT form (item stride ps, 0 = one plaintext for all items; x
// item stride xs, 0 = one input for all items); o = x + (p, 0).
int launch_mul_plain(secpe_ctx *ctx, const CtB &x, long long xs, const u64 *p, long long ps, const CtB &o, int nl,
                     bool acc = false);
int launch_add_plain(secpe_ctx *ctx, const CtB &x, const u64 *p, const CtB &o, int nl);
// o (+)= sum_t xs[t] (.) ps[t] (Montgomery-form plaintexts [nl][N], one for
// every item; at most kMaxPlainTerms terms), one pass
constexpr int kMaxPlainTerms = 32;
int launch_mul_plain_sum(secpe_ctx *ctx, const std::vector<CtB> &xs, const std::vector<const u64 *> &ps,
                         const CtB &o, int nl, bool acc);
// os[g] = sum_k xs[k] (.) ps[k][g] for up to kMaxGiant outputs in one pass
// (every xs[k] read once; all outputs with one layout)
constexpr int kMaxGiant = 2;
int launch_bsgs_inner(secpe_ctx *ctx, const std::vector<CtB> &xs, const std::vector<std::vector<const u64 *>> &ps,
                      const std::vector<CtB> &os, int nl);
// B plaintexts from host int64 coefficients m[B][N]: NTT-form residues of
// limbs 0..nl-1 (Montgomery form if mont) at dst [B][nl][N]; synchronous.
int upload_plain(secpe_ctx *ctx, const int64_t *m, int B, int nl, bool mont, u64 *dst);

// Hybrid key switching (keyswitch.cu): d = limbs 0..lv of one polynomial per
// item (NTT form) at d + item*d_item_stride; writes (or adds, per poly) the
// result into polys 0 and 1 of `out` (B items, level lv).
// Bootstrapping of a batch (boot.cu): labels kept, output at level L - 16.
int boot_batch(secpe_ctx *ctx, const secpe_keys *keys, const secpe_boot *bt, const Ct &in, Ct &out);
int boot_block(const secpe_boot *bt);
int boot_out_level(const secpe_ctx *ctx);

int keyswitch(secpe_ctx *ctx, const u64 *d, long long d_item_stride, int B, int lv, const u64 *key,
              const CtB &out, bool acc0, bool acc1);
// ModUp + key inner product only: acc [B][2][lv+1+k][N] (allocated here).
int keyswitch_acc(secpe_ctx *ctx, const u64 *d, long long d_item_stride, int B, int lv, const u64 *key, DevBuf &acc);
// Relinearise the 3-component tensor d [B][3][lv+1][N] and rescale: out at lv-1.
int relin_rescale_batch(secpe_ctx *ctx, const u64 *d, int B, int lv, const u64 *key, const CtB &out);
int rescale_batch(secpe_ctx *ctx, const CtB &in, const CtB &out, const long long *add_k = nullptr);
// Rotations of x by every Galois element gal[i] with keys[i] into outs[i]
// (B items, level of x), sharing one ModUp of x's second polynomial.
int rotate_hoisted(secpe_ctx *ctx, const CtB &x, const std::vector<unsigned> &gal, const std::vector<const u64 *> &keys,
                   const std::vector<CtB> &outs);
unsigned galois_elt(const secpe_ctx *ctx, int steps);
const u64 *galois_key(const secpe_keys *keys, unsigned g);
int sign_coeffs(double g[5], double f[5]);

// fused N = 2^16 paths (ntt_fused.cu)
bool fused_path(const secpe_ctx *ctx);
int modup_ip_fused(secpe_ctx *ctx, const u64 *d, long long d_item_stride, const u64 *dcoef, int B, int lv,
                   const KsDigits &dg, int tot, const u64 *key, u64 *ext, u64 *acc);
int moddown_fused(secpe_ctx *ctx, const u64 *acc, int B, int lv, const CtB &out, bool acc0, bool acc1, u64 *tmp);
int moddown_rescale_fused(secpe_ctx *ctx, u64 *acc, const u64 *d, int B, int lv, const CtB &out, u64 *tmp);
// add_k: optional constant k added to polynomial 0 of the result (a constant polynomial, as add_const)
int rescale_fused(secpe_ctx *ctx, const CtB &in, const u64 *y, const CtB &out, u64 *tmp,
                  const long long *add_k = nullptr);
