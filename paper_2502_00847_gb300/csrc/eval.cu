// Batched evaluator: every operation acts on B ciphertexts at once (same
// level and scale), so one launch per kernel serves the whole batch.  The
// circuit follows SecPE Sec. 3.2 / Alg. 1 with the readings stated in the
// header: Sign = f^df(g^dg) by a fixed depth-4 baby-step giant-step DAG per
// polynomial, Max by Eq. max, QuickMax over rotations by 2^i, refresh when a
// polynomial block would run out of levels.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>

#include "eval.h"

int ct_alloc(secpe_ctx *ctx, int B, int level, double scale, Ct &out) {
    out.buf = std::make_shared<DevBuf>();
    SECPE_CHECK(out.buf->alloc(ctx, sizeof(u64) * (size_t)B * 2 * (level + 1) * ctx->n));
    out.v.data = out.buf->u();
    out.v.B = B;
    out.v.cap = level + 1;
    out.v.stride = 2ll * (level + 1) * ctx->n;
    out.v.level = level;
    out.v.scale = scale;
    out.v.n = ctx->n;
    return SECPE_OK;
}

Ct ct_slice(const Ct &x, int s, int e) {
    Ct r = x;
    r.v.data = x.v.data + (long long)s * x.v.stride;
    r.v.B = e - s;
    return r;
}

Ct ct_drop(const Ct &x, int level) {
    Ct r = x;
    r.v.level = level;
    return r;
}

unsigned galois_elt(const secpe_ctx *ctx, int steps) {
    if (steps == SECPE_STEP_CONJ) return 2u * ctx->n - 1u;
    const int half = ctx->n / 2;
    long long r = steps;
    if (r < 0) r = half + r;
    r %= half;
    if (r < 0) r += half;
    unsigned long long g = 1, b = 5, m = 2ull * ctx->n;
    while (r) {
        if (r & 1) g = g * b % m;
        b = b * b % m;
        r >>= 1;
    }
    return (unsigned)g;
}

const u64 *galois_key(const secpe_keys *keys, unsigned g) {
    auto it = keys->gks.find(g);
    return it == keys->gks.end() ? nullptr : it->second;
}

// f_4 and g_4 of Cheon, Kim, Kim, Lee, Lee (Asiacrypt 2020), odd powers 1..9.
int sign_coeffs(double g[5], double f[5]) {
    static const double G[5] = {5850.0 / 1024, -34974.0 / 1024, 97015.0 / 1024, -113492.0 / 1024,
                                46623.0 / 1024};
    static const double F[5] = {315.0 / 128, -420.0 / 128, 378.0 / 128, -180.0 / 128, 35.0 / 128};
    for (int i = 0; i < 5; i++) {
        g[i] = G[i];
        f[i] = F[i];
    }
    return SECPE_OK;
}

static bool scales_match(double a, double b) { return std::fabs(a - b) <= a * std::ldexp(1.0, -40); }

int Eval::add(const Ct &a, const Ct &b, Ct &out) {
    if (a.B() != b.B()) return SECPE_EINVAL;
    if (!scales_match(a.scale(), b.scale())) return SECPE_ESCALE;
    const int lv = std::min(a.level(), b.level());
    Ct o;
    SECPE_CHECK(ct_alloc(ctx, a.B(), lv, a.scale(), o));
    SECPE_CHECK(launch_addsub(ctx, a.v, b.v, o.v, lv + 1, false));
    out = o;
    return SECPE_OK;
}

int Eval::sub(const Ct &a, const Ct &b, Ct &out) {
    if (a.B() != b.B()) return SECPE_EINVAL;
    if (!scales_match(a.scale(), b.scale())) return SECPE_ESCALE;
    const int lv = std::min(a.level(), b.level());
    Ct o;
    SECPE_CHECK(ct_alloc(ctx, a.B(), lv, a.scale(), o));
    SECPE_CHECK(launch_addsub(ctx, a.v, b.v, o.v, lv + 1, true));
    out = o;
    return SECPE_OK;
}

int Eval::rescale(const Ct &in, Ct &out, const long long *add_k) {
    const int lv = in.level();
    if (lv < 1) return SECPE_ELEVEL;
    Ct o;
    SECPE_CHECK(ct_alloc(ctx, in.B(), lv - 1, in.scale() / (double)ctx->primes[lv], o));
    SECPE_CHECK(rescale_batch(ctx, in.v, o.v, add_k));
    out = o;
    return SECPE_OK;
}

int Eval::tensor(const Ct &a, const Ct &b, Ct &out3) {
    if (a.B() != b.B()) return SECPE_EINVAL;
    const int lv = std::min(a.level(), b.level());
    const int B = a.B(), n = ctx->n;
    Ct d;
    d.buf = std::make_shared<DevBuf>();
    SECPE_CHECK(d.buf->alloc(ctx, sizeof(u64) * (size_t)B * 3 * (lv + 1) * n));
    SECPE_CHECK(launch_tensor(ctx, a.v, b.v, d.buf->u(), lv + 1));
    d.v.data = d.buf->u();
    d.v.B = B;
    d.v.cap = lv + 1;
    d.v.stride = 3ll * (lv + 1) * n;
    d.v.level = lv;
    d.v.scale = a.scale() * b.scale();
    d.v.n = n;
    out3 = d;
    return SECPE_OK;
}

int Eval::tensor2(const Ct &a, const Ct &b, const Ct &c, const Ct &e, Ct &out3) {
    if (a.B() != b.B() || a.B() != c.B() || a.B() != e.B()) return SECPE_EINVAL;
    if (!scales_match(a.scale() * b.scale(), c.scale() * e.scale())) return SECPE_ESCALE;
    const int lv = std::min(std::min(a.level(), b.level()), std::min(c.level(), e.level()));
    const int B = a.B(), n = ctx->n;
    Ct d;
    d.buf = std::make_shared<DevBuf>();
    SECPE_CHECK(d.buf->alloc(ctx, sizeof(u64) * (size_t)B * 3 * (lv + 1) * n));
    SECPE_CHECK(launch_tensor2(ctx, a.v, b.v, c.v, e.v, d.buf->u(), lv + 1));
    d.v.data = d.buf->u();
    d.v.B = B;
    d.v.cap = lv + 1;
    d.v.stride = 3ll * (lv + 1) * n;
    d.v.level = lv;
    d.v.scale = a.scale() * b.scale();
    d.v.n = n;
    out3 = d;
    return SECPE_OK;
}

int Eval::add3(const Ct &a3, const Ct &b3, Ct &out3) {
    if (a3.B() != b3.B() || a3.level() != b3.level()) return SECPE_EINVAL;
    if (!scales_match(a3.scale(), b3.scale())) return SECPE_ESCALE;
    const int lv = a3.level(), B = a3.B(), n = ctx->n;
    Ct o;
    o.buf = std::make_shared<DevBuf>();
    SECPE_CHECK(o.buf->alloc(ctx, sizeof(u64) * (size_t)B * 3 * (lv + 1) * n));
    o.v = a3.v;
    o.v.data = o.buf->u();
    o.v.cap = lv + 1;
    o.v.stride = 3ll * (lv + 1) * n;
    SECPE_CHECK(launch_addsub(ctx, a3.v, b3.v, o.v, lv + 1, false, 3));
    out3 = o;
    return SECPE_OK;
}

int Eval::relin_rescale(const Ct &d3, Ct &out) {
    const int lv = d3.level();
    if (lv < 1 + ctx->p.reserve) return SECPE_ELEVEL;
    if (!keys || !keys->rlk) return SECPE_EKEY;
    if (d3.v.cap != lv + 1 || d3.v.stride != 3ll * (lv + 1) * ctx->n) return SECPE_EINVAL;
    Ct o;
    SECPE_CHECK(ct_alloc(ctx, d3.B(), lv - 1, d3.scale() / (double)ctx->primes[lv], o));
    ctx->counters.relins += d3.B();
    SECPE_CHECK(relin_rescale_batch(ctx, d3.v.data, d3.B(), lv, keys->rlk, o.v));
    out = o;
    return SECPE_OK;
}

int Eval::mul(const Ct &a, const Ct &b, Ct &out) {
    if (a.B() != b.B()) return SECPE_EINVAL;
    const int lv = std::min(a.level(), b.level());
    if (lv < 1 + ctx->p.reserve) return SECPE_ELEVEL;
    if (!keys || !keys->rlk) return SECPE_EKEY;
    Ct d;
    SECPE_CHECK(tensor(a, b, d));
    return relin_rescale(d, out);
}

int Eval::mul_const(const Ct &x, const std::vector<double> &c, double target, int out_level, Ct &out) {
    return lincomb({&x}, {c}, target, out_level, out);
}

// sum_t c_t x_t at out_level with scale exactly `target`: every x_t dropped
// to out_level + 1 and multiplied by k_t = round(c_t target / s_t q),
// q = q_{out_level+1}; the products are added and the sum rescaled once.
int Eval::lincomb(const std::vector<const Ct *> &xs, const std::vector<std::vector<double>> &cs, double target,
                  int out_level, Ct &out, const double *add_c) {
    const int nt = (int)xs.size();
    if (nt < 1 || nt > 2 || (int)cs.size() != nt) return SECPE_EINVAL;
    if (out_level < ctx->p.reserve || out_level < 0 || out_level + 1 > ctx->L) return SECPE_ELEVEL;
    const int B = xs[0]->B();
    const double qf = (double)ctx->primes[out_level + 1];
    CtB v[2];
    std::vector<long long> k[2];
    for (int t = 0; t < nt; t++) {
        const Ct &x = *xs[t];
        if (x.level() < out_level + 1) return SECPE_ELEVEL;
        if (x.B() != B || (cs[t].size() != 1 && (int)cs[t].size() != B)) return SECPE_EINVAL;
        const Ct xd = ct_drop(x, out_level + 1);
        const double factor = target / xd.scale() * qf;
        for (double c : cs[t]) {
            const double kv = c * factor;
            if (!(std::fabs(kv) < 4.0e18)) return SECPE_EINVAL;
            k[t].push_back(hm::round_half_away(kv));
        }
        v[t] = xd.v;
    }
    Ct tsum;
    SECPE_CHECK(ct_alloc(ctx, B, out_level + 1, target * qf, tsum));
    SECPE_CHECK(launch_lincomb(ctx, v, k, nt, tsum.v, out_level + 2));
    long long ka = 0;
    if (add_c) {
        // add_const's constant at the result's scale (target)
        const double va = *add_c * target;
        if (!(std::fabs(va) < 4.0e18)) return SECPE_EINVAL;
        ka = hm::round_half_away(va);
    }
    SECPE_CHECK(rescale(tsum, out, add_c ? &ka : nullptr));
    out.v.scale = target;
    return SECPE_OK;
}

int Eval::add_const(const Ct &x, double c, Ct &out) {
    const double v = c * x.scale();
    if (!(std::fabs(v) < 4.0e18)) return SECPE_EINVAL;
    std::vector<long long> k(1, hm::round_half_away(v));
    Ct o;
    SECPE_CHECK(ct_alloc(ctx, x.B(), x.level(), x.scale(), o));
    SECPE_CHECK(launch_addconst(ctx, x.v, o.v, x.level() + 1, k));
    out = o;
    return SECPE_OK;
}

int Eval::rotate(const Ct &x, int steps, Ct &out) {
    const unsigned g = galois_elt(ctx, steps);
    const u64 *key = keys ? galois_key(keys, g) : nullptr;
    if (!key) return SECPE_EKEY;
    const int lv = x.level();
    Ct o;
    SECPE_CHECK(ct_alloc(ctx, x.B(), lv, x.scale(), o));
    SECPE_CHECK(launch_automorph(ctx, x.v, o.v, lv + 1, g));
    ctx->counters.rotations += x.B();
    SECPE_CHECK(keyswitch(ctx, o.v.data + o.v.pstride(), o.v.stride, x.B(), lv, key, o.v, true, false));
    out = o;
    return SECPE_OK;
}

int Eval::rotate_hoisted(const Ct &x, const std::vector<int> &steps, std::vector<Ct> &outs) {
    std::vector<unsigned> gal;
    std::vector<const u64 *> ks;
    std::vector<CtB> ov;
    outs.clear();
    for (int st : steps) {
        const unsigned g = galois_elt(ctx, st);
        const u64 *key = keys ? galois_key(keys, g) : nullptr;
        if (!key) return SECPE_EKEY;
        gal.push_back(g);
        ks.push_back(key);
    }
    for (size_t i = 0; i < steps.size(); i++) {
        Ct o;
        SECPE_CHECK(ct_alloc(ctx, x.B(), x.level(), x.scale(), o));
        ov.push_back(o.v);
        outs.push_back(o);
    }
    SECPE_CHECK(::rotate_hoisted(ctx, x.v, gal, ks, ov));
    ctx->counters.rotations += (unsigned long long)x.B() * steps.size();
    return SECPE_OK;
}

int Eval::refresh(const Ct &x, Ct &out) {
    if (ctx->boot) {
        // non-interactive: a bootstrap of the batch replaces the stand-in
        Ct o;
        SECPE_CHECK(boot_batch(ctx, keys, ctx->boot, x, o));
        ctx->counters.refreshes += x.B();
        ctx->counters.bootstraps += x.B();
        ridx++;
        out = o;
        return SECPE_OK;
    }
    if (!keys || !keys->s_ntt) return SECPE_EKEY;
    const int B = x.B(), lv = x.level(), n = ctx->n, L = ctx->L;
    if ((int)qseeds.size() != B || B > SECPE_MAX_BATCH_CONST) return SECPE_EINVAL;
    // the whole stand-in is one profiler range, so its share of a step can be measured
    KprofScope kp(ctx, "refresh", 0.0);
    DevBuf m, e, M, a;
    SECPE_CHECK(m.alloc(ctx, sizeof(u64) * (size_t)B * (lv + 1) * n));
    SECPE_CHECK(launch_dec_dot(ctx, x.v, keys->s_ntt, m.u(), lv + 1));
    LimbSet mls = make_limbset(m.u(), B, (long long)(lv + 1) * n, 1, 0, lv + 1, 0);
    SECPE_CHECK(ntt_limbset(ctx, mls, true));
    std::vector<u64> ke(B), ka(B);
    for (int b = 0; b < B; b++) {
        const u64 sd = hm::sm_stream(qseeds[b], DOM_REFRESH, ridx);
        ke[b] = hm::sm_stream(sd, DOM_ENC_E, 0);
        ka[b] = hm::sm_stream(sd, DOM_ENC_A, 0);
    }
    ridx++;
    SECPE_CHECK(e.alloc(ctx, sizeof(long long) * (size_t)B * n));
    SECPE_CHECK(launch_sample_small(ctx, ke, (long long *)e.p, 1));
    SECPE_CHECK(M.alloc(ctx, sizeof(u64) * (size_t)B * (L + 1) * n));
    SECPE_CHECK(launch_crt_lift(ctx, m.u(), lv, (const long long *)e.p, M.u(), (long long)(L + 1) * n, L + 1, B));
    LimbSet Mls = make_limbset(M.u(), B, (long long)(L + 1) * n, 1, 0, L + 1, 0);
    SECPE_CHECK(ntt_limbset(ctx, Mls, false));
    SECPE_CHECK(a.alloc(ctx, sizeof(u64) * (size_t)B * (L + 1) * n));
    PrimeList pl;
    pl.n = L + 1;
    for (int i = 0; i <= L; i++) pl.p[i] = i;
    SECPE_CHECK(launch_sample_uniform(ctx, ka, a.u(), (long long)(L + 1) * n, pl));
    Ct o;
    SECPE_CHECK(ct_alloc(ctx, B, L, x.scale(), o));
    SECPE_CHECK(launch_enc_finish(ctx, M.u(), (long long)(L + 1) * n, a.u(), (long long)(L + 1) * n, keys->s_ntt,
                                  o.v, L + 1));
    ctx->counters.refreshes += B;
    out = o;
    return SECPE_OK;
}

int Eval::ensure(const Ct &x, int k, Ct &out) {
    if (x.level() >= k + ctx->p.reserve) {
        out = x;
        return SECPE_OK;
    }
    SECPE_CHECK(refresh(x, out));
    // inside an Argmax: down to the plan's level for the range this refresh starts
    if (plan && ridx < plan->target.size() && out.level() > plan->target[ridx])
        out = ct_drop(out, plan->target[ridx]);
    return SECPE_OK;
}

int refresh_out_level(const secpe_ctx *ctx) { return ctx->boot ? boot_out_level(ctx) : ctx->L; }

namespace {

// The level tests of Alg. 1 on y at `entry` (r QuickMax rounds, then the
// final Sign at its lowest levels), step for step as Eval::argmax takes
// them, with each range starting at most at plan[j] (a refresh returns
// min(top, plan[j]) after refresh j).  Fills the indices of the tests that
// refresh; false if a refreshed step lacks its levels.  With lv and nref it
// also records y's level and the refresh count when each phase starts.
struct LevelWalk {
    int res, top, n_poly, r, entry;

    bool run(const std::vector<int> &plan, std::vector<int> &points, std::vector<int> *lv = nullptr,
             std::vector<int> *nref = nullptr) const {
        points.clear();
        int count = 0;
        bool ok = true;
        auto test = [&](int l, int k) {
            count++;
            if (l >= k + res) return l;
            points.push_back(count);
            const size_t j = points.size();
            const int out = j < plan.size() ? std::min(top, plan[j]) : top;
            ok = ok && out >= k + res;
            return out;
        };
        auto mark = [&](int l) {
            if (!lv) return;
            lv->push_back(l);
            nref->push_back((int)points.size());
        };
        int l = std::min(entry, plan[0]);
        for (int k = 0; k < r; k++) {  // QuickMax rounds
            mark(l);
            l = test(l, 1);
            const int ld = l;  // d = a - y stays at this level
            for (int i = 0; i < n_poly; i++) l = test(l, i == n_poly - 1 ? 5 : 4) - 4;
            l = std::min(ld, l) - 1;  // t = d * Sign(d)/2; Max at t's level
        }
        mark(l);
        for (int i = 0; i < n_poly; i++) l = std::min(test(l, 4), 4 * (n_poly - i) + res) - 4;
        if (nref) nref->push_back((int)points.size());
        return ok;
    }
};

}  // namespace

int make_level_plan(const secpe_ctx *ctx, int r, int entry, LevelPlan &plan) {
    return make_level_plan(ctx->p.reserve, ctx->p.sign_dg + ctx->p.sign_df, refresh_out_level(ctx), r, entry, plan);
}

// Range by range, in order, the lowest start that keeps every refresh at
// the same test and every refreshed step its levels.  A lower start never
// raises a later level, so those starts form an interval: lower one level
// at a time.  The whole circuit is walked for every trial, because a
// range's ciphertexts reach later ranges (Max multiplies d, computed before
// a refresh inside Sign(d), by the refreshed Sign).
int make_level_plan(int res, int np, int top, int r, int entry, LevelPlan &plan) {
    const LevelWalk w{res, top, np, r, entry};
    std::vector<int> points, trial_points;
    if (!w.run({entry}, points)) return SECPE_ELEVEL;
    plan.target.assign(points.size() + 1, top);
    plan.target[0] = entry;
    for (size_t j = 0; j < plan.target.size(); j++) {
        while (plan.target[j] > 0) {
            std::vector<int> trial = plan.target;
            trial[j]--;
            if (!w.run(trial, trial_points) || trial_points != points) break;
            plan.target[j]--;
        }
    }
    plan.lv.clear();
    plan.nref.clear();
    w.run(plan.target, trial_points, &plan.lv, &plan.nref);
    return SECPE_OK;
}

std::vector<int> LevelPlan::signature(int k) const {
    std::vector<int> s{lv[k], nref[k]};
    for (int j = nref[k] + 1; j <= nref[k + 1]; j++) s.push_back(target[j]);
    return s;
}

// Odd degree-9 p(x) = c1 x + c3 x^3 + c5 x^5 + c7 x^7 + c9 x^9 (Eq. comp),
// baby steps in y = x^2 and giant step x^4 (BSGS):
//   p = x (c1 + c3 y) + x^5 (c5 + c7 y + c9 y^2),
// at depth 4: x2 = x*x, x4 = x2*x2, x5 = x4*x; P1 = c7 x2 + c9 x4 + c5 and
// P0 = c3 x2 + c1 (one rescale each); the 3-component products x5 (x) P1
// and x (x) P0 are added and relinearised once (4 key switches per
// polynomial).  P1 lands at the scale that gives p the scale s_out, P0 at
// the scale that makes the two products' scales equal.
int Eval::poly9(const Ct &x, const double *c, double s_out, Ct &out) {
    const int lv = x.level();
    if (lv < 4 + ctx->p.reserve) return SECPE_ELEVEL;
    const double q3 = (double)ctx->primes[lv - 3];
    // temporaries are released as soon as they are dead (Ct() frees them)
    Ct x2, x4, x5, P1, P0, TU3;
    SECPE_CHECK(mul(x, x, x2));
    SECPE_CHECK(mul(x2, x2, x4));
    SECPE_CHECK(mul(x4, x, x5));
    const double s1 = s_out * q3 / x5.scale();
    // P1 = c7 x2 + c9 x4 + c5 and P0 = c3 x2 + c1, each constant added in the
    // rescale's last pass (the same residues as a separate add_const)
    SECPE_CHECK(lincomb({&x2, &x4}, {{c[3]}, {c[4]}}, s1, lv - 3, P1, &c[2]));
    x4 = Ct();
    const double s0 = x5.scale() * s1 / x.scale();
    SECPE_CHECK(lincomb({&x2}, {{c[1]}}, s0, lv - 3, P0, &c[0]));
    x2 = Ct();
    SECPE_CHECK(tensor2(x5, P1, x, P0, TU3));
    x5 = Ct();
    P1 = Ct();
    P0 = Ct();
    return relin_rescale(TU3, out);
}

// The last polynomial's coefficients are multiplied by last_factor, so the
// result is last_factor * Sign(x) at no extra level.  With `lowest` (the
// final Sign of Alg. 1, which nothing follows), the input of every
// polynomial is dropped to the levels the rest of the Sign needs,
// 4 (polynomials left) + out_levels + reserve, so that a polynomial after a
// refresh runs on as few limbs as possible; the refresh count is unchanged.
int Eval::sign(const Ct &x, int out_levels, Ct &out, double last_factor, bool lowest) {
    double g[5], f[5];
    sign_coeffs(g, f);
    ctx->counters.signs += x.B();
    const int np = ctx->p.sign_dg + ctx->p.sign_df;
    Ct cur = x;
    for (int i = 0; i < np; i++) {
        const bool last = i == np - 1;
        const int need = 4 + (last ? out_levels : 0);
        double c[5];
        for (int k = 0; k < 5; k++) c[k] = (i < ctx->p.sign_dg ? g[k] : f[k]) * (last ? last_factor : 1.0);
        Ct e, p;
        SECPE_CHECK(ensure(cur, need, e));
        const int keep = 4 * (np - i) + out_levels + ctx->p.reserve;
        if (lowest && e.level() > keep) e = ct_drop(e, keep);
        SECPE_CHECK(poly9(e, c, ctx->scale, p));
        cur = p;
    }
    out = cur;
    return SECPE_OK;
}

// Max(a, y) = (a+y)/2 + d * (Sign(d)/2), d = a - y: the 1/2 of the second
// term is folded into Sign's last polynomial, so t = d * (Sign(d)/2) keeps
// d's scale; (a+y) * 1/2 is brought to t's level and scale.
int Eval::max(const Ct &a, const Ct &y, Ct &out) {
    Ct d, s, t, apy, u;
    SECPE_CHECK(sub(a, y, d));
    SECPE_CHECK(sign(d, 1, s, 0.5));
    SECPE_CHECK(mul(d, s, t));
    SECPE_CHECK(add(a, y, apy));
    SECPE_CHECK(mul_const(apy, {0.5}, t.scale(), t.level(), u));
    return add(t, u, out);
}

static int log2_ceil_pow(int C, int &cp) {
    cp = 1;
    int r = 0;
    while (cp < C) {
        cp <<= 1;
        r++;
    }
    return r;
}

int Eval::argmax(const Ct &y, int C, Ct &out) {
    if (C < 2 || C > ctx->n / 2) return SECPE_EINVAL;
    int cp;
    const int r = log2_ceil_pow(C, cp);
    if (2 * cp > ctx->n / 2) return SECPE_EINVAL;
    Ct rot, y1, ydup;
    SECPE_CHECK(rotate(y, -cp, rot));
    SECPE_CHECK(add(y, rot, y1));
    ydup = y1;
    LevelPlan lp;
    SECPE_CHECK(make_level_plan(ctx, r, y1.level(), lp));
    struct Reset {
        const LevelPlan *&p;
        ~Reset() { p = nullptr; }
    } reset{plan};
    plan = &lp;
    if (y1.level() > lp.target[0]) y1 = ct_drop(y1, lp.target[0]);
    for (int i = 0; i < r; i++) {
        Ct ye, a, m;
        SECPE_CHECK(ensure(y1, 1, ye));
        SECPE_CHECK(rotate(ye, 1 << i, a));
        SECPE_CHECK(max(a, ye, m));
        y1 = m;
    }
    Ct al, d, s;
    SECPE_CHECK(mul_const(ydup, {1.0}, y1.scale(), y1.level(), al));
    SECPE_CHECK(sub(al, y1, d));
    SECPE_CHECK(sign(d, 0, s, 1.0, true));
    return add_const(s, 1.0, out);
}

// The Phoenix Argmax that SecPE Sec. 3.2 compares against: after the same
// duplication, every slot is compared with its m = C' - 1 cyclic
// neighbours, s = sum_{i=1..m} Sign(y - RotL(y, i)); the max slot has
// s = m, every other s <= m - 2, so z = (Sign((s - (m - 1)) / (2m)) + 1) / 2
// (the 1/2 folded into the last polynomial): m + 1 Signs and m + 1
// rotations.  The m comparisons start from the same ciphertext, so they run
// as one batch of m * B items (in chunks that bound memory).  Comparison i
// of query b takes its refresh randomness from the seed
// stream(qseed_b, DOM_PHOENIX, i), the final Sign from stream(qseed_b,
// DOM_PHOENIX, 0), each counting refreshes from 0.
int Eval::phoenix(const Ct &y, int C, Ct &out) {
    if (C < 2 || C > ctx->n / 2) return SECPE_EINVAL;
    int cp;
    log2_ceil_pow(C, cp);
    if (2 * cp > ctx->n / 2) return SECPE_EINVAL;
    const int m = cp - 1, B = y.B();
    if ((int)qseeds.size() != B) return SECPE_EINVAL;
    Ct rot, ydup;
    SECPE_CHECK(rotate(y, -cp, rot));
    SECPE_CHECK(add(y, rot, ydup));
    rot = Ct();
    const int lv = ydup.level();
    const int chunk = std::max(1, std::min(SECPE_MAX_BATCH_CONST, 128) / B);
    Ct s;
    for (int i0 = 1; i0 <= m; i0 += chunk) {
        const int nm = std::min(m + 1, i0 + chunk) - i0;
        Ct D, S;
        SECPE_CHECK(ct_alloc(ctx, nm * B, lv, ydup.scale(), D));
        Eval Ec{ctx, keys, {}, 0};
        for (int i = i0; i < i0 + nm; i++) {
            Ct r;
            SECPE_CHECK(rotate(ydup, i, r));
            Ct dst = ct_slice(D, (i - i0) * B, (i - i0 + 1) * B);
            SECPE_CHECK(launch_addsub(ctx, ydup.v, r.v, dst.v, lv + 1, true));
            for (int b = 0; b < B; b++) Ec.qseeds.push_back(hm::sm_stream(qseeds[b], DOM_PHOENIX, (u64)i));
        }
        SECPE_CHECK(Ec.sign(D, 1, S));
        D = Ct();
        for (int i = 0; i < nm; i++) {
            Ct Si = ct_slice(S, i * B, (i + 1) * B);
            if (!s.buf) {
                s = Si;
            } else {
                Ct sum;
                SECPE_CHECK(add(s, Si, sum));
                s = sum;
            }
        }
    }
    Ct t0, t;
    SECPE_CHECK(add_const(s, -(m - 1.0), t0));
    s = Ct();
    SECPE_CHECK(mul_const(t0, {1.0 / (2.0 * m)}, ctx->scale, t0.level() - 1, t));
    t0 = Ct();
    Eval Ef{ctx, keys, {}, 0};
    for (int b = 0; b < B; b++) Ef.qseeds.push_back(hm::sm_stream(qseeds[b], DOM_PHOENIX, 0));
    Ct zs;
    SECPE_CHECK(Ef.sign(t, 0, zs, 0.5, true));
    return add_const(zs, 0.5, out);
}

// ---------------------------------------------------------------- batch
// Queries are ordered by r = log2 C' (descending) so that at phase k the
// queries still in QuickMax form a prefix of the batch and the queries that
// finish at phase k the following contiguous range.  All queries of one
// range share level, scale and refresh history, so each range is a single
// batched evaluation.
static int argmax_batch_tenant(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q, int nq_);
static int phoenix_batch_tenant(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q, int nq_);
typedef int (*tenant_fn)(secpe_ctx *, const secpe_keys *, const secpe_query *, int);

// Queries of different tenants are evaluated as one batch per key set.
static int per_tenant(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q, int nq_, tenant_fn fn) {
    std::vector<const secpe_keys *> sets;
    for (int b = 0; b < nq_; b++) {
        const secpe_keys *k = q[b].keys ? q[b].keys : keys;
        if (!k) return SECPE_EINVAL;
        if (std::find(sets.begin(), sets.end(), k) == sets.end()) sets.push_back(k);
    }
    if (sets.size() == 1) return fn(ctx, sets[0], q, nq_);
    for (const secpe_keys *k : sets) {
        std::vector<secpe_query> part;
        for (int b = 0; b < nq_; b++)
            if ((q[b].keys ? q[b].keys : keys) == k) part.push_back(q[b]);
        SECPE_CHECK(fn(ctx, k, part.data(), (int)part.size()));
    }
    return SECPE_OK;
}

int argmax_batch_impl(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q, int nq_) {
    return per_tenant(ctx, keys, q, nq_, argmax_batch_tenant);
}

int phoenix_batch_impl(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q, int nq_) {
    return per_tenant(ctx, keys, q, nq_, phoenix_batch_tenant);
}

// Checks the queries and orders them by r = log2 C' (descending, stable).
// Every input ciphertext of the call must be at one level, *lin (the top
// level for fresh encryptions, lower after an upstream linear step).
static int sort_queries(const secpe_ctx *ctx, const secpe_query *q, int nq_, std::vector<int> &order,
                        std::vector<int> &rr, std::vector<int> &cps, int *lin) {
    const int n = ctx->n;
    *lin = -1;
    if (nq_ > SECPE_MAX_BATCH_CONST) return SECPE_EINVAL;
    order.resize(nq_);
    rr.resize(nq_);
    cps.resize(nq_);
    for (int b = 0; b < nq_; b++) {
        if (q[b].C < 2 || q[b].C > n / 2 || q[b].K < 1 || !q[b].cts || !q[b].z_out || !q[b].z_out->data || !aligned16(q[b].z_out->data))
            return SECPE_EINVAL;
        rr[b] = log2_ceil_pow(q[b].C, cps[b]);
        if (2 * cps[b] > n / 2) return SECPE_EINVAL;
        for (int i = 0; i < q[b].K; i++) {
            const secpe_ct &c = q[b].cts[i];
            if (*lin < 0) *lin = c.level;
            if (!c.data || !aligned16(c.data) || c.level != *lin || c.level > ctx->L || c.cap < c.level + 1)
                return SECPE_EINVAL;
            if (!scales_match(c.scale, ctx->scale)) return SECPE_ESCALE;
        }
    }
    if (*lin < ctx->p.reserve + 1) return SECPE_ELEVEL;
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return rr[x] > rr[y]; });
    return SECPE_OK;
}

// Ensemble aggregation of every query (SecPE Sec. 3.1 step 3, Eq. norm
// scale) into Yn in sorted order, at the inputs' level L - 1: one launch
// sums every query's K inputs, one scalar product per query applies
// 1/(K (D_max - D_min)).
static int aggregate_sorted(secpe_ctx *ctx, Eval &E, const secpe_query *q, const std::vector<int> &order, int L,
                            Ct &Yn) {
    const int nq_ = (int)order.size();
    Ct Y;
    SECPE_CHECK(ct_alloc(ctx, nq_, L, ctx->scale, Y));
    std::vector<const u64 *> src;
    std::vector<int> cap, qoff(1, 0);
    std::vector<double> w(nq_);
    for (int s = 0; s < nq_; s++) {
        const secpe_query &Q = q[order[s]];
        for (int i = 0; i < Q.K; i++) {
            src.push_back((const u64 *)Q.cts[i].data);
            cap.push_back(Q.cts[i].cap);
        }
        qoff.push_back((int)src.size());
        w[s] = 1.0 / (Q.K * (Q.d_max - Q.d_min));
    }
    SECPE_CHECK(launch_sum_cts(ctx, src, cap, qoff, Y.v, L + 1));
    return E.mul_const(Y, w, ctx->scale, L - 1, Yn);
}

// z of the sorted items [s, e) of z into the queries' z_out buffers.
static int copy_z(secpe_ctx *ctx, const secpe_query *q, const std::vector<int> &order, int s0, const Ct &z) {
    const int n = ctx->n;
    for (int s = s0; s < s0 + z.B(); s++) {
        secpe_ct *zo = q[order[s]].z_out;
        if (zo->cap < z.level() + 1) return SECPE_EINVAL;
        const u64 *src = z.v.data + (long long)(s - s0) * z.v.stride;
        SECPE_CUDA(cudaMemcpy2DAsync(zo->data, sizeof(u64) * zo->cap * n, src, sizeof(u64) * z.v.cap * n,
                                     sizeof(u64) * (z.level() + 1) * n, 2, cudaMemcpyDeviceToDevice, ctx->stream));
        zo->level = z.level();
        zo->scale = z.scale();
    }
    return SECPE_OK;
}

// The Phoenix baseline over a batch: aggregation as for SecPE, then one
// batched Eval::phoenix per group of equal C'.
static int phoenix_batch_tenant(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q, int nq_) {
    std::vector<int> order, rr, cps;
    int lin;
    SECPE_CHECK(sort_queries(ctx, q, nq_, order, rr, cps, &lin));
    Eval E{ctx, keys, {}, 0};
    Ct Yn;
    SECPE_CHECK(aggregate_sorted(ctx, E, q, order, lin, Yn));
    for (int s = 0; s < nq_;) {
        int e = s;
        while (e < nq_ && rr[order[e]] == rr[order[s]]) e++;
        Eval Eg{ctx, keys, {}, 0};
        for (int k = s; k < e; k++) Eg.qseeds.push_back(q[order[k]].qseed);
        Ct z;
        SECPE_CHECK(Eg.phoenix(ct_slice(Yn, s, e), q[order[s]].C, z));
        SECPE_CHECK(copy_z(ctx, q, order, s, z));
        s = e;
    }
    return SECPE_OK;
}

static int argmax_batch_tenant(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q, int nq_) {
    std::vector<int> order, rr, cps;
    int L;  // the inputs' level
    SECPE_CHECK(sort_queries(ctx, q, nq_, order, rr, cps, &L));
    Eval E{ctx, keys, {}, 0};

    // 1. aggregation into Yn (sorted order), level L - 1
    Ct Yn;
    SECPE_CHECK(aggregate_sorted(ctx, E, q, order, L, Yn));

    // 2. duplication y + RotR(y, C') per group of equal r
    std::vector<Ct> ydup_parts;
    Ct Ydup;
    SECPE_CHECK(ct_alloc(ctx, nq_, L - 1, ctx->scale, Ydup));
    for (int s = 0; s < nq_;) {
        int e = s;
        while (e < nq_ && rr[order[e]] == rr[order[s]]) e++;
        Eval Eg{ctx, keys, {}, 0};
        Ct part = ct_slice(Yn, s, e), rot, sum;
        SECPE_CHECK(Eg.rotate(part, -cps[order[s]], rot));
        Ct dst = ct_slice(Ydup, s, e);
        SECPE_CHECK(launch_addsub(ctx, part.v, rot.v, dst.v, L, false));
        s = e;
    }
    Yn = Ct();

    // 3. phases, level-aware: every query follows its plan (one per r).  A
    // run is a range of sorted queries whose levels have agreed so far; it
    // splits where their plans part (where one of them enters its last
    // range), so each batched step has one level.
    std::map<int, LevelPlan> plans;
    for (int s = 0; s < nq_; s++) {
        const int r = rr[order[s]];
        if (!plans.count(r)) SECPE_CHECK(make_level_plan(ctx, r, L - 1, plans[r]));
    }
    struct Run {
        int s, e;
        Ct y;
        u64 ridx;
    };
    std::vector<Run> runs{{0, nq_, Ydup, 0}};
    const int rmax = rr[order[0]];
    for (int k = 0; k <= rmax; k++) {
        int cnt_gt = 0, cnt_ge = 0;
        for (int s = 0; s < nq_; s++) {
            if (rr[order[s]] > k) cnt_gt++;
            if (rr[order[s]] >= k) cnt_ge++;
        }
        // queries finishing now (r = k, one plan): [cnt_gt, cnt_ge)
        for (const Run &ru : runs) {
            const int s = std::max(ru.s, cnt_gt), e = std::min(ru.e, cnt_ge);
            if (s >= e) continue;
            const LevelPlan &lp = plans[k];
            Eval Ef{ctx, keys, {}, ru.ridx, &lp};
            for (int b = s; b < e; b++) Ef.qseeds.push_back(q[order[b]].qseed);
            Ct yf = ct_slice(ru.y, s - ru.s, e - ru.s), df = ct_slice(Ydup, s, e);
            if (yf.level() != lp.lv[k]) return SECPE_ELEVEL;
            Ct al, d, sgn, z;
            SECPE_CHECK(Ef.mul_const(df, {1.0}, yf.scale(), yf.level(), al));
            SECPE_CHECK(Ef.sub(al, yf, d));
            SECPE_CHECK(Ef.sign(d, 0, sgn, 1.0, true));
            SECPE_CHECK(Ef.add_const(sgn, 1.0, z));
            SECPE_CHECK(copy_z(ctx, q, order, s, z));
        }
        if (cnt_gt == 0) break;
        // QuickMax round k of the queries with r > k: [0, cnt_gt)
        std::vector<Run> next;
        for (const Run &ru : runs) {
            const int e_act = std::min(ru.e, cnt_gt);
            for (int s = ru.s; s < e_act;) {
                const LevelPlan &lp = plans[rr[order[s]]];
                const std::vector<int> sig = lp.signature(k);
                int e = s + 1;
                while (e < e_act && plans[rr[order[e]]].signature(k) == sig) e++;
                Eval Er{ctx, keys, {}, ru.ridx, &lp};
                for (int b = s; b < e; b++) Er.qseeds.push_back(q[order[b]].qseed);
                Ct yr = ct_slice(ru.y, s - ru.s, e - ru.s), ye, a, m;
                if (yr.level() > lp.lv[k]) yr = ct_drop(yr, lp.lv[k]);
                if (yr.level() != lp.lv[k]) return SECPE_ELEVEL;
                SECPE_CHECK(Er.ensure(yr, 1, ye));
                SECPE_CHECK(Er.rotate(ye, 1 << k, a));
                SECPE_CHECK(Er.max(a, ye, m));
                next.push_back({s, e, m, Er.ridx});
                s = e;
            }
        }
        runs = std::move(next);
    }
    return SECPE_OK;
}
