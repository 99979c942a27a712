// Continuous-batching server for encrypted ensemble Argmax queries.
//
// A query moves through the phases of SecPE Alg. 1 (as split by the batched
// driver): phase -1 = aggregation + duplication (y + RotR(y, C')), phase
// k = 0..r-1 = QuickMax round k, phase r = final Sign(y_dup - y_max) + 1.
// All queries of one tenant (key set) at the same phase of the same
// class-count power C' share level, scale and refresh history, so the server
// runs one phase for a whole group as one batched evaluation.  Each call to
// secpe_server_step admits what fits, then enqueues one phase of every group
// of admitted queries (groups of at most max_batch queries, in the order of
// their oldest member): every query in flight advances by one phase per
// step, and a query submitted while others are mid-circuit starts its
// aggregation in the next step, its launches interleaved on the stream with
// theirs.
// Per-query state (y_dup, y) stays resident on the device between phases.
// Admission: a query is admitted when the state it will hold fits the HBM
// budget next to the keys, the states in flight and the largest scratch of
// one step; otherwise it waits in the host queue (or is rejected at submit
// if it could never fit).
#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <tuple>

#include "eval.h"

int argmax_batch_impl(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q, int nq_);

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct QState {
    int64_t ticket = 0;
    secpe_query q;
    const secpe_keys *keys = nullptr;  // the query's tenant key set
    int r = 0, cp = 1;
    int phase = -2;  // -2 waiting for admission, -1 aggregate+dup, 0..r-1 rounds, r final
    Ct ydup, y;
    u64 ridx = 0;
    LevelPlan plan;  // the query's levels (level-aware QuickMax)
    bool done = false, cancelled = false;
    cudaEvent_t done_ev = nullptr;
    double t_submit = 0, t_admit = 0;
    size_t state_bytes = 0;
};

}  // namespace

struct secpe_server {
    secpe_ctx *ctx;
    const secpe_keys *keys;            // default key set
    std::map<const secpe_keys *, size_t> key_sets;  // every key set seen, with its device bytes
    size_t budget, keys_bytes, scratch_bytes, in_flight_bytes = 0;
    int max_batch;
    int64_t next_ticket = 1;
    std::map<int64_t, QState> q;       // by ticket
    std::deque<int64_t> waiting;       // not admitted yet, FIFO
    std::vector<cudaEvent_t> free_events;
    int64_t completed = 0;
};

namespace {

size_t ct_bytes(const secpe_ctx *ctx, int level) { return sizeof(u64) * 2ull * (level + 1) * ctx->n; }

// device bytes of a key set: relinearisation + Galois keys, secret key
size_t key_set_bytes(const secpe_ctx *ctx, const secpe_keys *keys) {
    const size_t keyb = sizeof(u64) * (size_t)ctx->n * ctx->nprimes * 2 * ((ctx->L + ctx->alpha) / ctx->alpha);
    return keyb * (1 + keys->gks.size()) + sizeof(u64) * (size_t)ctx->n * ctx->nprimes;
}

// device bytes a query holds while in flight: y_dup + y + z (top level bound)
size_t query_state_bytes(const secpe_ctx *ctx) { return 3 * ct_bytes(ctx, ctx->L); }

// scratch of one batched step of B queries (key switch at the top level:
// INTT(d), extended limbs, accumulators, conversion), plus the poly9 temporaries
size_t step_scratch_bytes(const secpe_ctx *ctx, int B) {
    const size_t limb = sizeof(u64) * ctx->n;
    const int L = ctx->L, nt = L + 1 + ctx->npsp, ndig = (L + ctx->alpha) / ctx->alpha;
    const size_t ks = (size_t)B * limb * ((L + 1) + (size_t)ndig * nt + 2 * nt + 2 * (L + 1));
    return ks + (size_t)12 * B * ct_bytes(ctx, L);
}

int admit(secpe_server *s, QState &st) {
    st.phase = -1;
    st.t_admit = now_s();
    st.state_bytes = query_state_bytes(s->ctx);
    s->in_flight_bytes += st.state_bytes;
    return SECPE_OK;
}

void release(secpe_server *s, QState &st) {
    st.ydup = Ct();
    st.y = Ct();
    s->in_flight_bytes -= st.state_bytes;
    st.state_bytes = 0;
}

void try_admit(secpe_server *s) {
    while (!s->waiting.empty()) {
        QState &st = s->q[s->waiting.front()];
        if (st.cancelled) {
            s->waiting.pop_front();
            continue;
        }
        const size_t need = s->keys_bytes + s->in_flight_bytes + query_state_bytes(s->ctx) + s->scratch_bytes;
        if (need > s->budget) break;
        admit(s, st);
        s->waiting.pop_front();
    }
}

int cp_of(int C, int &r) {
    int cp = 1;
    r = 0;
    while (cp < C) {
        cp <<= 1;
        r++;
    }
    return cp;
}

// gather the y (or y_dup) of a group into one contiguous batch
int gather(secpe_ctx *ctx, const std::vector<QState *> &g, bool dup, Ct &out) {
    const Ct &first = dup ? g[0]->ydup : g[0]->y;
    SECPE_CHECK(ct_alloc(ctx, (int)g.size(), first.level(), first.scale(), out));
    const size_t n = ctx->n;
    for (size_t i = 0; i < g.size(); i++) {
        const Ct &c = dup ? g[i]->ydup : g[i]->y;
        if (c.level() != first.level()) return SECPE_EINVAL;
        SECPE_CUDA(cudaMemcpy2DAsync(out.v.data + i * out.v.stride, sizeof(u64) * out.v.cap * n, c.v.data,
                                     sizeof(u64) * c.v.cap * n, sizeof(u64) * (c.level() + 1) * n, 2,
                                     cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return SECPE_OK;
}

int run_group(secpe_server *s, std::vector<QState *> &g) {
    secpe_ctx *ctx = s->ctx;
    const int phase = g[0]->phase, r = g[0]->r;
    Eval E{ctx, g[0]->keys, {}, g[0]->ridx, &g[0]->plan};
    for (QState *st : g) E.qseeds.push_back(st->q.qseed);
    const int B = (int)g.size(), n = ctx->n, L = ctx->L;
    if (phase == -1) {
        // aggregation of each query (ragged K), then one batched duplication
        Ct Y;
        SECPE_CHECK(ct_alloc(ctx, B, L, ctx->scale, Y));
        std::vector<double> w(B);
        std::vector<const u64 *> src;
        std::vector<int> cap, qoff(1, 0);
        for (int b = 0; b < B; b++) {
            const secpe_query &Q = g[b]->q;
            for (int i = 0; i < Q.K; i++) {
                src.push_back((const u64 *)Q.cts[i].data);
                cap.push_back(Q.cts[i].cap);
            }
            qoff.push_back((int)src.size());
            w[b] = 1.0 / (Q.K * (Q.d_max - Q.d_min));
        }
        SECPE_CHECK(launch_sum_cts(ctx, src, cap, qoff, Y.v, L + 1));
        Ct Yn, rot, dup;
        SECPE_CHECK(E.mul_const(Y, w, ctx->scale, L - 1, Yn));
        Y = Ct();
        SECPE_CHECK(E.rotate(Yn, -g[0]->cp, rot));
        SECPE_CHECK(E.add(Yn, rot, dup));
        for (int b = 0; b < B; b++) {
            g[b]->ydup = ct_slice(dup, b, b + 1);
            g[b]->y = g[b]->ydup;
            g[b]->phase = 0;
        }
        return SECPE_OK;
    }
    Ct y;
    SECPE_CHECK(gather(ctx, g, false, y));
    const int planned = g[0]->plan.lv[phase];
    if (y.level() > planned) y = ct_drop(y, planned);
    if (y.level() != planned) return SECPE_ELEVEL;
    if (phase < r) {
        Ct ye, a, m;
        SECPE_CHECK(E.ensure(y, 1, ye));
        SECPE_CHECK(E.rotate(ye, 1 << phase, a));
        SECPE_CHECK(E.max(a, ye, m));
        for (int b = 0; b < B; b++) {
            g[b]->y = ct_slice(m, b, b + 1);
            g[b]->ridx = E.ridx;
            g[b]->phase++;
        }
        return SECPE_OK;
    }
    // final phase
    Ct yd, al, d, sg, z;
    SECPE_CHECK(gather(ctx, g, true, yd));
    SECPE_CHECK(E.mul_const(yd, {1.0}, y.scale(), y.level(), al));
    SECPE_CHECK(E.sub(al, y, d));
    SECPE_CHECK(E.sign(d, 0, sg, 1.0, true));
    SECPE_CHECK(E.add_const(sg, 1.0, z));
    for (int b = 0; b < B; b++) {
        secpe_ct *zo = g[b]->q.z_out;
        if (zo->cap < z.level() + 1) return SECPE_EINVAL;
        SECPE_CUDA(cudaMemcpy2DAsync(zo->data, sizeof(u64) * zo->cap * n, z.v.data + (long long)b * z.v.stride,
                                     sizeof(u64) * z.v.cap * n, sizeof(u64) * (z.level() + 1) * n, 2,
                                     cudaMemcpyDeviceToDevice, ctx->stream));
        zo->level = z.level();
        zo->scale = z.scale();
        SECPE_CUDA(cudaEventRecord(g[b]->done_ev, ctx->stream));
        g[b]->done = true;
        g[b]->phase = r + 1;
    }
    return SECPE_OK;
}

}  // namespace

extern "C" int secpe_server_create(secpe_ctx *ctx, const secpe_keys *keys, uint64_t hbm_budget_bytes, int max_batch,
                                   secpe_server **out) {
    if (!ctx || !keys || !out || max_batch < 1 || max_batch > SECPE_MAX_BATCH_CONST) return SECPE_EINVAL;
    secpe_server *s = new secpe_server();
    s->ctx = ctx;
    s->keys = keys;
    s->budget = hbm_budget_bytes;
    s->max_batch = max_batch;
    s->keys_bytes = key_set_bytes(ctx, keys);
    s->key_sets[keys] = s->keys_bytes;
    s->scratch_bytes = step_scratch_bytes(ctx, max_batch);
    if (s->keys_bytes + s->scratch_bytes + query_state_bytes(ctx) > s->budget) {
        delete s;
        return SECPE_EADMIT;
    }
    *out = s;
    return SECPE_OK;
}

extern "C" void secpe_server_destroy(secpe_server *s) {
    if (!s) return;
    cudaDeviceSynchronize();
    for (auto &kv : s->q)
        if (kv.second.done_ev) cudaEventDestroy(kv.second.done_ev);
    for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
    delete s;
}

extern "C" int secpe_server_submit(secpe_server *s, const secpe_query *q, int64_t *ticket) {
    if (!s || !q || !ticket || !q->cts || !q->z_out || !q->z_out->data || !aligned16(q->z_out->data) || q->K < 1 ||
        q->C < 2 || !(q->d_max > q->d_min))
        return SECPE_EINVAL;
    const secpe_ctx *ctx = s->ctx;
    if (q->C > ctx->n / 2) return SECPE_EINVAL;
    int r;
    const int cp = cp_of(q->C, r);
    if (2 * cp > ctx->n / 2) return SECPE_EINVAL;
    for (int i = 0; i < q->K; i++) {
        const secpe_ct &c = q->cts[i];
        if (!c.data || !aligned16(c.data) || c.level != ctx->L || c.cap < ctx->L + 1) return SECPE_EINVAL;
        if (std::fabs(c.scale - ctx->scale) > ctx->scale * std::ldexp(1.0, -40)) return SECPE_ESCALE;
    }
    const secpe_keys *keys = q->keys ? q->keys : s->keys;
    if (!keys->rlk || !galois_key(keys, galois_elt(ctx, -cp))) return SECPE_EKEY;
    for (int i = 0; i < r; i++)
        if (!galois_key(keys, galois_elt(ctx, 1 << i))) return SECPE_EKEY;
    if (!s->key_sets.count(keys)) {
        // a new tenant: its keys are resident from now on
        const size_t kb = key_set_bytes(ctx, keys);
        if (s->keys_bytes + kb + s->scratch_bytes + query_state_bytes(ctx) > s->budget) return SECPE_EADMIT;
        s->key_sets[keys] = kb;
        s->keys_bytes += kb;
    }
    QState st;
    SECPE_CHECK(make_level_plan(ctx, r, ctx->L - 1, st.plan));
    st.ticket = s->next_ticket++;
    st.q = *q;
    st.keys = keys;
    st.r = r;
    st.cp = cp;
    st.t_submit = now_s();
    if (!s->free_events.empty()) {
        st.done_ev = s->free_events.back();
        s->free_events.pop_back();
    } else if (cudaEventCreateWithFlags(&st.done_ev, cudaEventDisableTiming) != cudaSuccess) {
        return SECPE_ECUDA;
    }
    s->q[st.ticket] = st;
    s->waiting.push_back(st.ticket);
    *ticket = st.ticket;
    return SECPE_OK;
}

extern "C" int secpe_server_cancel(secpe_server *s, int64_t ticket) {
    if (!s) return SECPE_EINVAL;
    auto it = s->q.find(ticket);
    if (it == s->q.end() || it->second.done) return SECPE_EINVAL;
    QState &st = it->second;
    st.cancelled = true;
    if (st.phase >= -1) release(s, st);
    st.phase = st.r + 2;
    return SECPE_OK;
}

extern "C" int secpe_server_step(secpe_server *s, void *stream, int *launched) {
    if (!s) return SECPE_EINVAL;
    secpe_ctx *ctx = s->ctx;
    ctx->stream = (cudaStream_t)stream;
    if (launched) *launched = 0;
    try_admit(s);
    // queries at the same point of the circuit form a group: same tenant,
    // phase and kind (the duplication needs the same C' key; a QuickMax round
    // k is common to all queries with r > k; the final phase k is shared by
    // queries with r = k) and the same levels through the phase (their level
    // plans' signature for it)
    auto kind = [](const QState &st) { return st.phase < 0 ? 2 * st.cp : (st.phase < st.r ? 0 : 1); };
    std::map<std::tuple<const secpe_keys *, int, int, std::vector<int>>, std::vector<QState *>> groups;
    for (auto &kv : s->q) {
        QState &st = kv.second;
        if (st.cancelled || st.done || st.phase < -1) continue;
        const std::vector<int> sig = st.phase >= 0 ? st.plan.signature(st.phase) : std::vector<int>();
        groups[std::make_tuple(st.keys, st.phase, kind(st), sig)].push_back(&st);
    }
    std::vector<std::vector<QState *>> runs;
    auto older = [](const QState *a, const QState *b) { return a->t_admit < b->t_admit; };
    for (auto &kv : groups) {
        std::vector<QState *> &g = kv.second;
        std::sort(g.begin(), g.end(), older);
        for (size_t i = 0; i < g.size(); i += (size_t)s->max_batch)
            runs.emplace_back(g.begin() + i, g.begin() + std::min(g.size(), i + (size_t)s->max_batch));
    }
    std::sort(runs.begin(), runs.end(),
              [&](const std::vector<QState *> &a, const std::vector<QState *> &b) { return older(a[0], b[0]); });
    int total = 0;
    for (std::vector<QState *> &g : runs) {
        SECPE_CHECK(run_group(s, g));
        total += (int)g.size();
        for (QState *st : g)
            if (st->done) release(s, *st);
    }
    if (launched) *launched = total;
    return cudaGetLastError() == cudaSuccess ? SECPE_OK : SECPE_ECUDA;
}

extern "C" int secpe_server_poll(secpe_server *s, int64_t ticket, int *done) {
    if (!s || !done) return SECPE_EINVAL;
    auto it = s->q.find(ticket);
    if (it == s->q.end()) return SECPE_EINVAL;
    QState &st = it->second;
    if (st.cancelled) {
        *done = -1;
        return SECPE_OK;
    }
    if (!st.done) {
        *done = 0;
        return SECPE_OK;
    }
    const cudaError_t e = cudaEventQuery(st.done_ev);
    if (e == cudaErrorNotReady) {
        *done = 0;
        return SECPE_OK;
    }
    if (e != cudaSuccess) return SECPE_ECUDA;
    *done = 1;
    return SECPE_OK;
}

extern "C" int secpe_server_wait(secpe_server *s, int64_t ticket, double timeout_s) {
    if (!s) return SECPE_EINVAL;
    const double t0 = now_s();
    for (;;) {
        int d = 0;
        SECPE_CHECK(secpe_server_poll(s, ticket, &d));
        if (d == 1) return SECPE_OK;
        if (d == -1) return SECPE_EINVAL;
        if (now_s() - t0 > timeout_s) return SECPE_ETIMEOUT;
        if (!s->q[ticket].done) {
            int launched = 0;
            SECPE_CHECK(secpe_server_step(s, s->ctx->stream, &launched));
        }
    }
}

extern "C" int secpe_server_forget(secpe_server *s, int64_t ticket) {
    if (!s) return SECPE_EINVAL;
    auto it = s->q.find(ticket);
    if (it == s->q.end()) return SECPE_EINVAL;
    QState &st = it->second;
    if (!st.done && !st.cancelled) return SECPE_EINVAL;
    if (st.done_ev) s->free_events.push_back(st.done_ev);
    s->q.erase(it);
    return SECPE_OK;
}

extern "C" int secpe_server_stats(const secpe_server *s, secpe_server_stats_t *out) {
    if (!s || !out) return SECPE_EINVAL;
    int waiting = 0, active = 0, done = 0;
    for (auto &kv : s->q) {
        const QState &st = kv.second;
        if (st.cancelled) continue;
        if (st.done) done++;
        else if (st.phase < -1) waiting++;
        else active++;
    }
    out->waiting = waiting;
    out->active = active;
    out->done = done;
    out->in_flight_bytes = s->in_flight_bytes;
    out->keys_bytes = s->keys_bytes;
    out->scratch_bytes = s->scratch_bytes;
    return SECPE_OK;
}
