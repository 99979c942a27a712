// Kernel-launch helpers shared by the library's .cu files.
#pragma once
#include "internal.h"

// Records a profiler event: an external record (an event record node) while
// the stream is being captured, a plain record otherwise.
static inline void kprof_record(cudaEvent_t ev, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, st);
}

// Records a CUDA event pair around one launch, under the kernel's name, when
// the context's kernel profiler runs with the filter "*".
struct KprofLaunch {
    secpe_ctx *ctx;
    int idx = -1;
    KprofLaunch(secpe_ctx *c, const char *name) : ctx(c) {
        KProf &k = c->kprof;
        if (!k.active || !k.all || 2 * (k.used + 1) > (int)k.ev.size()) return;
        idx = k.used++;
        k.launches++;
        if ((int)k.names.size() <= idx) k.names.resize(idx + 1);
        k.names[idx] = name;
        kprof_record(k.ev[2 * idx], c->stream);
    }
    ~KprofLaunch() {
        if (idx >= 0) kprof_record(ctx->kprof.ev[2 * idx + 1], ctx->stream);
    }
};

// Launch on ctx->stream, count it, and turn a launch error into SECPE_ECUDA;
// the profiler sees the launch under `name`.
#define SECPE_LAUNCH_AS(ctx, name, kernel, grid, block, smem, ...)                      \
    do {                                                                                  \
        KprofLaunch _kpl((ctx), name);                                                    \
        kernel<<<(grid), (block), (smem), (ctx)->stream>>>(__VA_ARGS__);                  \
        (ctx)->counters.launches++;                                                       \
        cudaError_t _e = cudaGetLastError();                                              \
        if (_e != cudaSuccess) return SECPE_ECUDA;                                        \
    } while (0)
#define SECPE_LAUNCH(ctx, kernel, grid, block, smem, ...) \
    SECPE_LAUNCH_AS(ctx, #kernel, kernel, grid, block, smem, __VA_ARGS__)

#define SECPE_CHECK(expr)                  \
    do {                                   \
        int _s = (expr);                   \
        if (_s != SECPE_OK) return _s;     \
    } while (0)

#define SECPE_CUDA(expr)                               \
    do {                                               \
        if ((expr) != cudaSuccess) return SECPE_ECUDA; \
    } while (0)

// Records a CUDA event pair around the launches made in its lifetime when
// the context's kernel profiler is active and `name` matches its filter.
// Under stream capture the records become event record nodes of the graph
// (each replay re-records them).
// `bytes` are the launch's share of its operation's algorithmic bytes,
// `model` (default: the same) what the launch itself reads and writes,
// `mul32` its algorithmic 32-bit multiplies (MUL32_* below).
struct KprofScope {
    secpe_ctx *ctx;
    int idx = -1;
    KprofScope(secpe_ctx *c, const char *name, double bytes, double model = -1.0, double mul32 = 0.0) : ctx(c) {
        KProf &k = c->kprof;
        if (!k.active || k.all || std::string(name).find(k.filter) == std::string::npos) return;
        if (2 * (k.used + 1) > (int)k.ev.size()) return;
        idx = k.used++;
        k.launches++;
        k.bytes += bytes;
        k.model_bytes += model < 0.0 ? bytes : model;
        k.mul32 += mul32;
        kprof_record(k.ev[2 * idx], c->stream);
    }
    ~KprofScope() {
        if (idx >= 0) kprof_record(ctx->kprof.ev[2 * idx + 1], ctx->stream);
    }
};

// Algorithmic 32-bit multiplies (one mul.lo or mul.hi on 32-bit words each)
// of the 64-bit operations as the kernels form them from 32 x 32 partial
// products: the high half of a 64 x 64 product takes 7 (three of the four
// partial products in both halves and the high half of the lowest), the low
// half 4 (the lowest in both halves, the two cross products' low halves),
// the full 128-bit product or multiply-accumulate 8.
//   Shoup product x*w - hi(x*w')*q:              7 + 4 + 4 = 15
//   Montgomery reduction (lo*q') then hi(m*q):   4 + 7     = 11
//   Montgomery product: full product + reduction          = 19
// One radix-2 pass of 8 stages over a residue costs 8 half-butterflies of
// one Shoup product each: 60 per residue; the inverse transform's last stage
// adds one more Shoup product per butterfly (the folded N^-1): 7.5.
constexpr double MUL32_SHOUP = 15.0, MUL32_REDC = 11.0, MUL32_MAC = 8.0, MUL32_MONT = 19.0;
constexpr double MUL32_PASS = 60.0, MUL32_INV_LAST = 7.5;

static inline unsigned grid1d(long long work, int block) {
    return (unsigned)((work + block - 1) / block);
}

// ---------------------------------------------------------------------------
// NTT entry points (ntt.cu)
// ---------------------------------------------------------------------------
// Forward or inverse NTT of every limb of `ls`; in place, or reading from
// the limbs of `src` (same shape) when src is not null.
// For the N = 2^16 inverse, `scale_tab` (device, pairs) replaces the final
// N^-1 of limb j by scale_tab[2 (scale_off + j)] (and the folded twiddle by
// the next entry): the INTT then also applies a per-limb constant.
// `alg_per_limb` is the algorithmic bytes the transform is charged per limb
// in the profiler: by default 16 N (a transform reads and writes every
// residue once); transforms inside an operation charge what the operation
// reads or writes through them (8 N for an input read once, 0 for an
// intermediate).
int ntt_limbset(secpe_ctx *ctx, const LimbSet &ls, bool inverse, const LimbSet *src = nullptr,
                const ulonglong2 *scale_tab = nullptr, int scale_off = 0, double alg_per_limb = -1.0);

// N = 2^16 only: the row pass (last 8 stages of the forward NTT, first 8 of
// the inverse) alone, in place.
int ntt_rowpass_only(secpe_ctx *ctx, const LimbSet &ls, bool inverse);
// One N = 2^16 pass (TuneSlot TUNE_COLPASS..TUNE_IROWPASS) of every limb of
// ls, in place, with the context's launch configuration for it.
int ntt16_pass(secpe_ctx *ctx, int slot, const LimbSet &ls);
// Bounded-wait self-test kernel (ntt_fused.cu).
int wait_selftest(secpe_ctx *ctx, int arrive, long polls);
// One ModUp-shaped base-conversion pass over buf (ntt_fused.cu).
int bconv_pass_probe(secpe_ctx *ctx, u64 *buf, int nitem, int ntgt);
// Precision variant (ntt_tc.cu): NTT/INTT with both passes on the tensor pipe.
int ntt_limbset_tc(secpe_ctx *ctx, const LimbSet &ls, bool inverse);
void tc_forget_ctx(const secpe_ctx *ctx);

// Convenience: LimbSet for `nitem` ciphertext-like objects of `npoly`
// polynomials, limbs [l0, l0 + nlimb) mapped to primes [p0, p0 + nlimb).
LimbSet make_limbset(u64 *base, int nitem, long long item_stride, int npoly,
                     long long poly_stride, int nlimb, int prime0);
