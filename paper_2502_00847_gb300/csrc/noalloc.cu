// Allocation-free rescale.
//
// secpe_rescale normally takes its scratch buffers (the inverse NTT of the
// last limb and the converted limbs) from the CUDA stream-ordered allocator.
// Some callers cannot allow any allocation during the call: serving loops
// that must keep a fixed device memory footprint and never touch the
// allocator on the critical path, and hosts that manage all device memory
// through their own pool and forbid hidden allocations.  secpe_rescale_noalloc serves them: its scratch is
// one file-scope __device__ array of fixed size that every GPU holding this
// library keeps until the process exits.  Under CUDA's default lazy module
// loading the array is reserved on a device when this file's module is
// first loaded there, which is the first call's set-up (cudaGetSymbolAddress):
// that first call can still fail with SECPE_ECUDA if the device is full, so
// make one warm-up call per device at start-up, before admitting requests
// and before any stream capture.
//
// Limits and contract:
//  * the scratch holds SECPE_NOALLOC_SCRATCH_WORDS 64-bit words; a call
//    needs 2 * N * (level + 1) words and is rejected with SECPE_EINVAL when
//    that is larger (N = 2^16 allows levels up to 23);
//  * the device address of the array is looked up once per device, with
//    that device current, by the first call on it (which also loads the
//    module and so reserves the array); make that first call at start-up,
//    before any stream capture;
//  * out may be in itself (same data and cap: every output residue depends
//    only on the input residue at the same position and on the scratch);
//    any other overlap of the two buffers is rejected with SECPE_EINVAL;
//  * all calls share the one array and it keeps the last call's contents:
//    calls whose kernels may overlap on the GPU (different streams without
//    ordering) race on it and must not be issued.
#include <mutex>

#include "eval.h"

#define SECPE_NOALLOC_SCRATCH_WORDS (2ull * 65536ull * 24ull)

static __device__ __align__(256) u64 g_noalloc_scratch[SECPE_NOALLOC_SCRATCH_WORDS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
u64 *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device (set-up on
// first use per device).
int scratch_address(u64 **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SECPE_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SECPE_ECUDA;
        }
        g_scratch_ptr[dev] = (u64 *)p;
    }
    *out = g_scratch_ptr[dev];
    return SECPE_OK;
}

}  // namespace

extern "C" int secpe_rescale_noalloc(secpe_ctx *ctx, const secpe_ct *in, secpe_ct *out, void *stream) {
    // the validation of secpe_rescale, with its error codes
    if (!ctx || !in || !out || !in->data || !out->data || !aligned16(in->data) || !aligned16(out->data))
        return SECPE_EINVAL;
    if (in->level < 0 || in->level > ctx->L || in->cap < in->level + 1 || !(in->scale > 0.0)) return SECPE_EINVAL;
    if (in->level < 1) return SECPE_ELEVEL;
    if (out->cap < in->level) return SECPE_EINVAL;
    {
        // out is written while in is still read: only the exact in-place layout is safe
        const u64 *ib = (const u64 *)in->data, *ie = ib + 2ull * in->cap * ctx->n;
        const u64 *ob = (const u64 *)out->data, *oe = ob + 2ull * out->cap * ctx->n;
        const bool overlap = ob < ie && ib < oe;
        if (overlap && !(ob == ib && out->cap == in->cap)) return SECPE_EINVAL;
    }
    const int n = ctx->n, lv = in->level;
    const unsigned long long need = 2ull * n * (lv + 1);
    if (need > SECPE_NOALLOC_SCRATCH_WORDS) return SECPE_EINVAL;
    u64 *scratch = nullptr;
    SECPE_CHECK(scratch_address(&scratch));
    ctx->stream = (cudaStream_t)stream;
    u64 *y = scratch;               // [2][N]: inverse NTT of the last limb
    u64 *z = scratch + 2ull * n;    // [2][lv][N]: converted limbs
    CtB x = {(u64 *)in->data, 1, 2ll * in->cap * n, in->cap, lv, in->scale, n};
    CtB o = {(u64 *)out->data, 1, 2ll * out->cap * n, out->cap, lv - 1, in->scale / (double)ctx->primes[lv], n};
    LimbSet ysrc = make_limbset(x.data + (size_t)lv * n, 1, x.stride, 2, x.pstride(), 1, lv);
    LimbSet ydst = make_limbset(y, 1, 2ll * n, 2, n, 1, lv);
    SECPE_CHECK(ntt_limbset(ctx, ydst, true, &ysrc));
    if (fused_path(ctx)) {
        SECPE_CHECK(rescale_fused(ctx, x, y, o, z));
    } else {
        SECPE_CHECK(launch_rescale_prep(ctx, y, z, 1, lv));
        LimbSet zls = make_limbset(z, 1, 2ll * lv * n, 2, (long long)lv * n, lv, 0);
        SECPE_CHECK(ntt_limbset(ctx, zls, false));
        SECPE_CHECK(launch_rescale_fin(ctx, x, z, o, lv));
    }
    if (cudaGetLastError() != cudaSuccess) return SECPE_ECUDA;
    out->level = lv - 1;
    out->scale = o.scale;
    return SECPE_OK;
}
