// Kernel-launch helpers shared by the library's .cu files.
#pragma once
#include "internal.h"

// Launch on ctx->stream, count it, and turn a launch error into SECPE_ECUDA.
#define SECPE_LAUNCH(ctx, kernel, grid, block, smem, ...)                               \
    do {                                                                                  \
        kernel<<<(grid), (block), (smem), (ctx)->stream>>>(__VA_ARGS__);                  \
        (ctx)->counters.launches++;                                                       \
        cudaError_t _e = cudaGetLastError();                                              \
        if (_e != cudaSuccess) return SECPE_ECUDA;                                        \
    } while (0)

#define SECPE_CHECK(expr)                  \
    do {                                   \
        int _s = (expr);                   \
        if (_s != SECPE_OK) return _s;     \
    } while (0)

#define SECPE_CUDA(expr)                               \
    do {                                               \
        if ((expr) != cudaSuccess) return SECPE_ECUDA; \
    } while (0)

static inline unsigned grid1d(long long work, int block) {
    return (unsigned)((work + block - 1) / block);
}

// ---------------------------------------------------------------------------
// NTT entry points (ntt.cu)
// ---------------------------------------------------------------------------
// Forward or inverse NTT of every limb of `ls`; in place, or reading from
// the limbs of `src` (same shape) when src is not null.
int ntt_limbset(secpe_ctx *ctx, const LimbSet &ls, bool inverse, const LimbSet *src = nullptr);

// Convenience: LimbSet for `nitem` ciphertext-like objects of `npoly`
// polynomials, limbs [l0, l0 + nlimb) mapped to primes [p0, p0 + nlimb).
LimbSet make_limbset(u64 *base, int nitem, long long item_stride, int npoly,
                     long long poly_stride, int nlimb, int prime0);
