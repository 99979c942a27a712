// Device building blocks of the NTT kernels (shared by ntt.cu and
// ntt_fused.cu): limb addressing, radix-16 register rounds with lazy
// (Harvey) butterflies, final corrections.  See ntt.cu for the network.
#pragma once
#include "internal.h"

#define PADR(p) ((p) + ((p) >> 4))

struct LimbRef {
    u64 *ptr;
    int prime;
};

static __device__ __forceinline__ LimbRef limb_of(const LimbSet &ls, int n, long long lid) {
    int j = (int)(lid % ls.nlimb);
    long long t2 = lid / ls.nlimb;
    int poly = (int)(t2 % ls.npoly);
    long long item = t2 / ls.npoly;
    LimbRef r;
    r.ptr = ls.base + item * ls.item_stride + poly * ls.poly_stride + (long long)j * n;
    r.prime = ls.prime_of[poly * ls.nlimb + j];
    return r;
}

// Butterflies use D. Harvey's lazy reduction ("Faster arithmetic for
// number-theoretic transforms", 2014): the forward network keeps values in
// [0, 4q), the inverse in [0, 2q); one correction to [0, q) is applied when
// the last pass stores.  Within a round, the twiddle of stage bit sb for
// register k depends only on k >> (sb + 1) (p0 has no bits in the round's
// window), so each distinct twiddle is loaded once.
template <int LOGP, int LO>
static __device__ __forceinline__ void fwd_round(u64 (&x)[16], int p0, const ulonglong2 *__restrict__ tw,
                                          int base, u64 q) {
    const u64 q2 = 2 * q;
#pragma unroll
    for (int sb = 3; sb >= 0; --sb) {
        const int s = LO + sb;
        const int st = LOGP - 1 - s;
        const int ibase = (base << st) + (p0 >> (s + 1));
        ulonglong2 w[8];
#pragma unroll
        for (int g = 0; g < 8; ++g)
            if (g < (8 >> sb)) w[g] = tw[ibase + g];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (k & (1 << sb)) continue;
            const ulonglong2 ww = w[k >> (sb + 1)];
            u64 u = x[k];
            u = u >= q2 ? u - q2 : u;
            const u64 t = mul_shoup_lazy(x[k | (1 << sb)], ww.x, ww.y, q);
            x[k] = u + t;
            x[k | (1 << sb)] = u - t + q2;
        }
    }
}

template <int LOGP, int LO, bool LAST>
static __device__ __forceinline__ void inv_round(u64 (&x)[16], int p0, const ulonglong2 *__restrict__ tw,
                                          int base, u64 q, ulonglong2 ninv, ulonglong2 ninv_w1) {
    const u64 q2 = 2 * q;
#pragma unroll
    for (int sb = 0; sb < 4; ++sb) {
        const int s = LO + sb;
        const int st = LOGP - 1 - s;
        const bool last = LAST && s == LOGP - 1;
        const int ibase = (base << st) + (p0 >> (s + 1));
        ulonglong2 w[8];
#pragma unroll
        for (int g = 0; g < 8; ++g)
            if (g < (8 >> sb)) w[g] = last ? ninv_w1 : tw[ibase + g];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (k & (1 << sb)) continue;
            const ulonglong2 ww = w[k >> (sb + 1)];
            const u64 u = x[k];
            const u64 v = x[k | (1 << sb)];
            if (last) {
                x[k] = mul_shoup_lazy(u + v, ninv.x, ninv.y, q);
            } else {
                const u64 sum = u + v;
                x[k] = sum >= q2 ? sum - q2 : sum;
            }
            x[k | (1 << sb)] = mul_shoup_lazy(u - v + q2, ww.x, ww.y, q);
        }
    }
}

// [0, 4q) -> [0, q)
static __device__ __forceinline__ u64 reduce4(u64 v, u64 q) {
    v = v >= 2 * q ? v - 2 * q : v;
    return v >= q ? v - q : v;
}
// [0, 2q) -> [0, q)
static __device__ __forceinline__ u64 reduce2(u64 v, u64 q) { return v >= q ? v - q : v; }


// Asks L2 to fetch the 128-byte line holding p (no register result).
static __device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Prefetches a contiguous 32 KiB tile (16 rows of 256 words) to L2: 256
// lines, one per thread of a 256-thread block.
static __device__ __forceinline__ void prefetch_tile_l2(const u64 *tile) {
    prefetch_l2(tile + 16 * threadIdx.x);
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, cp.async.bulk) from global to shared memory,
// completed on a shared-memory mbarrier.  Every wait is bounded: a wait that
// gives up records SECPE_ETIMEOUT in the context's status word.
#define SECPE_WAIT_LIMIT (1L << 22)

static __device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
static __device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Arms the barrier for `bytes` of incoming copies (one arrival).
static __device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// Copies `bytes` (a multiple of 16; both addresses 16-byte aligned).
static __device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
static __device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for phase `parity` of the barrier; false after `limit` polls.
static __device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long limit = SECPE_WAIT_LIMIT) {
    for (long i = 0; i < limit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
