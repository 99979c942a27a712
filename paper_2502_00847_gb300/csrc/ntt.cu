// Negacyclic NTT / INTT kernels for sm_103a.
//
// Forward transform (natural order in, bit-reversed order out):
//   out[j] = sum_k a[k] psi^((2 brv(j) + 1) k),
// computed by the Cooley-Tukey network whose butterfly in group i of the
// stage with m groups uses the twiddle psi^brv(m + i).  The inverse is the
// Gentleman-Sande network with psi^-brv(m + i), followed by N^-1, which is
// folded into the last stage.
//
// Fast paths (256 threads, a 4096-word tile per CTA, 16 residues per thread):
//  * N = 2^16: two passes of 8 stages.  Pass A transforms 16 adjacent
//    columns (stride-256 elements) per CTA, pass B 16 adjacent rows.  Within
//    a pass, each thread runs 4 stages on 16 registers (radix-16), the tile
//    is exchanged through shared memory once, and the remaining 4 stages run
//    on the new registers.  Global loads/stores are whole 128-byte lines.
//  * N = 2^12: one CTA per limb, three radix-16 rounds in shared memory.
//  * any other N: one launch per radix-2 stage (slow, exact).
// The twiddle of local stage st, local group i, in a pass whose transforms
// start at global group `base` is psi^brv(base * 2^st + i): base = 1 for
// pass A / single pass, base = 256 + row for the rows of pass B.
#include "internal.h"
#include "launch.h"
#include "ntt_core.cuh"

namespace {

struct NttArgs {
    DevCtx c;
    LimbSet ls;   // destination (and source when has_src == 0)
    LimbSet src;  // source of the first pass when has_src != 0
    int has_src;
    int tiles;    // CTAs per limb
    // inverse only: final scaling of limb j is scale_tab[2 (scale_off + j)] (and
    // [.. + 1] for the folded twiddle) instead of N^-1, when not null
    const ulonglong2 *scale_tab;
    int scale_off;
};

// ---------------------------------------------------------------- N = 2^16
// Pass A: columns.  Tile = 16 adjacent columns c0..c0+15, all 256 rows.
// thread t: col = t & 15, u = t >> 4.
template <bool INV, int MINB>
__global__ void __launch_bounds__(256, MINB) k_ntt16_colpass(const __grid_constant__ NttArgs a) {
    __shared__ u64 sm[4096];
    const long long lid = blockIdx.x / a.tiles;
    const int c0 = (blockIdx.x % a.tiles) * 16;
    const LimbRef L = limb_of(a.ls, a.c.n, lid);
    u64 *__restrict__ g = L.ptr;
    const u64 q = a.c.q[L.prime];
    const int col = threadIdx.x & 15, u = threadIdx.x >> 4;
    u64 x[16];
    if (!INV) {
        const ulonglong2 *tw = a.c.tw_fwd + (size_t)L.prime * a.c.n;
        const u64 *__restrict__ gs = a.has_src ? limb_of(a.src, a.c.n, lid).ptr : g;
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = gs[((k << 4) | u) * 256 + c0 + col];
        fwd_round<8, 4>(x, u, tw, 1, q);
#pragma unroll
        for (int k = 0; k < 16; k++) sm[((k << 4) | u) * 16 + col] = x[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = sm[((u << 4) | k) * 16 + col];
        fwd_round<8, 0>(x, u << 4, tw, 1, q);
#pragma unroll
        for (int k = 0; k < 16; k++) g[((u << 4) | k) * 256 + c0 + col] = x[k];
    } else {
        const ulonglong2 *tw = a.c.tw_inv + (size_t)L.prime * a.c.n;
        const int sj = a.scale_off + (int)(lid % a.ls.nlimb);
        const ulonglong2 ni = a.scale_tab ? a.scale_tab[2 * sj] : a.c.ninv[L.prime];
        const ulonglong2 nw = a.scale_tab ? a.scale_tab[2 * sj + 1] : a.c.ninv_w1[L.prime];
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = g[((u << 4) | k) * 256 + c0 + col];
        inv_round<8, 0, false>(x, u << 4, tw, 1, q, ni, nw);
#pragma unroll
        for (int k = 0; k < 16; k++) sm[((u << 4) | k) * 16 + col] = x[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = sm[((k << 4) | u) * 16 + col];
        inv_round<8, 4, true>(x, u, tw, 1, q, ni, nw);
#pragma unroll
        for (int k = 0; k < 16; k++) g[((k << 4) | u) * 256 + c0 + col] = reduce2(x[k], q);
    }
}

// Pass B: rows.  Tile = 16 adjacent rows r0..r0+15 (256 contiguous words
// each).  thread t: u = t & 15, row = t >> 4.  Shared layout per row is
// padded (17 words per 16) so that both register assignments are free of
// bank conflicts.
template <bool INV, int MINB>
__global__ void __launch_bounds__(256, MINB) k_ntt16_rowpass(const __grid_constant__ NttArgs a) {
    __shared__ u64 sm[16 * 272];
    const long long lid = blockIdx.x / a.tiles;
    const int r0 = (blockIdx.x % a.tiles) * 16;
    const LimbRef L = limb_of(a.ls, a.c.n, lid);
    u64 *__restrict__ g = L.ptr + (size_t)r0 * 256;
    const u64 q = a.c.q[L.prime];
    const int u = threadIdx.x & 15, row = threadIdx.x >> 4;
    const int base = 256 + r0 + row;
    u64 *__restrict__ srow = sm + row * 272;
    u64 x[16];
    if (!INV) {
        const ulonglong2 *tw = a.c.tw_fwd + (size_t)L.prime * a.c.n;
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = g[row * 256 + ((k << 4) | u)];
        fwd_round<8, 4>(x, u, tw, base, q);
#pragma unroll
        for (int k = 0; k < 16; k++) srow[PADR((k << 4) | u)] = x[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = srow[PADR((u << 4) | k)];
        fwd_round<8, 0>(x, u << 4, tw, base, q);
#pragma unroll
        for (int k = 0; k < 16; k++) srow[PADR((u << 4) | k)] = reduce4(x[k], q);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const int e = threadIdx.x + 256 * i;
            const int r = e >> 8, p = e & 255;
            g[r * 256 + p] = sm[r * 272 + PADR(p)];
        }
    } else {
        const ulonglong2 *tw = a.c.tw_inv + (size_t)L.prime * a.c.n;
        const ulonglong2 ni = a.c.ninv[L.prime], nw = a.c.ninv_w1[L.prime];
        const u64 *__restrict__ gs = a.has_src ? limb_of(a.src, a.c.n, lid).ptr + (size_t)r0 * 256 : g;
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const int e = threadIdx.x + 256 * i;
            const int r = e >> 8, p = e & 255;
            sm[r * 272 + PADR(p)] = gs[r * 256 + p];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = srow[PADR((u << 4) | k)];
        inv_round<8, 0, false>(x, u << 4, tw, base, q, ni, nw);
#pragma unroll
        for (int k = 0; k < 16; k++) srow[PADR((u << 4) | k)] = x[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = srow[PADR((k << 4) | u)];
        inv_round<8, 4, false>(x, u, tw, base, q, ni, nw);
#pragma unroll
        for (int k = 0; k < 16; k++) g[row * 256 + ((k << 4) | u)] = x[k];
    }
}

// ---------------------------------------------------------------- N = 2^12
// One CTA per limb; thread t = u (8 bits); rounds on bits [8,12), [4,8), [0,4).
template <bool INV>
__global__ void __launch_bounds__(256) k_ntt12(const __grid_constant__ NttArgs a) {
    __shared__ u64 sm[4096 + 256];
    const LimbRef L = limb_of(a.ls, a.c.n, blockIdx.x);
    u64 *__restrict__ g = L.ptr;
    const u64 q = a.c.q[L.prime];
    const int u = threadIdx.x;
    const int p1 = ((u >> 4) << 8) | (u & 15);  // round-1 base point
    u64 x[16];
    if (!INV) {
        const ulonglong2 *tw = a.c.tw_fwd + (size_t)L.prime * a.c.n;
        const u64 *__restrict__ gs = a.has_src ? limb_of(a.src, a.c.n, blockIdx.x).ptr : g;
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = gs[(k << 8) | u];
        fwd_round<12, 8>(x, u, tw, 1, q);
#pragma unroll
        for (int k = 0; k < 16; k++) sm[PADR((k << 8) | u)] = x[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = sm[PADR(p1 | (k << 4))];
        fwd_round<12, 4>(x, p1, tw, 1, q);
#pragma unroll
        for (int k = 0; k < 16; k++) sm[PADR(p1 | (k << 4))] = x[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = sm[PADR((u << 4) | k)];
        fwd_round<12, 0>(x, u << 4, tw, 1, q);
#pragma unroll
        for (int k = 0; k < 16; k++) sm[PADR((u << 4) | k)] = reduce4(x[k], q);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const int e = threadIdx.x + 256 * i;
            g[e] = sm[PADR(e)];
        }
    } else {
        const ulonglong2 *tw = a.c.tw_inv + (size_t)L.prime * a.c.n;
        const ulonglong2 ni = a.c.ninv[L.prime], nw = a.c.ninv_w1[L.prime];
        const u64 *__restrict__ gs = a.has_src ? limb_of(a.src, a.c.n, blockIdx.x).ptr : g;
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const int e = threadIdx.x + 256 * i;
            sm[PADR(e)] = gs[e];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = sm[PADR((u << 4) | k)];
        inv_round<12, 0, false>(x, u << 4, tw, 1, q, ni, nw);
#pragma unroll
        for (int k = 0; k < 16; k++) sm[PADR((u << 4) | k)] = x[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = sm[PADR(p1 | (k << 4))];
        inv_round<12, 4, false>(x, p1, tw, 1, q, ni, nw);
#pragma unroll
        for (int k = 0; k < 16; k++) sm[PADR(p1 | (k << 4))] = x[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = sm[PADR((k << 8) | u)];
        inv_round<12, 8, true>(x, u, tw, 1, q, ni, nw);
#pragma unroll
        for (int k = 0; k < 16; k++) g[(k << 8) | u] = reduce2(x[k], q);
    }
}

// ------------------------------------------------------------ any N: slow
// One thread per butterfly of one radix-2 stage (m groups of size 2t).
__global__ void k_ntt_stage(const __grid_constant__ NttArgs a, int m, int t, int inverse,
                            long long total) {
    long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const int half = a.c.n >> 1;
    const long long lid = gid / half;
    const int b = (int)(gid % half);
    const LimbRef L = limb_of(a.ls, a.c.n, lid);
    const u64 q = a.c.q[L.prime];
    const int i = b / t;
    const int j = 2 * i * t + (b % t);
    u64 *g = L.ptr;
    if (!inverse) {
        const ulonglong2 w = a.c.tw_fwd[(size_t)L.prime * a.c.n + m + i];
        const u64 v = mul_shoup(g[j + t], w.x, w.y, q);
        const u64 uu = g[j];
        g[j] = add_mod(uu, v, q);
        g[j + t] = sub_mod(uu, v, q);
    } else {
        const ulonglong2 w = a.c.tw_inv[(size_t)L.prime * a.c.n + m + i];
        const u64 uu = g[j], v = g[j + t];
        g[j] = add_mod(uu, v, q);
        g[j + t] = mul_shoup(uu + q - v, w.x, w.y, q);
    }
}

__global__ void k_copy_limbs(const __grid_constant__ NttArgs a, long long total) {
    long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const long long lid = gid / a.c.n;
    const int e = (int)(gid % a.c.n);
    limb_of(a.ls, a.c.n, lid).ptr[e] = limb_of(a.src, a.c.n, lid).ptr[e];
}

__global__ void k_scale_ninv(const __grid_constant__ NttArgs a, long long total) {
    long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const long long lid = gid / a.c.n;
    const int e = (int)(gid % a.c.n);
    const LimbRef L = limb_of(a.ls, a.c.n, lid);
    const ulonglong2 ni = a.c.ninv[L.prime];
    L.ptr[e] = mul_shoup(L.ptr[e], ni.x, ni.y, a.c.q[L.prime]);
}

}  // namespace

// One N = 2^16 pass with the context's tuned launch configuration.
static int launch_pass16(secpe_ctx *ctx, int slot, const NttArgs &a, long long nl) {
    const unsigned grid = (unsigned)(nl * 16);
    const bool four = ctx->tune.ctas[slot] == 4;
    void (*kf)(NttArgs) = nullptr;
    const char *name = nullptr;
    switch (slot) {
        case TUNE_COLPASS:
            kf = four ? k_ntt16_colpass<false, 4> : k_ntt16_colpass<false, 3>;
            name = "k_ntt16_colpass<false>";
            break;
        case TUNE_ROWPASS:
            kf = four ? k_ntt16_rowpass<false, 4> : k_ntt16_rowpass<false, 3>;
            name = "k_ntt16_rowpass<false>";
            break;
        case TUNE_ICOLPASS:
            kf = four ? k_ntt16_colpass<true, 4> : k_ntt16_colpass<true, 3>;
            name = "k_ntt16_colpass<true>";
            break;
        case TUNE_IROWPASS:
            kf = four ? k_ntt16_rowpass<true, 4> : k_ntt16_rowpass<true, 3>;
            name = "k_ntt16_rowpass<true>";
            break;
        default: return SECPE_EINVAL;
    }
    SECPE_LAUNCH_AS(ctx, name, kf, grid, 256, 0, a);
    return SECPE_OK;
}

int ntt16_pass(secpe_ctx *ctx, int slot, const LimbSet &ls) {
    const long long nl = (long long)ls.nitem * ls.npoly * ls.nlimb;
    if (ctx->log_n != 16 || nl == 0 || nl * 16 >= (1ll << 31)) return SECPE_EINVAL;
    NttArgs a;
    a.c = ctx->dev;
    a.ls = ls;
    a.src = ls;
    a.has_src = 0;
    a.tiles = 16;
    a.scale_tab = nullptr;
    a.scale_off = 0;
    return launch_pass16(ctx, slot, a, nl);
}

int ntt_rowpass_only(secpe_ctx *ctx, const LimbSet &ls, bool inverse) {
    const long long nl = (long long)ls.nitem * ls.npoly * ls.nlimb;
    if (nl == 0) return SECPE_OK;
    if (ctx->log_n != 16 || ls.npoly * ls.nlimb > SECPE_MAX_LIMBSET) return SECPE_EINVAL;
    NttArgs a;
    a.c = ctx->dev;
    a.ls = ls;
    a.src = ls;
    a.has_src = 0;
    a.tiles = 16;
    a.scale_tab = nullptr;
    a.scale_off = 0;
    return launch_pass16(ctx, inverse ? TUNE_IROWPASS : TUNE_ROWPASS, a, nl);
}

LimbSet make_limbset(u64 *base, int nitem, long long item_stride, int npoly, long long poly_stride,
                     int nlimb, int prime0) {
    LimbSet ls;
    ls.base = base;
    ls.nitem = nitem;
    ls.item_stride = item_stride;
    ls.npoly = npoly;
    ls.poly_stride = poly_stride;
    ls.nlimb = nlimb;
    for (int p = 0; p < npoly; p++)
        for (int j = 0; j < nlimb; j++) {
            ls.prime_of[p * nlimb + j] = (int8_t)(prime0 + j);
            ls.aux[p * nlimb + j] = 0;
        }
    return ls;
}

int ntt_limbset(secpe_ctx *ctx, const LimbSet &ls, bool inverse, const LimbSet *src, const ulonglong2 *scale_tab,
                int scale_off, double alg_per_limb) {
    const long long nl = (long long)ls.nitem * ls.npoly * ls.nlimb;
    if (nl == 0) return SECPE_OK;
    if (ls.npoly * ls.nlimb > SECPE_MAX_LIMBSET) return SECPE_EINVAL;
    if (scale_tab && (!inverse || ctx->log_n != 16)) return SECPE_EINVAL;
    NttArgs a;
    a.c = ctx->dev;
    a.ls = ls;
    a.scale_tab = scale_tab;
    a.scale_off = scale_off;
    a.has_src = src ? 1 : 0;
    a.src = src ? *src : ls;
    if (ctx->tc_mode && ctx->log_n == 16) {
        // precision variant: both passes on the tensor pipe (no folded scalings)
        if (scale_tab) return SECPE_EINVAL;
        if (src) {
            a.tiles = 1;
            SECPE_LAUNCH(ctx, k_copy_limbs, grid1d(nl * ctx->n, 256), 256, 0, a, nl * ctx->n);
        }
        return ntt_limbset_tc(ctx, ls, inverse);
    }
    if (src && ctx->log_n != 16 && ctx->log_n != 12) {
        a.tiles = 1;
        SECPE_LAUNCH(ctx, k_copy_limbs, grid1d(nl * ctx->n, 256), 256, 0, a, nl * ctx->n);
        a.has_src = 0;
    }
    if (ctx->log_n == 16) {
        a.tiles = 16;
        if (nl * 16 >= (1ll << 31)) return SECPE_EINVAL;
        // each pass reads and writes every residue (model); the transform as
        // a whole is charged alg_per_limb, half to each pass
        const double model = 16.0 * ctx->n * nl;
        const double alg = 0.5 * (alg_per_limb < 0.0 ? 16.0 * ctx->n : alg_per_limb) * nl;
        const double mul = MUL32_PASS * ctx->n * nl;
        if (!inverse) {
            {
                KprofScope kp(ctx, "ntt16_colpass", alg, model, mul);
                SECPE_CHECK(launch_pass16(ctx, TUNE_COLPASS, a, nl));
            }
            KprofScope kp(ctx, "ntt16_rowpass", alg, model, mul);
            SECPE_CHECK(launch_pass16(ctx, TUNE_ROWPASS, a, nl));
        } else {
            {
                KprofScope kp(ctx, "intt16_rowpass", alg, model, mul);
                SECPE_CHECK(launch_pass16(ctx, TUNE_IROWPASS, a, nl));
            }
            KprofScope kp(ctx, "intt16_colpass", alg, model, mul + MUL32_INV_LAST * ctx->n * nl);
            SECPE_CHECK(launch_pass16(ctx, TUNE_ICOLPASS, a, nl));
        }
        return SECPE_OK;
    }
    if (ctx->log_n == 12) {
        a.tiles = 1;
        if (!inverse)
            SECPE_LAUNCH(ctx, k_ntt12<false>, (unsigned)nl, 256, 0, a);
        else
            SECPE_LAUNCH(ctx, k_ntt12<true>, (unsigned)nl, 256, 0, a);
        return SECPE_OK;
    }
    a.tiles = 1;
    const int n = ctx->n;
    const long long total = nl * (n / 2);
    if (!inverse) {
        int t = n;
        for (int m = 1; m < n; m <<= 1) {
            t >>= 1;
            SECPE_LAUNCH(ctx, k_ntt_stage, grid1d(total, 256), 256, 0, a, m, t, 0, total);
        }
    } else {
        int t = 1;
        for (int m = n >> 1; m >= 1; m >>= 1) {
            SECPE_LAUNCH(ctx, k_ntt_stage, grid1d(total, 256), 256, 0, a, m, t, 1, total);
            t <<= 1;
        }
        SECPE_LAUNCH(ctx, k_scale_ninv, grid1d(nl * n, 256), 256, 0, a, nl * n);
    }
    return SECPE_OK;
}
