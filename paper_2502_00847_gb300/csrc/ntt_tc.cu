// Precision variant of the N = 2^16 NTT: the column pass (the first 8
// stages of the forward transform, the last 8 of the inverse) as an exact
// dense integer contraction on the tensor pipe; the row pass stays on CUDA
// cores.  Results are bit-identical to ntt.cu.
//
// The column pass applies one fixed 256 x 256 matrix per prime to every
// column: W (forward) or V (inverse, including N^-1).  Both matrices are
// obtained on the host by running the exact column network on unit vectors,
// so they are the same linear map as the CUDA-core kernels.  Residues are
// split into 8-bit limbs, x = sum_b x_b 2^(8b), W = sum_a W_a 2^(8a); the
// products W_a X_b are computed with mma.sync m16n8k32 u8 x u8 -> s32 from
// operand tiles staged in shared memory, and
// the 15 diagonal sums S_d = sum_{a+b=d} W_a X_b (each < 8 * 256 * 255^2 <
// 2^31, exact in INT32) are recombined as sum_d S_d 2^(8d) mod q with one
// Montgomery reduction.  (sm_103a has no tcgen05 kind::i8; the u8 mma.sync
// form is the integer tensor path the compiler accepts for this target.)
#include <mutex>

#include "eval.h"
#include "ntt_core.cuh"

namespace {

struct TcArgs {
    DevCtx c;
    LimbSet ls;                  // limbs to transform
    const unsigned char *planes; // [nprimes][2][8][256][256] W (fwd), V (inv) byte planes
    const u64 *cmont;            // [nprimes][15]  2^(8d) * 2^64 mod q
    const unsigned char *xt;     // [nlimbs][8][256 (col)][256 (row)] byte planes of the input, transposed
    int inverse;
};

// Byte planes of each limb, transposed: xt[l][b][col][row] = byte b of x[row][col].
__global__ void k_tc_split(const __grid_constant__ TcArgs a) {
    __shared__ u64 tile[32][33];
    const long long lid = blockIdx.z;
    const LimbRef L = limb_of(a.ls, a.c.n, lid);
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int i = ty; i < 32; i += 8) tile[i][tx] = L.ptr[(r0 + i) * 256 + c0 + tx];
    __syncthreads();
    unsigned char *dst = const_cast<unsigned char *>(a.xt) + lid * 8ll * 65536;
    for (int i = ty; i < 32; i += 8) {
        const u64 v = tile[tx][i];  // row r0 + tx, col c0 + i
        for (int b = 0; b < 8; b++) dst[(size_t)b * 65536 + (size_t)(c0 + i) * 256 + r0 + tx] = (unsigned char)(v >> (8 * b));
    }
}

__device__ __forceinline__ void mma_u8(int (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                       uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// CTA tile: 32 output rows x 64 columns of one limb.  All 8 byte planes of
// the 32 matrix rows and of the 64 input columns are staged in shared memory
// once (rows padded to 272 bytes, so that the fragment loads of a warp hit 32
// distinct banks), and every limb pair (a, b) is computed from there: no
// operand is read from global memory twice by a CTA.  8 warps as 2 x 4, each
// 16 rows x 16 columns (two m16n8 tiles); the diagonal sums S_d accumulate
// in the s32 fragments (at most 8 * 256 * 255^2 < 2^31).  The legacy integer
// mma path of this part runs near 130 int8 TOPS here (about 16 us per limb),
// so the pass stays a precision variant, not a fast path.
constexpr int TC_BM = 32, TC_BN = 64, TC_PITCH = 272;
constexpr int TC_SMEM = 8 * (TC_BM + TC_BN) * TC_PITCH;  // 208,896 bytes

__global__ void __launch_bounds__(256, 1) k_tc_colpass(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(16) unsigned char tsm[];
    unsigned char *Ws = tsm;                         // [8][32][272]
    unsigned char *Xs = tsm + 8 * TC_BM * TC_PITCH;  // [8][64][272]
    const long long lid = blockIdx.z;
    const LimbRef L = limb_of(a.ls, a.c.n, lid);
    const int row0 = blockIdx.y * TC_BM, col0 = blockIdx.x * TC_BN;
    const unsigned char *W = a.planes + ((size_t)L.prime * 2 + (a.inverse ? 1 : 0)) * 8 * 65536;
    const unsigned char *X = a.xt + lid * 8ll * 65536;
    for (int i = threadIdx.x; i < 8 * TC_BM * 16; i += 256) {
        const int pl = i / (TC_BM * 16), r = (i >> 4) % TC_BM, ch = i & 15;
        *(uint4 *)(Ws + (pl * TC_BM + r) * TC_PITCH + ch * 16) =
            __ldg((const uint4 *)(W + (size_t)pl * 65536 + (size_t)(row0 + r) * 256 + ch * 16));
    }
    for (int i = threadIdx.x; i < 8 * TC_BN * 16; i += 256) {
        const int pl = i / (TC_BN * 16), r = (i >> 4) % TC_BN, ch = i & 15;
        *(uint4 *)(Xs + (pl * TC_BN + r) * TC_PITCH + ch * 16) =
            *(const uint4 *)(X + (size_t)pl * 65536 + (size_t)(col0 + r) * 256 + ch * 16);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int wr = (warp & 1) * 16, wc = (warp >> 1) * 16;
    const u64 q = a.c.q[L.prime], qinv = a.c.qinv_neg[L.prime];
    acc128 acc[2][4];
#pragma unroll
    for (int nt = 0; nt < 2; nt++)
#pragma unroll
        for (int e = 0; e < 4; e++) acc[nt][e] = {0, 0};
    for (int d = 0; d < 15; d++) {
        int s[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
        const int alo = d > 7 ? d - 7 : 0, ahi = d < 7 ? d : 7;
        for (int pa = alo; pa <= ahi; pa++) {
            const unsigned char *Wa = Ws + (pa * TC_BM + wr) * TC_PITCH + 4 * t;
            const unsigned char *Xb = Xs + ((d - pa) * TC_BN + wc) * TC_PITCH + 4 * t;
#pragma unroll 4
            for (int kc = 0; kc < 256; kc += 32) {
                const uint32_t a0 = *(const uint32_t *)(Wa + g * TC_PITCH + kc);
                const uint32_t a1 = *(const uint32_t *)(Wa + (g + 8) * TC_PITCH + kc);
                const uint32_t a2 = *(const uint32_t *)(Wa + g * TC_PITCH + kc + 16);
                const uint32_t a3 = *(const uint32_t *)(Wa + (g + 8) * TC_PITCH + kc + 16);
#pragma unroll
                for (int nt = 0; nt < 2; nt++) {
                    const unsigned char *xb = Xb + (nt * 8 + g) * TC_PITCH + kc;
                    mma_u8(s[nt], a0, a1, a2, a3, *(const uint32_t *)xb, *(const uint32_t *)(xb + 16));
                }
            }
        }
        const u64 cd = a.cmont[(size_t)L.prime * 15 + d];
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) mac(acc[nt][e], (u64)(uint32_t)s[nt][e], cd);
    }
    // fragment element e: row g (+8 for e >= 2), columns 2t, 2t+1
#pragma unroll
    for (int nt = 0; nt < 2; nt++)
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int r = row0 + wr + g + (e >> 1) * 8, cl = col0 + wc + nt * 8 + 2 * t + (e & 1);
            L.ptr[r * 256 + cl] = redc(acc[nt][e].hi, acc[nt][e].lo, q, qinv);
        }
}

// ------------------------------------------------------------ host tables
std::mutex g_tc_mutex;

// exact column network on one 256-vector (mirrors k_ntt16_colpass)
void col_fwd_host(std::vector<u64> &x, u64 q, const std::vector<u64> &tw) {
    int t = 256;
    for (int m = 1; m < 256; m <<= 1) {
        t >>= 1;
        for (int i = 0; i < m; i++) {
            const u64 w = tw[m + i];
            for (int j = 2 * i * t; j < 2 * i * t + t; j++) {
                const u64 u = x[j], v = hm::mulmod(x[j + t], w, q);
                x[j] = (u + v) % q;
                x[j + t] = (u + q - v) % q;
            }
        }
    }
}

void col_inv_host(std::vector<u64> &x, u64 q, const std::vector<u64> &tw, u64 ninv) {
    int t = 1;
    for (int m = 128; m >= 1; m >>= 1) {
        for (int i = 0; i < m; i++) {
            const u64 w = tw[m + i];
            for (int j = 2 * i * t; j < 2 * i * t + t; j++) {
                const u64 u = x[j], v = x[j + t];
                x[j] = (u + v) % q;
                x[j + t] = hm::mulmod((u + q - v) % q, w, q);
            }
        }
        t <<= 1;
    }
    for (auto &v : x) v = hm::mulmod(v, ninv, q);
}

}  // namespace

struct TcTables {
    unsigned char *planes = nullptr;
    u64 *cmont = nullptr;
};

static std::vector<std::pair<const secpe_ctx *, TcTables>> g_tc_tables;

static int tc_tables(secpe_ctx *ctx, TcTables &out) {
    std::lock_guard<std::mutex> lock(g_tc_mutex);
    for (auto &p : g_tc_tables)
        if (p.first == ctx) {
            out = p.second;
            return SECPE_OK;
        }
    const int np = ctx->nprimes, n = ctx->n;
    std::vector<unsigned char> planes((size_t)np * 2 * 8 * 65536);
    std::vector<u64> cm((size_t)np * 15);
    for (int p = 0; p < np; p++) {
        const u64 q = ctx->primes[p], psi = ctx->psi[p];
        const u64 psi_inv = hm::invmod(psi, q);
        std::vector<u64> twf(256), twi(256);
        for (int i = 1; i < 256; i++) {
            const uint32_t b = hm::bitrev(i, ctx->log_n);
            twf[i] = hm::powmod(psi, b, q);
            twi[i] = hm::powmod(psi_inv, b, q);
        }
        const u64 ninv = hm::invmod((u64)n, q);
        for (int dir = 0; dir < 2; dir++) {
            unsigned char *P = planes.data() + ((size_t)p * 2 + dir) * 8 * 65536;
            for (int k = 0; k < 256; k++) {
                std::vector<u64> e(256, 0);
                e[k] = 1;
                if (dir == 0) col_fwd_host(e, q, twf);
                else col_inv_host(e, q, twi, ninv);
                for (int j = 0; j < 256; j++)
                    for (int b = 0; b < 8; b++) P[(size_t)b * 65536 + (size_t)j * 256 + k] = (unsigned char)(e[j] >> (8 * b));
            }
        }
        for (int d = 0; d < 15; d++) {
            // 2^(8d) * 2^64 mod q
            u128 v = ((u128)1) << 64;
            for (int i = 0; i < d; i++) v = (v << 8) % q;
            cm[(size_t)p * 15 + d] = (u64)(v % q);
        }
    }
    TcTables t;
    if (cudaMalloc(&t.planes, planes.size()) != cudaSuccess) return SECPE_ENOMEM;
    if (cudaMalloc(&t.cmont, cm.size() * sizeof(u64)) != cudaSuccess) {
        cudaFree(t.planes);
        return SECPE_ENOMEM;
    }
    if (cudaMemcpy(t.planes, planes.data(), planes.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t.cmont, cm.data(), cm.size() * sizeof(u64), cudaMemcpyHostToDevice) != cudaSuccess)
        return SECPE_ECUDA;
    ctx->allocations.push_back(t.planes);
    ctx->allocations.push_back(t.cmont);
    g_tc_tables.push_back({ctx, t});
    out = t;
    return SECPE_OK;
}

void tc_forget_ctx(const secpe_ctx *ctx) {
    std::lock_guard<std::mutex> lock(g_tc_mutex);
    for (size_t i = 0; i < g_tc_tables.size(); i++)
        if (g_tc_tables[i].first == ctx) {
            g_tc_tables.erase(g_tc_tables.begin() + i);
            return;
        }
}

// Column pass on the tensor pipe for every limb of ls (in place).
static int tc_colpass(secpe_ctx *ctx, const LimbSet &ls, bool inverse, const TcTables &tb) {
    const long long nl = (long long)ls.nitem * ls.npoly * ls.nlimb;
    if (nl == 0) return SECPE_OK;
    if (nl > 65535) return SECPE_EINVAL;
    DevBuf xt;
    SECPE_CHECK(xt.alloc(ctx, (size_t)nl * 8 * 65536));
    TcArgs a;
    a.c = ctx->dev;
    a.ls = ls;
    a.planes = tb.planes;
    a.cmont = tb.cmont;
    a.xt = (const unsigned char *)xt.p;
    a.inverse = inverse ? 1 : 0;
    SECPE_LAUNCH(ctx, k_tc_split, dim3(8, 8, (unsigned)nl), dim3(32, 8), 0, a);
    KprofScope kp(ctx, "tc_colpass", 16.0 * ctx->n * nl);
    static bool attr_set[64];
    int dev = 0;
    SECPE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SECPE_ECUDA;
    if (!attr_set[dev]) {
        SECPE_CUDA(cudaFuncSetAttribute(k_tc_colpass, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
        attr_set[dev] = true;
    }
    SECPE_LAUNCH(ctx, k_tc_colpass, dim3(256 / TC_BN, 256 / TC_BM, (unsigned)nl), 256, TC_SMEM, a);
    return SECPE_OK;
}

// Full NTT / INTT with the tensor-pipe column pass (N = 2^16 only).
int ntt_limbset_tc(secpe_ctx *ctx, const LimbSet &ls, bool inverse) {
    if (ctx->log_n != 16) return SECPE_EINVAL;
    TcTables tb;
    SECPE_CHECK(tc_tables(ctx, tb));
    if (!inverse) {
        SECPE_CHECK(tc_colpass(ctx, ls, false, tb));
        return ntt_rowpass_only(ctx, ls, false);
    }
    SECPE_CHECK(ntt_rowpass_only(ctx, ls, true));
    return tc_colpass(ctx, ls, true, tb);
}
