// Precision variant: the N = 2^16 NTT / INTT and the key inner product of
// hybrid key switching as exact dense integer contractions on the tensor
// pipe (mma.sync u8 x u8 -> s32), bit-identical to the CUDA-core kernels.
//
// Transform.  Write a limb as a 256 x 256 array, a[r][c] = a[256 r + c].
// The negacyclic transform of the ring R_Q (Sec. 2.2),
//   out[j] = sum_k a[k] psi^((2 brv16(j) + 1) k),
// factors (four-step form, with brv16(256 r + t) = 256 brv8(t) + brv8(r)) into
//   1. columns: v[r][c] = sum_r' W[r][r'] a[r'][c],   W[r][r'] = psi^(256 (2 brv8(r) + 1) r'),
//   2. twist:   v[r][c] *= psi^((2 brv8(r) + 1) c),
//   3. rows:    out[256 r + t] = sum_c F[t][c] v[r][c],   F[t][c] = psi^(512 brv8(t) c).
// The inverse runs the rows with F*[c][t] = psi^(-512 brv8(t) c), the twist
// psi^(-(2 brv8(r) + 1) c), and the columns with V = 256^-1 W^-1 (the two
// together carry N^-1).  W and V are obtained by running the CUDA-core
// column network on unit vectors; F, F* and the twists are their closed
// forms.
//
// Every matrix product is exact: residues and matrix entries are split into
// 8-bit limbs, x = sum_b x_b 2^(8b); the 64 limb-pair products are 256^3 u8
// GEMMs with s32 accumulation; the 15 diagonal sums S_d = sum_{a+b=d} M_a X_b
// (< 8 * 256 * 255^2 < 2^31) are recombined as sum_d S_d 2^(8d) mod q with
// one Montgomery reduction; the twist is one more Montgomery product.
//
// Key inner product.  For target prime p, coefficient e and items b,
//   acc_s[b] = sum_j x_j[b] k_{j,s} mod p     (s = 0, 1; j over the digits),
// is a (2 x digits) by (digits x items) product per coefficient.  With 8-bit
// limbs it is one u8 GEMM per coefficient: row (s, d) of the left operand
// holds byte d - a of k_{j,s} at column (j, a) (a Toeplitz band built in
// registers from the key residue), column b of the right operand holds the
// bytes of x_j[b], so S[(s, d)][b] = sum_j sum_{a+a'=d} x_{j,a} k_{j,s,a'}
// is the d-th diagonal sum of the limb products (at most 8 limb pairs per
// digit and 8 digits: < 64 * 255^2 < 2^31).  The keys are stored in
// Montgomery form (k 2^64 mod p), so the recombination constants are the
// plain powers 2^(8d) mod p and the one Montgomery reduction also removes
// the key's factor 2^64.
//
// sm_103a has no tcgen05 kind::i8; the u8 mma.sync form is the integer
// tensor path the compiler accepts for this target.
#include <mutex>

#include "eval.h"
#include "ntt_core.cuh"

namespace {

enum { MAT_W = 0, MAT_V = 1, MAT_F = 2, MAT_FI = 3, NMAT = 4 };
constexpr size_t PLANES_PER_LIMB = 8ull * 65536ull;  // bytes of the 8 byte planes of one limb

struct TcArgs {
    DevCtx c;
    LimbSet ls;                  // limbs: read by the splits, written by the products
    const unsigned char *mats;   // [nprimes][NMAT][8][256][256] byte planes of M[out][in]
    const u64 *cmont;            // [nprimes][16] 2^(8d) 2^64 mod q (entry 15 = 0)
    const u64 *twist;            // [nprimes][2][65536] twist factors (forward, inverse), Montgomery form
    const unsigned char *xp;     // [nlimbs][8][256][256] byte planes of the limb data
    int mat;                     // matrix of this product
    int a_is_mat;                // 1: columns (A = matrix, B = transposed data); 0: rows (A = data, B = matrix)
    int twist_dir;               // -1: none; 0 / 1: multiply output (m, n) by twist[dir][256 m + n]
};

// Transposed byte planes: xp[l][b][c][r] = byte b of a[r][c] (the column
// product contracts over r, which must be the contiguous index).
__global__ void k_tc_split_t(const __grid_constant__ TcArgs a) {
    __shared__ u64 tile[32][33];
    const long long lid = blockIdx.z;
    const LimbRef L = limb_of(a.ls, a.c.n, lid);
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int i = ty; i < 32; i += 8) tile[i][tx] = L.ptr[(r0 + i) * 256 + c0 + tx];
    __syncthreads();
    unsigned char *dst = const_cast<unsigned char *>(a.xp) + lid * (long long)PLANES_PER_LIMB;
    for (int i = ty; i < 32; i += 8) {
        const u64 v = tile[tx][i];  // row r0 + tx, column c0 + i
        for (int b = 0; b < 8; b++)
            dst[(size_t)b * 65536 + (size_t)(c0 + i) * 256 + r0 + tx] = (unsigned char)(v >> (8 * b));
    }
}

// Byte planes in natural layout: xp[l][b][r][c] = byte b of a[r][c] (the
// row product contracts over c).  Each thread packs 4 adjacent residues.
__global__ void k_tc_split_n(const __grid_constant__ TcArgs a) {
    const long long lid = blockIdx.y;
    const LimbRef L = limb_of(a.ls, a.c.n, lid);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // group of 4 residues, < 16384
    const ulonglong2 v0 = ((const ulonglong2 *)L.ptr)[2 * i], v1 = ((const ulonglong2 *)L.ptr)[2 * i + 1];
    uint32_t *dst = (uint32_t *)(a.xp + lid * (long long)PLANES_PER_LIMB) + i;
#pragma unroll
    for (int b = 0; b < 8; b++) {
        const int s = 8 * b;
        dst[b * 16384] = (uint32_t)((v0.x >> s) & 0xff) | ((uint32_t)((v0.y >> s) & 0xff) << 8) |
                         ((uint32_t)((v1.x >> s) & 0xff) << 16) | ((uint32_t)((v1.y >> s) & 0xff) << 24);
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

// One 256 x 256 x 256 modular matrix product per limb, out[m][n] = sum_k
// A[m][k] B[n][k] mod q (times the twist), written to the limb.  CTA tile:
// 32 output rows x 64 columns.  All 8 byte planes of the 32 A rows and of
// the 64 B rows are staged in shared memory once (rows padded to 272 bytes,
// so that the fragment loads of a warp hit 32 distinct banks), and every
// limb pair is computed from there.  8 warps as 2 x 4, each 16 rows x 16
// columns (two m16n8 tiles); the diagonal sums S_d accumulate in the s32
// fragments.
constexpr int TC_BM = 32, TC_BN = 64, TC_PITCH = 272;
constexpr int TC_SMEM = 8 * (TC_BM + TC_BN) * TC_PITCH;  // 208,896 bytes

__global__ void __launch_bounds__(256, 1) k_tc_gemm(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(16) unsigned char tsm[];
    unsigned char *As = tsm;                         // [8][32][272]
    unsigned char *Bs = tsm + 8 * TC_BM * TC_PITCH;  // [8][64][272]
    const long long lid = blockIdx.z;
    const LimbRef L = limb_of(a.ls, a.c.n, lid);
    const int row0 = blockIdx.y * TC_BM, col0 = blockIdx.x * TC_BN;
    const unsigned char *M = a.mats + ((size_t)L.prime * NMAT + a.mat) * PLANES_PER_LIMB;
    const unsigned char *X = a.xp + lid * (long long)PLANES_PER_LIMB;
    const unsigned char *A = a.a_is_mat ? M : X;
    const unsigned char *B = a.a_is_mat ? X : M;
    for (int i = threadIdx.x; i < 8 * TC_BM * 16; i += 256) {
        const int pl = i / (TC_BM * 16), r = (i >> 4) % TC_BM, ch = i & 15;
        *(uint4 *)(As + (pl * TC_BM + r) * TC_PITCH + ch * 16) =
            __ldg((const uint4 *)(A + (size_t)pl * 65536 + (size_t)(row0 + r) * 256 + ch * 16));
    }
    for (int i = threadIdx.x; i < 8 * TC_BN * 16; i += 256) {
        const int pl = i / (TC_BN * 16), r = (i >> 4) % TC_BN, ch = i & 15;
        *(uint4 *)(Bs + (pl * TC_BN + r) * TC_PITCH + ch * 16) =
            __ldg((const uint4 *)(B + (size_t)pl * 65536 + (size_t)(col0 + r) * 256 + ch * 16));
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
            const unsigned char *Aa = As + (pa * TC_BM + wr) * TC_PITCH + 4 * t;
            const unsigned char *Bb = Bs + ((d - pa) * TC_BN + wc) * TC_PITCH + 4 * t;
#pragma unroll 4
            for (int kc = 0; kc < 256; kc += 32) {
                const uint32_t a0 = *(const uint32_t *)(Aa + g * TC_PITCH + kc);
                const uint32_t a1 = *(const uint32_t *)(Aa + (g + 8) * TC_PITCH + kc);
                const uint32_t a2 = *(const uint32_t *)(Aa + g * TC_PITCH + kc + 16);
                const uint32_t a3 = *(const uint32_t *)(Aa + (g + 8) * TC_PITCH + kc + 16);
#pragma unroll
                for (int nt = 0; nt < 2; nt++) {
                    const unsigned char *bb = Bb + (nt * 8 + g) * TC_PITCH + kc;
                    mma_u8(s[nt], a0, a1, a2, a3, *(const uint32_t *)bb, *(const uint32_t *)(bb + 16));
                }
            }
        }
        const u64 cd = a.cmont[(size_t)L.prime * 16 + d];
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) mac(acc[nt][e], (u64)(uint32_t)s[nt][e], cd);
    }
    const u64 *tw = a.twist_dir >= 0 ? a.twist + ((size_t)L.prime * 2 + a.twist_dir) * 65536 : nullptr;
    // fragment element e: row g (+8 for e >= 2), columns 2t, 2t+1
#pragma unroll
    for (int nt = 0; nt < 2; nt++)
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int r = row0 + wr + g + (e >> 1) * 8, cl = col0 + wc + nt * 8 + 2 * t + (e & 1);
            u64 v = redc(acc[nt][e].hi, acc[nt][e].lo, q, qinv);
            if (tw) v = mont_mul(v, tw[r * 256 + cl], q, qinv);
            L.ptr[r * 256 + cl] = v;
        }
}

// ------------------------------------------------------ key inner product
struct TcIpArgs {
    DevCtx c;
    const u64 *d;       // digit-own limbs: d + item*dis + t*N (NTT form)
    long long dis;
    const u64 *ext;     // extended limbs: ext + item*eis + (off_j + tt)*N (NTT form)
    long long eis;
    KsDigits dg;
    const u64 *key;     // [dnum][2][nprimes][N] Montgomery form
    u64 *acc;           // [nitem][2][nt][N]
    const u64 *cplain;  // [nprimes][16] 2^(8d) mod q (entry 15 = 0)
    int lv, nitem;
};

constexpr int TCIP_CPW = 8;  // coefficients per warp

// Residue of digit j's extension for target t, item `item`, coefficient e
// (0 when the digit or the item does not exist).
__device__ __forceinline__ u64 ip_x(const TcIpArgs &a, int j, int item, int t, int e) {
    if (j >= a.dg.ndig || item >= a.nitem) return 0;
    const int lo = a.dg.lo[j], hi = a.dg.hi[j];
    if (t >= lo && t < hi) return a.d[item * a.dis + (long long)t * a.c.n + e];
    const int tt = t < lo ? t : t - (hi - lo);
    return a.ext[item * a.eis + (long long)(a.dg.off[j] + tt) * a.c.n + e];
}

// Four bytes of k's Toeplitz band: byte i (i < 4) = byte u - i of k (0
// outside bytes 0..7), for -4 <= u <= 15.
__device__ __forceinline__ uint32_t band4(u64 k, int u) {
    const int sh = 8 * (u - 3);
    const u64 w = sh >= 64 ? 0ull : (sh >= 0 ? k >> sh : k << (-sh));
    return __byte_perm((uint32_t)w, 0u, 0x0123);
}

__device__ __forceinline__ void add128(acc128 &a, const acc128 &b) {
    const u64 lo = a.lo + b.lo;
    a.hi += b.hi + (lo < b.lo ? 1ull : 0ull);
    a.lo = lo;
}

// Block: target blockIdx.y, 8 warps x TCIP_CPW coefficients.  Per
// coefficient a warp builds the two m16 tiles of the key band (s = 0, 1;
// rows d = 0..15) for NKC chunks of 4 digits, then runs over the items in
// groups of 8 (the n8 columns).  Fragment element (row d, column b) of the
// s32 result is S[(s, d)][b]; the 16 diagonals of one (s, b) sit in the 8
// lanes of a quad column (d = g and g + 8) and are combined by shuffles.
template <int NKC>
__global__ void __launch_bounds__(256) k_tc_ksk_ip(const __grid_constant__ TcIpArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const int t = blockIdx.y, lv = a.lv, n = a.c.n;
    const int pt = t <= lv ? t : a.c.nq + (t - lv - 1);
    const int nt = lv + 1 + a.c.np_special;
    const u64 q = a.c.q[pt], qinv = a.c.qinv_neg[pt];
    const u64 cp_lo = a.cplain[pt * 16 + g], cp_hi = a.cplain[pt * 16 + g + 8];
    const long long kpoly = (long long)a.c.nprimes * n;
    const int a0 = 4 * (tq & 1);
    const int e0 = (blockIdx.x * 8 + warp) * TCIP_CPW;
    for (int e = e0; e < e0 + TCIP_CPW; e++) {
        uint32_t A[NKC][2][4];
#pragma unroll
        for (int kc = 0; kc < NKC; kc++) {
            const int jl = 4 * kc + (tq >> 1), jh = jl + 2;
#pragma unroll
            for (int s = 0; s < 2; s++) {
                const u64 kl = jl < a.dg.ndig ? a.key[jl * 2 * kpoly + s * kpoly + (long long)pt * n + e] : 0ull;
                const u64 kh = jh < a.dg.ndig ? a.key[jh * 2 * kpoly + s * kpoly + (long long)pt * n + e] : 0ull;
                A[kc][s][0] = band4(kl, g - a0);
                A[kc][s][1] = band4(kl, g + 8 - a0);
                A[kc][s][2] = band4(kh, g - a0);
                A[kc][s][3] = band4(kh, g + 8 - a0);
            }
        }
        for (int ig = 0; ig * 8 < a.nitem; ig++) {
            int S[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
#pragma unroll
            for (int kc = 0; kc < NKC; kc++) {
                const u64 xl = ip_x(a, 4 * kc + (tq >> 1), ig * 8 + g, t, e);
                const u64 xh = ip_x(a, 4 * kc + 2 + (tq >> 1), ig * 8 + g, t, e);
                const uint32_t b0 = (tq & 1) ? (uint32_t)(xl >> 32) : (uint32_t)xl;
                const uint32_t b1 = (tq & 1) ? (uint32_t)(xh >> 32) : (uint32_t)xh;
#pragma unroll
                for (int s = 0; s < 2; s++) mma_u8(S[s], A[kc][s][0], A[kc][s][1], A[kc][s][2], A[kc][s][3], b0, b1);
            }
            // (s, parity ip): columns 2 tq + ip; diagonals g and g + 8, summed over the 8 lanes of the quad column
            acc128 tot[2][2];
#pragma unroll
            for (int s = 0; s < 2; s++)
#pragma unroll
                for (int ip = 0; ip < 2; ip++) {
                    acc128 p = mul_full((u64)(uint32_t)S[s][ip], cp_lo);
                    mac(p, (u64)(uint32_t)S[s][2 + ip], cp_hi);
#pragma unroll
                    for (int off = 4; off < 32; off <<= 1) {
                        acc128 o;
                        o.lo = __shfl_xor_sync(0xffffffffu, p.lo, off);
                        o.hi = __shfl_xor_sync(0xffffffffu, p.hi, off);
                        add128(p, o);
                    }
                    tot[s][ip] = p;
                }
            if (g < 4) {
                const int s = g >> 1, ip = g & 1;
                const int item = ig * 8 + 2 * tq + ip;
                const acc128 v = s == 0 ? (ip == 0 ? tot[0][0] : tot[0][1]) : (ip == 0 ? tot[1][0] : tot[1][1]);
                if (item < a.nitem)
                    a.acc[(long long)item * 2 * nt * n + (long long)s * nt * n + (long long)t * n + e] =
                        redc(v.hi, v.lo, q, qinv);
            }
        }
    }
}

// ------------------------------------------------------------ host tables
std::mutex g_tc_mutex;

// exact column network on one 256-vector (the first 8 stages of the
// CUDA-core forward transform)
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

// the last 8 stages of the CUDA-core inverse transform, then N^-1
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

// 2^64 * v mod q
u64 to_mont(u64 v, u64 q) { return (u64)((((u128)v) << 64) % q); }

}  // namespace

struct TcTables {
    unsigned char *mats = nullptr;
    u64 *cmont = nullptr;
    u64 *cplain = nullptr;
    u64 *twist = nullptr;
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
    std::vector<unsigned char> mats((size_t)np * NMAT * PLANES_PER_LIMB);
    std::vector<u64> cm((size_t)np * 16, 0), cpl((size_t)np * 16, 0), tws((size_t)np * 2 * 65536);
    auto put = [&](int p, int mat, int out_i, int in_i, u64 v) {
        unsigned char *P = mats.data() + ((size_t)p * NMAT + mat) * PLANES_PER_LIMB;
        for (int b = 0; b < 8; b++) P[(size_t)b * 65536 + (size_t)out_i * 256 + in_i] = (unsigned char)(v >> (8 * b));
    };
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
        // W (forward columns) and V (inverse columns) from the network on unit vectors
        for (int k = 0; k < 256; k++) {
            std::vector<u64> e(256, 0), f(256, 0);
            e[k] = 1;
            f[k] = 1;
            col_fwd_host(e, q, twf);
            col_inv_host(f, q, twi, ninv);
            for (int j = 0; j < 256; j++) {
                put(p, MAT_W, j, k, e[j]);
                put(p, MAT_V, j, k, f[j]);
            }
        }
        // F[t][c] = omega^(brv8(t) c), F*[c][t] = omega^(-brv8(t) c), omega = psi^512
        const u64 om = hm::powmod(psi, 512, q), om_inv = hm::powmod(psi_inv, 512, q);
        for (int t = 0; t < 256; t++) {
            const uint32_t bt = hm::bitrev(t, 8);
            const u64 wf = hm::powmod(om, bt, q), wi = hm::powmod(om_inv, bt, q);
            u64 vf = 1, vi = 1;
            for (int c = 0; c < 256; c++) {
                put(p, MAT_F, t, c, vf);
                put(p, MAT_FI, c, t, vi);
                vf = hm::mulmod(vf, wf, q);
                vi = hm::mulmod(vi, wi, q);
            }
        }
        // twists psi^(+-(2 brv8(r) + 1) c) at (r, c), Montgomery form
        for (int r = 0; r < 256; r++) {
            const uint32_t er = 2 * hm::bitrev(r, 8) + 1;
            const u64 bf = hm::powmod(psi, er, q), bi = hm::powmod(psi_inv, er, q);
            u64 vf = 1, vi = 1;
            for (int c = 0; c < 256; c++) {
                tws[((size_t)p * 2 + 0) * 65536 + r * 256 + c] = to_mont(vf, q);
                tws[((size_t)p * 2 + 1) * 65536 + r * 256 + c] = to_mont(vi, q);
                vf = hm::mulmod(vf, bf, q);
                vi = hm::mulmod(vi, bi, q);
            }
        }
        for (int d = 0; d < 15; d++) {
            u64 v = 1 % q;
            for (int i = 0; i < d; i++) v = (u64)((((u128)v) << 8) % q);
            cpl[(size_t)p * 16 + d] = v;                // 2^(8d) mod q
            cm[(size_t)p * 16 + d] = to_mont(v, q);     // 2^(8d) 2^64 mod q
        }
    }
    TcTables t;
    const size_t cbytes = cm.size() * sizeof(u64), tbytes = tws.size() * sizeof(u64);
    void *m = nullptr, *c1 = nullptr, *c2 = nullptr, *tw = nullptr;
    if (cudaMalloc(&m, mats.size()) != cudaSuccess) return SECPE_ENOMEM;
    ctx->allocations.push_back(m);
    if (cudaMalloc(&c1, cbytes) != cudaSuccess) return SECPE_ENOMEM;
    ctx->allocations.push_back(c1);
    if (cudaMalloc(&c2, cbytes) != cudaSuccess) return SECPE_ENOMEM;
    ctx->allocations.push_back(c2);
    if (cudaMalloc(&tw, tbytes) != cudaSuccess) return SECPE_ENOMEM;
    ctx->allocations.push_back(tw);
    if (cudaMemcpy(m, mats.data(), mats.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c1, cm.data(), cbytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c2, cpl.data(), cbytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(tw, tws.data(), tbytes, cudaMemcpyHostToDevice) != cudaSuccess)
        return SECPE_ECUDA;
    t.mats = (unsigned char *)m;
    t.cmont = (u64 *)c1;
    t.cplain = (u64 *)c2;
    t.twist = (u64 *)tw;
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

static int tc_gemm_attr() {
    static bool attr_set[64];
    int dev = 0;
    SECPE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SECPE_ECUDA;
    if (!attr_set[dev]) {
        SECPE_CUDA(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
        attr_set[dev] = true;
    }
    return SECPE_OK;
}

// split the limbs of a.ls into byte planes (transposed or natural), then one
// modular matrix product per limb
static int tc_pass(secpe_ctx *ctx, TcArgs &a, long long nl, int mat, bool columns, int twist_dir) {
    if (columns)
        SECPE_LAUNCH(ctx, k_tc_split_t, dim3(8, 8, (unsigned)nl), dim3(32, 8), 0, a);
    else
        SECPE_LAUNCH(ctx, k_tc_split_n, dim3(64, (unsigned)nl), 256, 0, a);
    a.mat = mat;
    a.a_is_mat = columns ? 1 : 0;
    a.twist_dir = twist_dir;
    KprofScope kp(ctx, "tc_gemm", 16.0 * ctx->n * nl);
    SECPE_LAUNCH(ctx, k_tc_gemm, dim3(256 / TC_BN, 256 / TC_BM, (unsigned)nl), 256, TC_SMEM, a);
    return SECPE_OK;
}

// Full NTT / INTT of every limb of ls (in place) with both passes on the
// tensor pipe (N = 2^16 only).
int ntt_limbset_tc(secpe_ctx *ctx, const LimbSet &ls, bool inverse) {
    if (ctx->log_n != 16) return SECPE_EINVAL;
    const int per = ls.npoly * ls.nlimb;
    const long long nl = (long long)ls.nitem * per;
    if (nl == 0) return SECPE_OK;
    if (per <= 0 || per > SECPE_MAX_LIMBSET) return SECPE_EINVAL;
    TcTables tb;
    SECPE_CHECK(tc_tables(ctx, tb));
    SECPE_CHECK(tc_gemm_attr());
    // at most 2048 limbs (1 GiB of byte planes) per chunk of items
    const int chunk = std::max(1, 2048 / per);
    DevBuf xp;
    SECPE_CHECK(xp.alloc(ctx, (size_t)std::min<long long>(nl, (long long)chunk * per) * PLANES_PER_LIMB));
    TcArgs a;
    a.c = ctx->dev;
    a.mats = tb.mats;
    a.cmont = tb.cmont;
    a.twist = tb.twist;
    a.xp = (const unsigned char *)xp.p;
    for (int i0 = 0; i0 < ls.nitem; i0 += chunk) {
        a.ls = ls;
        a.ls.base = ls.base + (long long)i0 * ls.item_stride;
        a.ls.nitem = std::min(chunk, ls.nitem - i0);
        const long long snl = (long long)a.ls.nitem * per;
        if (!inverse) {
            SECPE_CHECK(tc_pass(ctx, a, snl, MAT_W, true, 0));    // columns, then the forward twist
            SECPE_CHECK(tc_pass(ctx, a, snl, MAT_F, false, -1));  // rows
        } else {
            SECPE_CHECK(tc_pass(ctx, a, snl, MAT_FI, false, 1));  // rows, then the inverse twist
            SECPE_CHECK(tc_pass(ctx, a, snl, MAT_V, true, -1));   // columns (with N^-1)
        }
    }
    return SECPE_OK;
}

// Key inner product on the tensor pipe: acc[item][s][t] = sum_j x_j k_{j,s}
// for every target t of Q_lv u P (canonical residues, the same values as
// the CUDA-core inner product).
int launch_ksk_ip_tc(secpe_ctx *ctx, const u64 *d, long long d_item_stride, const u64 *ext,
                     long long ext_item_stride, const KsDigits &dg, const u64 *key, u64 *acc, int B, int lv) {
    if (ctx->log_n != 16 || dg.ndig < 1 || dg.ndig > 8 || B < 1) return SECPE_EINVAL;
    TcTables tb;
    SECPE_CHECK(tc_tables(ctx, tb));
    TcIpArgs a;
    a.c = ctx->dev;
    a.d = d;
    a.dis = d_item_stride;
    a.ext = ext;
    a.eis = ext_item_stride;
    a.dg = dg;
    a.key = key;
    a.acc = acc;
    a.cplain = tb.cplain;
    a.lv = lv;
    a.nitem = B;
    const int nt = lv + 1 + ctx->npsp;
    const dim3 grid((unsigned)(ctx->n / (8 * TCIP_CPW)), (unsigned)nt);
    KprofScope kp(ctx, "tc_ksk_ip", 8.0 * ctx->n * ((double)B * dg.ndig * nt + 2.0 * dg.ndig * nt + 2.0 * B * nt));
    if (dg.ndig <= 4)
        SECPE_LAUNCH(ctx, k_tc_ksk_ip<1>, grid, 256, 0, a);
    else
        SECPE_LAUNCH(ctx, k_tc_ksk_ip<2>, grid, 256, 0, a);
    return SECPE_OK;
}
