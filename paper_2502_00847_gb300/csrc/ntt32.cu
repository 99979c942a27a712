// Word-size probe: the negacyclic NTT and the fast base conversion on 32-bit
// residues (NTT-friendly primes q < 2^30), N = 2^16.
//
// The transform is the network of the 64-bit one (ntt.cu): forward
// Cooley-Tukey, natural order in and bit-reversed order out, twiddle
// psi^brv(m + i) for group i of the stage with m groups; inverse
// Gentleman-Sande with psi^-brv(m + i), N^-1 folded into its last stage.
// Two passes of 8 stages (columns, then rows; rows first for the inverse),
// 256 threads and 16 residues per thread, D. Harvey's lazy butterflies: the
// forward values stay in [0, 4q), the inverse ones in [0, 2q), both below
// 2^32 for q < 2^30.  A product by a fixed twiddle w is V. Shoup's: with
// w' = floor(w 2^32 / q), x w - floor(x w' / 2^32) q lies in [0, 2q) for any
// 32-bit x: one high and two low 32-bit multiplies, against 15 for a 64-bit
// residue of a prime up to 2^60.
//
// FastBConv (the base conversion of ModUp and ModDown), per coefficient:
// y_i = [x_i Qhat_i^-1]_{q_i}, out_j = sum_i y_i [Qhat_i]_{p_j} mod p_j,
// the products (< 2^60) summed exactly in 64 bits (at most 16 inputs) and
// reduced once.
#include <algorithm>
#include <vector>

#include "internal.h"
#include "launch.h"

#define PAD17(p) ((p) + ((p) >> 4))  // 17 shared words per 16

struct secpe_ntt32_table {
    int log_n = 0, n = 0, np = 0;
    std::vector<uint32_t> q;
    uint32_t *d_q = nullptr;
    uint2 *d_twf = nullptr, *d_twi = nullptr;      // [np][N]: (w, w')
    uint2 *d_ninv = nullptr, *d_ninvw1 = nullptr;  // [np]
};

namespace {

constexpr int kMaxLimbs32 = 256;   // limbs per launch
constexpr int kMaxIn32 = 16;       // FastBConv inputs
constexpr int kMaxOut32 = 64;      // FastBConv outputs

__device__ __forceinline__ uint32_t shoup32(uint32_t x, uint32_t w, uint32_t wp, uint32_t q) {
    return x * w - __umulhi(x, wp) * q;  // [0, 2q)
}
__device__ __forceinline__ uint32_t red2_32(uint32_t v, uint32_t q) { return v >= q ? v - q : v; }
__device__ __forceinline__ uint32_t red4_32(uint32_t v, uint32_t q) {
    v = v >= 2 * q ? v - 2 * q : v;
    return v >= q ? v - q : v;
}

// Radix-16 rounds on 16 registers: stage bits [LO, LO + 4) of a 2^LOGP-point
// pass; p0 holds the bits of the register's point outside the window.
template <int LOGP, int LO>
__device__ __forceinline__ void fwd16(uint32_t (&x)[16], int p0, const uint2 *__restrict__ tw, int base,
                                      uint32_t q) {
    const uint32_t q2 = 2 * q;
#pragma unroll
    for (int sb = 3; sb >= 0; --sb) {
        const int s = LO + sb;
        const int st = LOGP - 1 - s;
        const int ibase = (base << st) + (p0 >> (s + 1));
        uint2 w[8];
#pragma unroll
        for (int g = 0; g < 8; ++g)
            if (g < (8 >> sb)) w[g] = tw[ibase + g];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (k & (1 << sb)) continue;
            const uint2 ww = w[k >> (sb + 1)];
            uint32_t u = x[k];
            u = u >= q2 ? u - q2 : u;
            const uint32_t t = shoup32(x[k | (1 << sb)], ww.x, ww.y, q);
            x[k] = u + t;
            x[k | (1 << sb)] = u - t + q2;
        }
    }
}

template <int LOGP, int LO, bool LAST>
__device__ __forceinline__ void inv16(uint32_t (&x)[16], int p0, const uint2 *__restrict__ tw, int base, uint32_t q,
                                      uint2 ninv, uint2 ninv_w1) {
    const uint32_t q2 = 2 * q;
#pragma unroll
    for (int sb = 0; sb < 4; ++sb) {
        const int s = LO + sb;
        const int st = LOGP - 1 - s;
        const bool last = LAST && s == LOGP - 1;
        const int ibase = (base << st) + (p0 >> (s + 1));
        uint2 w[8];
#pragma unroll
        for (int g = 0; g < 8; ++g)
            if (g < (8 >> sb)) w[g] = last ? ninv_w1 : tw[ibase + g];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (k & (1 << sb)) continue;
            const uint2 ww = w[k >> (sb + 1)];
            const uint32_t u = x[k], v = x[k | (1 << sb)];
            if (last) {
                x[k] = shoup32(u + v, ninv.x, ninv.y, q);
            } else {
                const uint32_t sum = u + v;
                x[k] = sum >= q2 ? sum - q2 : sum;
            }
            x[k | (1 << sb)] = shoup32(u - v + q2, ww.x, ww.y, q);
        }
    }
}

struct Ntt32Args {
    uint32_t *data;  // limb i of the launch at data + i N
    const uint32_t *q;
    const uint2 *tw;  // [np][N], forward or inverse
    const uint2 *ninv, *ninvw1;
    uint8_t prime_of[kMaxLimbs32];
};

// Column-pass shared layout: row r of the 16-column tile at 16 words, rows
// r and r ^ 1 swapped when bit 4 of r is set, so that both register
// assignments touch 32 distinct banks per warp.
__device__ __forceinline__ int col_sm(int r, int col) { return ((r ^ ((r >> 4) & 1)) << 4) | col; }

// Pass A: 16 adjacent columns (stride-256 elements), all 256 rows.
template <bool INV>
__global__ void __launch_bounds__(256) k_ntt32_colpass(const __grid_constant__ Ntt32Args a) {
    __shared__ uint32_t sm[4096];
    const int lid = blockIdx.x >> 4, c0 = (blockIdx.x & 15) * 16;
    const int pi = a.prime_of[lid];
    uint32_t *__restrict__ g = a.data + (size_t)lid * 65536;
    const uint32_t q = a.q[pi];
    const uint2 *tw = a.tw + (size_t)pi * 65536;
    const int col = threadIdx.x & 15, u = threadIdx.x >> 4;
    uint32_t x[16];
    if (!INV) {
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = g[((k << 4) | u) * 256 + c0 + col];
        fwd16<8, 4>(x, u, tw, 1, q);
#pragma unroll
        for (int k = 0; k < 16; k++) sm[col_sm((k << 4) | u, col)] = x[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = sm[col_sm((u << 4) | k, col)];
        fwd16<8, 0>(x, u << 4, tw, 1, q);
#pragma unroll
        for (int k = 0; k < 16; k++) g[((u << 4) | k) * 256 + c0 + col] = x[k];
    } else {
        const uint2 ni = a.ninv[pi], nw = a.ninvw1[pi];
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = g[((u << 4) | k) * 256 + c0 + col];
        inv16<8, 0, false>(x, u << 4, tw, 1, q, ni, nw);
#pragma unroll
        for (int k = 0; k < 16; k++) sm[col_sm((u << 4) | k, col)] = x[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = sm[col_sm((k << 4) | u, col)];
        inv16<8, 4, true>(x, u, tw, 1, q, ni, nw);
#pragma unroll
        for (int k = 0; k < 16; k++) g[((k << 4) | u) * 256 + c0 + col] = red2_32(x[k], q);
    }
}

// Pass B: 16 adjacent rows of 256 contiguous words; per-row shared layout
// padded to 17 words per 16.
template <bool INV>
__global__ void __launch_bounds__(256) k_ntt32_rowpass(const __grid_constant__ Ntt32Args a) {
    __shared__ uint32_t sm[16 * 272];
    const int lid = blockIdx.x >> 4, r0 = (blockIdx.x & 15) * 16;
    const int pi = a.prime_of[lid];
    uint32_t *__restrict__ g = a.data + (size_t)lid * 65536 + (size_t)r0 * 256;
    const uint32_t q = a.q[pi];
    const uint2 *tw = a.tw + (size_t)pi * 65536;
    const int u = threadIdx.x & 15, row = threadIdx.x >> 4;
    const int base = 256 + r0 + row;
    uint32_t *__restrict__ srow = sm + row * 272;
    uint32_t x[16];
    if (!INV) {
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = g[row * 256 + ((k << 4) | u)];
        fwd16<8, 4>(x, u, tw, base, q);
#pragma unroll
        for (int k = 0; k < 16; k++) srow[PAD17((k << 4) | u)] = x[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = srow[PAD17((u << 4) | k)];
        fwd16<8, 0>(x, u << 4, tw, base, q);
#pragma unroll
        for (int k = 0; k < 16; k++) srow[PAD17((u << 4) | k)] = red4_32(x[k], q);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const int e = threadIdx.x + 256 * i;
            const int r = e >> 8, p = e & 255;
            g[r * 256 + p] = sm[r * 272 + PAD17(p)];
        }
    } else {
        const uint2 ni = a.ninv[pi], nw = a.ninvw1[pi];
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const int e = threadIdx.x + 256 * i;
            const int r = e >> 8, p = e & 255;
            sm[r * 272 + PAD17(p)] = g[r * 256 + p];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = srow[PAD17((u << 4) | k)];
        inv16<8, 0, false>(x, u << 4, tw, base, q, ni, nw);
#pragma unroll
        for (int k = 0; k < 16; k++) srow[PAD17((u << 4) | k)] = x[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = srow[PAD17((k << 4) | u)];
        inv16<8, 4, false>(x, u, tw, base, q, ni, nw);
#pragma unroll
        for (int k = 0; k < 16; k++) g[row * 256 + ((k << 4) | u)] = x[k];
    }
}

struct BConv32Args {
    const uint32_t *in;  // [batch][n_in][N]
    uint32_t *out;       // [batch][n_out][N]
    int n_in, n_out;
    uint32_t qin[kMaxIn32];
    uint2 qhinv[kMaxIn32];            // ([Qhat_i^-1]_{q_i}, Shoup companion)
    uint32_t M[kMaxIn32][kMaxOut32];  // [Qhat_i]_{p_j}
    uint32_t p[kMaxOut32];
    uint2 r32[kMaxOut32];             // (2^32 mod p_j, Shoup companion)
    uint32_t m32[kMaxOut32];          // floor(2^32 / p_j)
};

// Four adjacent coefficients of one item per thread (grid: N/1024 x batch):
// 16-byte loads and stores, and each constant [Qhat_i]_{p_j}, staged in
// shared memory, serves four products.
__global__ void __launch_bounds__(256) k_bconv32(const __grid_constant__ BConv32Args a) {
    __shared__ uint32_t Ms[kMaxIn32 * kMaxOut32];
    for (int e = threadIdx.x; e < a.n_in * a.n_out; e += 256) Ms[e] = a.M[e / a.n_out][e % a.n_out];
    __syncthreads();
    const int c = (blockIdx.x * 256 + threadIdx.x) * 4;
    const size_t item = blockIdx.y;
    const uint32_t *__restrict__ in = a.in + item * a.n_in * 65536 + c;
    uint32_t *__restrict__ out = a.out + item * a.n_out * 65536 + c;
    uint32_t y[kMaxIn32][4];
#pragma unroll
    for (int i = 0; i < kMaxIn32; i++) {
        if (i >= a.n_in) break;
        const uint4 v = *reinterpret_cast<const uint4 *>(in + (size_t)i * 65536);
        const uint32_t qi = a.qin[i], w = a.qhinv[i].x, wp = a.qhinv[i].y;
        y[i][0] = red2_32(shoup32(v.x, w, wp, qi), qi);
        y[i][1] = red2_32(shoup32(v.y, w, wp, qi), qi);
        y[i][2] = red2_32(shoup32(v.z, w, wp, qi), qi);
        y[i][3] = red2_32(shoup32(v.w, w, wp, qi), qi);
    }
    for (int j = 0; j < a.n_out; j++) {
        unsigned long long acc[4] = {0, 0, 0, 0};
#pragma unroll
        for (int i = 0; i < kMaxIn32; i++) {
            if (i >= a.n_in) break;
            const unsigned long long m = Ms[i * a.n_out + j];
#pragma unroll
            for (int b = 0; b < 4; b++) acc[b] += y[i][b] * m;
        }
        const uint32_t p = a.p[j], rw = a.r32[j].x, rwp = a.r32[j].y, m32 = a.m32[j];
        uint32_t r[4];
#pragma unroll
        for (int b = 0; b < 4; b++) {
            // acc = hi 2^32 + lo: [hi 2^32]_p by Shoup (in [0, 2p)), lo - floor(lo m / 2^32) p in [0, 2p)
            const uint32_t hi = (uint32_t)(acc[b] >> 32), lo = (uint32_t)acc[b];
            r[b] = red4_32(shoup32(hi, rw, rwp, p) + (lo - __umulhi(lo, m32) * p), p);
        }
        *reinterpret_cast<uint4 *>(out + (size_t)j * 65536) = make_uint4(r[0], r[1], r[2], r[3]);
    }
}

uint32_t shoup32_host(uint32_t w, uint32_t q) { return (uint32_t)(((u64)w << 32) / q); }

int check_limbs(const secpe_ntt32_table *t, const void *p, const int32_t *idx, int count) {
    if (!t || !p || !idx || count < 0 || !aligned16(p)) return SECPE_EINVAL;
    for (int i = 0; i < count; i++)
        if (idx[i] < 0 || idx[i] >= t->np) return SECPE_EINVAL;
    return SECPE_OK;
}

}  // namespace

extern "C" int secpe_ntt32_create(int log_n, const uint32_t *primes, int n_primes, secpe_ntt32_table **out) {
    if (log_n != 16 || !primes || n_primes < 1 || n_primes > 128 || !out) return SECPE_EINVAL;
    const int n = 1 << log_n;
    for (int t = 0; t < n_primes; t++) {
        const uint32_t q = primes[t];
        if (q >= (1u << 30) || q < 3 || (q - 1) % (2u * n) != 0 || !hm::is_prime(q)) return SECPE_EINVAL;
    }
    secpe_ntt32_table *t = new secpe_ntt32_table;
    t->log_n = log_n;
    t->n = n;
    t->np = n_primes;
    t->q.assign(primes, primes + n_primes);
    std::vector<uint2> twf((size_t)n_primes * n), twi((size_t)n_primes * n), ni(n_primes), niw(n_primes);
    for (int s = 0; s < n_primes; s++) {
        const u64 q = primes[s];
        const u64 psi = hm::find_psi(q, n), psi_inv = hm::invmod(psi, q);
        std::vector<u64> pw(n), ipw(n);
        pw[0] = ipw[0] = 1;
        for (int i = 1; i < n; i++) {
            pw[i] = hm::mulmod(pw[i - 1], psi, q);
            ipw[i] = hm::mulmod(ipw[i - 1], psi_inv, q);
        }
        for (int i = 0; i < n; i++) {
            const uint32_t b = hm::bitrev(i, log_n);
            twf[(size_t)s * n + i] = make_uint2((uint32_t)pw[b], shoup32_host((uint32_t)pw[b], (uint32_t)q));
            twi[(size_t)s * n + i] = make_uint2((uint32_t)ipw[b], shoup32_host((uint32_t)ipw[b], (uint32_t)q));
        }
        const u64 nv = hm::invmod((u64)n, q), nw1 = hm::mulmod(nv, ipw[hm::bitrev(1, log_n)], q);
        ni[s] = make_uint2((uint32_t)nv, shoup32_host((uint32_t)nv, (uint32_t)q));
        niw[s] = make_uint2((uint32_t)nw1, shoup32_host((uint32_t)nw1, (uint32_t)q));
    }
    bool ok = cudaMalloc(&t->d_q, 4 * (size_t)n_primes) == cudaSuccess &&
              cudaMalloc(&t->d_twf, sizeof(uint2) * twf.size()) == cudaSuccess &&
              cudaMalloc(&t->d_twi, sizeof(uint2) * twi.size()) == cudaSuccess &&
              cudaMalloc(&t->d_ninv, sizeof(uint2) * n_primes) == cudaSuccess &&
              cudaMalloc(&t->d_ninvw1, sizeof(uint2) * n_primes) == cudaSuccess;
    ok = ok && cudaMemcpy(t->d_q, primes, 4 * (size_t)n_primes, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(t->d_twf, twf.data(), sizeof(uint2) * twf.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(t->d_twi, twi.data(), sizeof(uint2) * twi.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(t->d_ninv, ni.data(), sizeof(uint2) * n_primes, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(t->d_ninvw1, niw.data(), sizeof(uint2) * n_primes, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        secpe_ntt32_destroy(t);
        return SECPE_ECUDA;
    }
    *out = t;
    return SECPE_OK;
}

extern "C" void secpe_ntt32_destroy(secpe_ntt32_table *t) {
    if (!t) return;
    cudaFree(t->d_q);
    cudaFree(t->d_twf);
    cudaFree(t->d_twi);
    cudaFree(t->d_ninv);
    cudaFree(t->d_ninvw1);
    delete t;
}

extern "C" int secpe_ntt32(const secpe_ntt32_table *t, uint32_t *limbs, const int32_t *prime_idx, int count, int inverse,
                           void *stream) {
    SECPE_CHECK(check_limbs(t, limbs, prime_idx, count));
    cudaStream_t s = (cudaStream_t)stream;
    for (int c0 = 0; c0 < count; c0 += kMaxLimbs32) {
        const int nl = std::min(kMaxLimbs32, count - c0);
        Ntt32Args a;
        a.data = limbs + (size_t)c0 * t->n;
        a.q = t->d_q;
        a.tw = inverse ? t->d_twi : t->d_twf;
        a.ninv = t->d_ninv;
        a.ninvw1 = t->d_ninvw1;
        for (int i = 0; i < nl; i++) a.prime_of[i] = (uint8_t)prime_idx[c0 + i];
        if (!inverse) {
            k_ntt32_colpass<false><<<nl * 16, 256, 0, s>>>(a);
            k_ntt32_rowpass<false><<<nl * 16, 256, 0, s>>>(a);
        } else {
            k_ntt32_rowpass<true><<<nl * 16, 256, 0, s>>>(a);
            k_ntt32_colpass<true><<<nl * 16, 256, 0, s>>>(a);
        }
    }
    return cudaGetLastError() == cudaSuccess ? SECPE_OK : SECPE_ECUDA;
}

extern "C" int secpe_bconv32(const secpe_ntt32_table *t, const uint32_t *in, const int32_t *in_idx, int n_in,
                             uint32_t *out, const int32_t *out_idx, int n_out, int batch, void *stream) {
    SECPE_CHECK(check_limbs(t, in, in_idx, n_in));
    SECPE_CHECK(check_limbs(t, out, out_idx, n_out));
    if (n_in < 1 || n_in > kMaxIn32 || n_out < 1 || n_out > kMaxOut32 || batch < 1 || batch > 65535)
        return SECPE_EINVAL;
    for (int i = 0; i < n_in; i++)
        for (int k = 0; k < i; k++)
            if (in_idx[i] == in_idx[k]) return SECPE_EINVAL;
    BConv32Args a;
    a.in = in;
    a.out = out;
    a.n_in = n_in;
    a.n_out = n_out;
    for (int i = 0; i < n_in; i++) {
        const u64 qi = t->q[in_idx[i]];
        u64 qhat = 1;  // Q / q_i mod q_i
        for (int k = 0; k < n_in; k++)
            if (k != i) qhat = hm::mulmod(qhat, t->q[in_idx[k]] % qi, qi);
        const u64 inv = hm::invmod(qhat, qi);
        a.qin[i] = (uint32_t)qi;
        a.qhinv[i] = make_uint2((uint32_t)inv, shoup32_host((uint32_t)inv, (uint32_t)qi));
        for (int j = 0; j < n_out; j++) {
            const u64 pj = t->q[out_idx[j]];
            u64 m = 1;
            for (int k = 0; k < n_in; k++)
                if (k != i) m = hm::mulmod(m, t->q[in_idx[k]] % pj, pj);
            a.M[i][j] = (uint32_t)m;
        }
    }
    for (int j = 0; j < n_out; j++) {
        const uint32_t pj = t->q[out_idx[j]];
        const uint32_t r = (uint32_t)((1ull << 32) % pj);
        a.p[j] = pj;
        a.r32[j] = make_uint2(r, shoup32_host(r, pj));
        a.m32[j] = (uint32_t)((1ull << 32) / pj);
    }
    k_bconv32<<<dim3(t->n / 1024, batch), 256, 0, (cudaStream_t)stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? SECPE_OK : SECPE_ECUDA;
}
