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
    std::vector<u64> h_tw1;  // psi^-brv(1) per prime (the inverse's last twiddle)
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
    // inverse only, optional: limb i's final scaling N^-1 s_i (and its
    // product with the last twiddle) instead of N^-1, both with Shoup parts
    int has_scale;
    uint2 scale[2 * kMaxLimbs32];
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
        const uint2 ni = a.has_scale ? a.scale[2 * lid] : a.ninv[pi];
        const uint2 nw = a.has_scale ? a.scale[2 * lid + 1] : a.ninvw1[pi];
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
    const uint32_t *in;  // item b at in + b * in_stride, limbs [n_in][N]
    uint32_t *out;       // item b at out + b * out_stride, limbs [n_out][N]
    long long in_stride, out_stride;
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
    const uint32_t *__restrict__ in = a.in + item * a.in_stride + c;
    uint32_t *__restrict__ out = a.out + item * a.out_stride + c;
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
        t->h_tw1.push_back(ipw[hm::bitrev(1, log_n)]);
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

namespace {
int ntt32_run(const secpe_ntt32_table *t, uint32_t *limbs, const int32_t *prime_idx, int count, int inverse,
              const uint32_t *scale_by, cudaStream_t stream);
}  // namespace

extern "C" int secpe_ntt32(const secpe_ntt32_table *t, uint32_t *limbs, const int32_t *prime_idx, int count, int inverse,
                           void *stream) {
    SECPE_CHECK(check_limbs(t, limbs, prime_idx, count));
    return ntt32_run(t, limbs, prime_idx, count, inverse, nullptr, (cudaStream_t)stream);
}

namespace {

// scale_by (inverse only, optional): limb i's result multiplied by
// scale_by[i] (a residue of its prime) within the final N^-1 scaling
int ntt32_run(const secpe_ntt32_table *t, uint32_t *limbs, const int32_t *prime_idx, int count, int inverse,
              const uint32_t *scale_by, cudaStream_t stream) {
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
        a.has_scale = scale_by && inverse ? 1 : 0;
        if (a.has_scale)
            for (int i = 0; i < nl; i++) {
                const u64 q = t->q[prime_idx[c0 + i]];
                const u64 ni = hm::mulmod(hm::invmod((u64)t->n, q), scale_by[c0 + i] % q, q);
                const u64 w1 = t->h_tw1[prime_idx[c0 + i]];
                const u64 nw = hm::mulmod(ni, w1, q);
                a.scale[2 * i] = make_uint2((uint32_t)ni, shoup32_host((uint32_t)ni, (uint32_t)q));
                a.scale[2 * i + 1] = make_uint2((uint32_t)nw, shoup32_host((uint32_t)nw, (uint32_t)q));
            }
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

}  // namespace

namespace {

// FastBConv of `batch` items with the given item strides (in words).
int bconv32(const secpe_ntt32_table *t, const uint32_t *in, long long in_stride, const int32_t *in_idx, int n_in,
            uint32_t *out, long long out_stride, const int32_t *out_idx, int n_out, int batch, cudaStream_t stream) {
    if (n_in < 1 || n_in > kMaxIn32 || n_out < 1 || n_out > kMaxOut32 || batch < 1 || batch > 65535)
        return SECPE_EINVAL;
    for (int i = 0; i < n_in; i++)
        for (int k = 0; k < i; k++)
            if (in_idx[i] == in_idx[k]) return SECPE_EINVAL;
    BConv32Args a;
    a.in = in;
    a.out = out;
    a.in_stride = in_stride;
    a.out_stride = out_stride;
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
    k_bconv32<<<dim3(t->n / 1024, batch), 256, 0, stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? SECPE_OK : SECPE_ECUDA;
}

}  // namespace

extern "C" int secpe_bconv32(const secpe_ntt32_table *t, const uint32_t *in, const int32_t *in_idx, int n_in,
                             uint32_t *out, const int32_t *out_idx, int n_out, int batch, void *stream) {
    SECPE_CHECK(check_limbs(t, in, in_idx, n_in));
    SECPE_CHECK(check_limbs(t, out, out_idx, n_out));
    return bconv32(t, in, (long long)n_in * t->n, in_idx, n_in, out, (long long)n_out * t->n, out_idx, n_out, batch,
                   (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Hybrid key switching on 32-bit residues (the word-size probe's key switch;
// the steps of keyswitch.cu on the 64-bit path): INTT of d, per digit
// FastBConv to every other prime and NTT, the key inner product, then ModDown
// (rounded division by P: [x + h]_P with h = floor(P/2) on every coefficient
// of the special limbs, FastBConv to the q primes, minus h on every
// coefficient, NTT, out_i = (x_i - conv_i) P^-1).

namespace {

constexpr int kMaxDig32 = 16;
constexpr int kMaxTgt32 = 64;

// x mod p for a 64-bit x = hi 2^32 + lo: [hi 2^32]_p by Shoup, lo by a
// quotient estimate, each in [0, 2p).
__device__ __forceinline__ uint32_t red64_32(unsigned long long x, uint32_t p, uint2 r32, uint32_t m32) {
    const uint32_t hi = (uint32_t)(x >> 32), lo = (uint32_t)x;
    return red4_32(shoup32(hi, r32.x, r32.y, p) + (lo - __umulhi(lo, m32) * p), p);
}

struct Ip32Args {
    const uint32_t *d;    // [B][nq][N] NTT form
    const uint32_t *ext;  // [B][tot][N]: digit j's other primes at off[j]
    const uint32_t *key;  // [dnum][2][nt][N]
    uint32_t *acc;        // [B][2][nt][N]
    int nq, nt, tot, ndig;
    int lo[kMaxDig32], hi[kMaxDig32], off[kMaxDig32];
    uint32_t p[kMaxTgt32];
    uint2 r32[kMaxTgt32];
    uint32_t m32[kMaxTgt32];
};

// grid: (N / 256, nt * B); the items sharing one key limb run back to back
__global__ void __launch_bounds__(256) k_ip32(const __grid_constant__ Ip32Args a) {
    const int nitem = gridDim.y / a.nt;
    const int t = blockIdx.y / nitem, item = blockIdx.y % nitem;
    const int e = blockIdx.x * 256 + threadIdx.x;
    unsigned long long s0 = 0, s1 = 0;
    const size_t plane = (size_t)a.nt * 65536;
    for (int j = 0; j < a.ndig; j++) {
        uint32_t x;
        if (t >= a.lo[j] && t < a.hi[j]) {
            x = a.d[((size_t)item * a.nq + t) * 65536 + e];
        } else {
            const int tt = t < a.lo[j] ? t : t - (a.hi[j] - a.lo[j]);
            x = a.ext[((size_t)item * a.tot + a.off[j] + tt) * 65536 + e];
        }
        const uint32_t *kb = a.key + (size_t)j * 2 * plane + (size_t)t * 65536 + e;
        s0 += (unsigned long long)x * kb[0];
        s1 += (unsigned long long)x * kb[plane];
    }
    uint32_t *o = a.acc + ((size_t)item * 2 * a.nt + t) * 65536 + e;
    o[0] = red64_32(s0, a.p[t], a.r32[t], a.m32[t]);
    o[plane] = red64_32(s1, a.p[t], a.r32[t], a.m32[t]);
}

// x[row][limb l][N] += c[l] mod prime of limb l (rows of nl limbs)
struct AddC32Args {
    uint32_t *x;
    int nl;
    uint32_t c[kMaxTgt32], q[kMaxTgt32];
};

__global__ void __launch_bounds__(256) k_addc32(const __grid_constant__ AddC32Args a) {
    const int li = blockIdx.y, l = li % a.nl;
    const int e = blockIdx.x * 256 + threadIdx.x;
    uint32_t *p = a.x + (size_t)li * 65536 + e;
    const uint32_t v = *p + a.c[l];
    *p = v >= a.q[l] ? v - a.q[l] : v;
}

// out[b][k][i] = (acc[b][k][i] - conv[b][k][i]) * P^-1 mod q_i, conv the
// NTT of FastBConv([x + h]_P) - h
struct Epi32Args {
    const uint32_t *acc;   // [B][2][nt][N]
    const uint32_t *conv;  // [B][2][nq][N] (NTT form)
    uint32_t *out;         // [B][2][nq][N]
    int nq, nt;
    uint32_t q[kMaxTgt32];
    uint2 pinv[kMaxTgt32];
};

__global__ void __launch_bounds__(256) k_epi32(const __grid_constant__ Epi32Args a) {
    const int li = blockIdx.y;  // (item, poly, i)
    const int i = li % a.nq, kp = li / a.nq;
    const int e = blockIdx.x * 256 + threadIdx.x;
    const uint32_t q = a.q[i];
    const uint32_t x = a.acc[((size_t)kp * a.nt + i) * 65536 + e];
    const uint32_t c = a.conv[((size_t)kp * a.nq + i) * 65536 + e];
    const uint32_t v = x >= c ? x - c : x + q - c;  // [0, q)
    a.out[((size_t)kp * a.nq + i) * 65536 + e] = red2_32(shoup32(v, a.pinv[i].x, a.pinv[i].y, q), q);
}

void red_consts(const secpe_ntt32_table *t, int pi, uint32_t &p, uint2 &r, uint32_t &m) {
    p = t->q[pi];
    const uint32_t rr = (uint32_t)((1ull << 32) % p);
    r = make_uint2(rr, shoup32_host(rr, p));
    m = (uint32_t)((1ull << 32) / p);
}

}  // namespace

// Fused ModUp and inner product (the 64-bit path's k_colpass_bconv and
// k_rowpass_ip on 32-bit words).  Pass A: for one extended limb (item,
// digit j, target prime) and 16 columns, the FastBConv of the digit's
// pre-multiplied coefficients y (the INTT applied [Qhat_i^-1]) straight
// into registers, then the forward column rounds; pass B + inner product:
// for one target limb and 16 rows, every digit's row rounds (or the input's
// own limb) multiplied by the key and accumulated modulo the target prime.
namespace {

constexpr int kFusedSrc32 = 16;

struct ModUpA32Args {
    const uint32_t *y;     // [B][nq][N] coefficient form, times [Qhat_i^-1]
    uint32_t *ext;         // [B][tot][N] pass-A output (lazy, [0, 4p))
    const uint32_t *q;     // device prime table
    const uint2 *tw;       // forward twiddles [np][N]
    int nq, tot;
    uint8_t lo[kMaxLimbs32], ns[kMaxLimbs32], prime_of[kMaxLimbs32];
    uint32_t M[kMaxLimbs32][kFusedSrc32];  // [Qhat_r]_p of source r for extended limb l
    uint2 r32[kMaxLimbs32];
    uint32_t m32[kMaxLimbs32];
};

__global__ void __launch_bounds__(256) k_modup_a32(const __grid_constant__ ModUpA32Args a) {
    __shared__ uint32_t sm[4096];
    const int lid = blockIdx.x >> 4, c0 = (blockIdx.x & 15) * 16;
    const int item = lid / a.tot, el = lid % a.tot;
    const int pi = a.prime_of[el], lo = a.lo[el], ns = a.ns[el];
    const uint32_t p = a.q[pi];
    const uint2 *tw = a.tw + (size_t)pi * 65536;
    const uint32_t *y = a.y + ((size_t)item * a.nq + lo) * 65536;
    const int col = threadIdx.x & 15, u = threadIdx.x >> 4;
    uint32_t x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) {
        const int e = ((k << 4) | u) * 256 + c0 + col;
        unsigned long long acc = 0;
        for (int r = 0; r < ns; r++) acc += (unsigned long long)y[(size_t)r * 65536 + e] * a.M[el][r];
        x[k] = red64_32(acc, p, a.r32[el], a.m32[el]);
    }
    fwd16<8, 4>(x, u, tw, 1, p);
#pragma unroll
    for (int k = 0; k < 16; k++) sm[col_sm((k << 4) | u, col)] = x[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = sm[col_sm((u << 4) | k, col)];
    fwd16<8, 0>(x, u << 4, tw, 1, p);
    uint32_t *g = a.ext + ((size_t)item * a.tot + el) * 65536;
#pragma unroll
    for (int k = 0; k < 16; k++) g[((u << 4) | k) * 256 + c0 + col] = x[k];
}

struct IpB32Args {
    const uint32_t *d;    // [B][nq][N] NTT form
    const uint32_t *ext;  // pass-A output
    const uint32_t *key;  // [dnum][2][nt][N]
    uint32_t *acc;        // [B][2][nt][N]
    const uint32_t *q;
    const uint2 *tw;
    int nq, nt, tot, ndig, B;
    int lo[kMaxDig32], hi[kMaxDig32], off[kMaxDig32];
    uint8_t prime_of[kMaxTgt32];
    uint2 r32[kMaxTgt32];
    uint32_t m32[kMaxTgt32];
};

// grid: ((t * 16 + tile) * B + item)
__global__ void __launch_bounds__(256) k_ip_b32(const __grid_constant__ IpB32Args a) {
    __shared__ uint32_t sm[16 * 272];
    const int item = blockIdx.x % a.B, tt16 = blockIdx.x / a.B;
    const int tile = tt16 & 15, t = tt16 >> 4, r0 = tile * 16;
    const int pi = a.prime_of[t];
    const uint32_t p = a.q[pi];
    const uint2 *tw = a.tw + (size_t)pi * 65536;
    const int u = threadIdx.x & 15, row = threadIdx.x >> 4, base = 256 + r0 + row;
    uint32_t *__restrict__ srow = sm + row * 272;
    const size_t plane = (size_t)a.nt * 65536, toff = (size_t)t * 65536 + (size_t)r0 * 256;
    uint32_t acc0[16], acc1[16];
#pragma unroll
    for (int i = 0; i < 16; i++) acc0[i] = acc1[i] = 0;
    for (int j = 0; j < a.ndig; j++) {
        const bool own = t >= a.lo[j] && t < a.hi[j];
        if (!own) {
            const int ti = t < a.lo[j] ? t : t - (a.hi[j] - a.lo[j]);
            const uint32_t *g = a.ext + ((size_t)item * a.tot + a.off[j] + ti) * 65536 + (size_t)r0 * 256;
            uint32_t x[16];
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] = g[row * 256 + ((k << 4) | u)];
            fwd16<8, 4>(x, u, tw, base, p);
#pragma unroll
            for (int k = 0; k < 16; k++) srow[PAD17((k << 4) | u)] = x[k];
            __syncthreads();
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] = srow[PAD17((u << 4) | k)];
            fwd16<8, 0>(x, u << 4, tw, base, p);
#pragma unroll
            for (int k = 0; k < 16; k++) srow[PAD17((u << 4) | k)] = red4_32(x[k], p);
            __syncthreads();
        }
        const uint32_t *kb = a.key + (size_t)j * 2 * plane + toff;
        const uint32_t *dd = a.d + ((size_t)item * a.nq + t) * 65536 + (size_t)r0 * 256;
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const int e = threadIdx.x + 256 * i;
            const uint32_t v = own ? dd[e] : sm[(e >> 8) * 272 + PAD17(e & 255)];
            const uint32_t k0 = kb[e], k1 = kb[plane + e];
            acc0[i] = red2_32(acc0[i] + red64_32((unsigned long long)v * k0, p, a.r32[t], a.m32[t]), p);
            acc1[i] = red2_32(acc1[i] + red64_32((unsigned long long)v * k1, p, a.r32[t], a.m32[t]), p);
        }
        if (!own) __syncthreads();
    }
    uint32_t *o = a.acc + (size_t)item * 2 * plane + toff;
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const int e = threadIdx.x + 256 * i;
        o[e] = acc0[i];
        o[plane + e] = acc1[i];
    }
}

// steps 1-3 fused: INTT of d with the ModUp pre-multipliers, pass A with
// FastBConv for every extended limb, pass B + inner product for every target
int modup_ip_fused32(const secpe_ntt32_table *t, const uint32_t *d, const int32_t *q_idx, int nq,
                     const std::vector<int32_t> &tgt, int alpha, int ndig, const Ip32Args &ia, int tot,
                     const uint32_t *key, uint32_t *coef, uint32_t *ext, uint32_t *acc, int batch, cudaStream_t st) {
    const int n = t->n, nt = (int)tgt.size();
    if (tot > kMaxLimbs32 || alpha > kFusedSrc32) return SECPE_EINVAL;
    // [Qhat_i^-1]_{q_i} of every limb within its digit
    std::vector<uint32_t> qhinv(nq);
    for (int j = 0; j < ndig; j++)
        for (int i = ia.lo[j]; i < ia.hi[j]; i++) {
            const u64 qi = t->q[q_idx[i]];
            u64 qh = 1;
            for (int k = ia.lo[j]; k < ia.hi[j]; k++)
                if (k != i) qh = hm::mulmod(qh, t->q[q_idx[k]] % qi, qi);
            qhinv[i] = (uint32_t)hm::invmod(qh, qi);
        }
    if (cudaMemcpyAsync(coef, d, sizeof(uint32_t) * n * batch * nq, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SECPE_ECUDA;
    std::vector<int32_t> pidx;
    std::vector<uint32_t> sc;
    for (int b = 0; b < batch; b++) {
        pidx.insert(pidx.end(), q_idx, q_idx + nq);
        sc.insert(sc.end(), qhinv.begin(), qhinv.end());
    }
    SECPE_CHECK(ntt32_run(t, coef, pidx.data(), batch * nq, 1, sc.data(), st));
    ModUpA32Args ma;
    ma.y = coef;
    ma.ext = ext;
    ma.q = t->d_q;
    ma.tw = t->d_twf;
    ma.nq = nq;
    ma.tot = tot;
    for (int j = 0; j < ndig; j++) {
        int el = ia.off[j];
        for (int i = 0; i < nt; i++) {
            if (i >= ia.lo[j] && i < ia.hi[j]) continue;
            const u64 pt = t->q[tgt[i]];
            ma.lo[el] = (uint8_t)ia.lo[j];
            ma.ns[el] = (uint8_t)(ia.hi[j] - ia.lo[j]);
            ma.prime_of[el] = (uint8_t)tgt[i];
            for (int r = 0; r < ia.hi[j] - ia.lo[j]; r++) {
                u64 m = 1;
                for (int k = ia.lo[j]; k < ia.hi[j]; k++)
                    if (k != ia.lo[j] + r) m = hm::mulmod(m, t->q[q_idx[k]] % pt, pt);
                ma.M[el][r] = (uint32_t)m;
            }
            uint32_t pp;
            red_consts(t, tgt[i], pp, ma.r32[el], ma.m32[el]);
            el++;
        }
    }
    k_modup_a32<<<(unsigned)(batch * tot * 16), 256, 0, st>>>(ma);
    if (cudaGetLastError() != cudaSuccess) return SECPE_ECUDA;
    IpB32Args ib;
    ib.d = d;
    ib.ext = ext;
    ib.key = key;
    ib.acc = acc;
    ib.q = t->d_q;
    ib.tw = t->d_twf;
    ib.nq = nq;
    ib.nt = nt;
    ib.tot = tot;
    ib.ndig = ndig;
    ib.B = batch;
    for (int j = 0; j < ndig; j++) {
        ib.lo[j] = ia.lo[j];
        ib.hi[j] = ia.hi[j];
        ib.off[j] = ia.off[j];
    }
    for (int i = 0; i < nt; i++) {
        uint32_t pp;
        ib.prime_of[i] = (uint8_t)tgt[i];
        red_consts(t, tgt[i], pp, ib.r32[i], ib.m32[i]);
    }
    k_ip_b32<<<(unsigned)(nt * 16 * batch), 256, 0, st>>>(ib);
    return cudaGetLastError() == cudaSuccess ? SECPE_OK : SECPE_ECUDA;
}

}  // namespace

extern "C" int secpe_keyswitch32(const secpe_ntt32_table *t, const uint32_t *d, const int32_t *q_idx, int nq,
                                 const int32_t *p_idx, int np, int alpha, const uint32_t *key, uint32_t *out,
                                 int batch, int fused, void *stream) {
    SECPE_CHECK(check_limbs(t, d, q_idx, nq));
    SECPE_CHECK(check_limbs(t, out, q_idx, nq));
    SECPE_CHECK(check_limbs(t, key, p_idx, np));
    const int nt = nq + np, ndig = alpha > 0 ? (nq + alpha - 1) / alpha : 0;
    if (nq < 1 || np < 1 || nt > kMaxTgt32 || alpha < 1 || alpha > kMaxIn32 || np > kMaxIn32 || ndig > kMaxDig32 ||
        batch < 1 || (long long)batch * 2 * nt > 65535)
        return SECPE_EINVAL;
    const int n = t->n;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> tgt(q_idx, q_idx + nq);
    tgt.insert(tgt.end(), p_idx, p_idx + np);
    for (int i = 0; i < nt; i++)
        for (int k = 0; k < i; k++)
            if (tgt[i] == tgt[k]) return SECPE_EINVAL;
    Ip32Args ia;
    int tot = 0;
    for (int j = 0; j < ndig; j++) {
        ia.lo[j] = j * alpha;
        ia.hi[j] = std::min(nq, (j + 1) * alpha);
        ia.off[j] = tot;
        tot += nt - (ia.hi[j] - ia.lo[j]);
    }
    uint32_t *coef = nullptr, *ext = nullptr, *acc = nullptr, *spec = nullptr, *conv = nullptr;
    const size_t W = sizeof(uint32_t) * n;
    bool ok = cudaMallocAsync((void **)&coef, W * batch * nq, st) == cudaSuccess &&
              cudaMallocAsync((void **)&ext, W * batch * tot, st) == cudaSuccess &&
              cudaMallocAsync((void **)&acc, W * batch * 2 * nt, st) == cudaSuccess &&
              cudaMallocAsync((void **)&spec, W * batch * 2 * np, st) == cudaSuccess &&
              cudaMallocAsync((void **)&conv, W * batch * 2 * nq, st) == cudaSuccess;
    int rc = ok ? SECPE_OK : SECPE_ENOMEM;
    std::vector<int32_t> pidx;
    if (fused) {
        rc = rc == SECPE_OK ? modup_ip_fused32(t, d, q_idx, nq, tgt, alpha, ndig, ia, tot, key, coef, ext, acc, batch, st)
                            : rc;
    } else {
    // 1. INTT of d
    if (rc == SECPE_OK && cudaMemcpyAsync(coef, d, W * batch * nq, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        rc = SECPE_ECUDA;
    for (int b = 0; b < batch; b++) pidx.insert(pidx.end(), q_idx, q_idx + nq);
    if (rc == SECPE_OK) rc = secpe_ntt32(t, coef, pidx.data(), batch * nq, 1, stream);
    // 2. ModUp per digit, NTT of the extended limbs
    std::vector<int32_t> eidx;
    for (int j = 0; j < ndig && rc == SECPE_OK; j++) {
        std::vector<int32_t> others;
        for (int i = 0; i < nt; i++)
            if (i < ia.lo[j] || i >= ia.hi[j]) others.push_back(tgt[i]);
        rc = bconv32(t, coef + (size_t)ia.lo[j] * n, (long long)nq * n, q_idx + ia.lo[j], ia.hi[j] - ia.lo[j],
                     ext + (size_t)ia.off[j] * n, (long long)tot * n, others.data(), (int)others.size(), batch, st);
        eidx.insert(eidx.end(), others.begin(), others.end());
    }
    pidx.clear();
    for (int b = 0; b < batch; b++) pidx.insert(pidx.end(), eidx.begin(), eidx.end());
    if (rc == SECPE_OK) rc = secpe_ntt32(t, ext, pidx.data(), batch * tot, 0, stream);
    // 3. key inner product
    if (rc == SECPE_OK) {
        ia.d = d;
        ia.ext = ext;
        ia.key = key;
        ia.acc = acc;
        ia.nq = nq;
        ia.nt = nt;
        ia.tot = tot;
        ia.ndig = ndig;
        for (int i = 0; i < nt; i++) red_consts(t, tgt[i], ia.p[i], ia.r32[i], ia.m32[i]);
        k_ip32<<<dim3(n / 256, nt * batch), 256, 0, st>>>(ia);
        if (cudaGetLastError() != cudaSuccess) rc = SECPE_ECUDA;
    }
    }
    // 4. ModDown of both polynomials
    if (rc == SECPE_OK &&
        cudaMemcpy2DAsync(spec, W * np, acc + (size_t)nq * n, W * nt, W * np, (size_t)batch * 2,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        rc = SECPE_ECUDA;
    pidx.clear();
    for (int r = 0; r < 2 * batch; r++) pidx.insert(pidx.end(), p_idx, p_idx + np);
    if (rc == SECPE_OK) rc = secpe_ntt32(t, spec, pidx.data(), 2 * batch * np, 1, stream);
    // h = floor(P / 2) mod each prime: P = prod p_r
    std::vector<u64> hmod(nt);
    for (int i = 0; i < nt; i++) {
        const u64 m = t->q[tgt[i]];
        // floor(P/2) mod m = (P - (P mod 2)) / 2 mod m; P is odd, so (P - 1) * 2^-1 mod m
        u64 pm = 1;
        for (int r = 0; r < np; r++) pm = hm::mulmod(pm, t->q[p_idx[r]] % m, m);
        hmod[i] = hm::mulmod((pm + m - 1) % m, hm::invmod(2, m), m);
    }
    if (rc == SECPE_OK) {
        AddC32Args ca;
        ca.x = spec;
        ca.nl = np;
        for (int r = 0; r < np; r++) {
            ca.c[r] = (uint32_t)hmod[nq + r];
            ca.q[r] = t->q[p_idx[r]];
        }
        k_addc32<<<dim3(n / 256, 2 * batch * np), 256, 0, st>>>(ca);
        if (cudaGetLastError() != cudaSuccess) rc = SECPE_ECUDA;
    }
    if (rc == SECPE_OK)
        rc = bconv32(t, spec, (long long)np * n, p_idx, np, conv, (long long)nq * n, q_idx, nq, 2 * batch, st);
    if (rc == SECPE_OK) {
        // - h on every coefficient of the conversion
        AddC32Args ca;
        ca.x = conv;
        ca.nl = nq;
        for (int i = 0; i < nq; i++) {
            ca.q[i] = t->q[q_idx[i]];
            ca.c[i] = (uint32_t)((ca.q[i] - hmod[i]) % ca.q[i]);
        }
        k_addc32<<<dim3(n / 256, 2 * batch * nq), 256, 0, st>>>(ca);
        if (cudaGetLastError() != cudaSuccess) rc = SECPE_ECUDA;
    }
    pidx.clear();
    for (int r = 0; r < 2 * batch; r++) pidx.insert(pidx.end(), q_idx, q_idx + nq);
    if (rc == SECPE_OK) rc = secpe_ntt32(t, conv, pidx.data(), 2 * batch * nq, 0, stream);
    if (rc == SECPE_OK) {
        Epi32Args ea;
        ea.acc = acc;
        ea.conv = conv;
        ea.out = out;
        ea.nq = nq;
        ea.nt = nt;
        for (int i = 0; i < nq; i++) {
            const u64 q = t->q[q_idx[i]];
            u64 pm = 1;
            for (int r = 0; r < np; r++) pm = hm::mulmod(pm, t->q[p_idx[r]] % q, q);
            const u64 pinv = hm::invmod(pm, q);
            ea.q[i] = (uint32_t)q;
            ea.pinv[i] = make_uint2((uint32_t)pinv, shoup32_host((uint32_t)pinv, (uint32_t)q));
        }
        k_epi32<<<dim3(n / 256, 2 * batch * nq), 256, 0, st>>>(ea);
        if (cudaGetLastError() != cudaSuccess) rc = SECPE_ECUDA;
    }
    cudaFreeAsync(coef, st);
    cudaFreeAsync(ext, st);
    cudaFreeAsync(acc, st);
    cudaFreeAsync(spec, st);
    cudaFreeAsync(conv, st);
    return rc;
}
