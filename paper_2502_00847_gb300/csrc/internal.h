// Internal declarations of the SecPE GB300 library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/secpe.h"
#include "modarith.cuh"

#define SECPE_MAX_PRIMES 64
#define SECPE_MAX_LIMBSET 256

// ---------------------------------------------------------------------------
// Device-resident tables, passed to kernels by value.
// ---------------------------------------------------------------------------
struct DevCtx {
    int log_n, n;
    int nq, np_special, nprimes;  // nprimes = nq + np_special
    int dnum, alpha;
    const u64 *q;          // [nprimes]
    const u64 *qinv_neg;   // [nprimes]  -q^-1 mod 2^64
    const u64 *r2;         // [nprimes]  2^128 mod q
    const u64 *mu;         // [nprimes]  floor(2^64 / q)
    const u64 *mont_one;   // [nprimes]  2^64 mod q (Montgomery form of 1)
    const ulonglong2 *tw_fwd;  // [nprimes][N]  (psi^brv(k), shoup)
    const ulonglong2 *tw_inv;  // [nprimes][N]  (psi^-brv(k), shoup)
    const ulonglong2 *ninv;    // [nprimes]     (N^-1, shoup)
    const ulonglong2 *ninv_w1; // [nprimes]     (psi^-brv(1) * N^-1, shoup)
    // INTT final scalings that also apply a base-conversion pre-multiplier:
    // [lv*nq + i][2]: N^-1 * [Qhat_i^-1]_{q_i} of prime i's digit at level lv (and * psi^-brv(1))
    const ulonglong2 *ninv_modup;
    // [j][2]: N^-1 * [Phat_j^-1]_{p_j} (and * psi^-brv(1)) for special prime j
    const ulonglong2 *ninv_moddown;
    // ModUp base conversion, per (level, digit): digit prime i (< alpha)
    const ulonglong2 *mu_inv;  // [(L+1)*dnum*alpha]  [Qhat_i^-1]_{q_i} (shoup)
    const u64 *mu_hat;         // [(L+1)*dnum*alpha*nprimes] Montgomery form of Qhat_i mod t
    // ModDown from the special primes
    const ulonglong2 *md_inv;  // [np_special] [Phat_j^-1]_{p_j} (shoup)
    const u64 *md_hat;         // [np_special*nq] Montgomery form of Phat_j mod q_i
    const ulonglong2 *md_pinv; // [nq] P^-1 mod q_i (shoup)
    const u64 *md_hP;          // [nprimes] floor(P/2) mod t
    // Relinearisation's ModDown fused with the rescale at level l: division by
    // M = P q_l from the sources s = (q_l, p_0, .., p_{k-1}), per level l:
    const ulonglong2 *mdr_ninv;  // [(l*(k+1) + j)*2 + {0,1}] INTT scaling N^-1 [(M/s_j)^-1]_{s_j} (and * psi^-brv(1))
    const ulonglong2 *mdr_inv;   // [l*(k+1) + j] [(M/s_j)^-1]_{s_j} (shoup)
    const u64 *mdr_pre;          // [l*(k+1) + j] floor(M/2) mod s_j
    const u64 *mdr_hat;          // [(l*(k+1) + j)*nq + i] Montgomery form of (M/s_j) mod q_i
    const u64 *mdr_post;         // [l*nq + i] floor(M/2) mod q_i
    const ulonglong2 *mdr_w;     // [l*nq + i] M^-1 mod q_i (shoup)
    const u64 *pmod;             // [nprimes] P mod prime t
    // Rescale by q_l, per level l: [l*nq + i]
    const ulonglong2 *rs_qinv; // q_l^-1 mod q_i (shoup)
    const u64 *rs_hmod;        // floor(q_l/2) mod q_i
    // Mixed-radix CRT over q_0..q_l
    const ulonglong2 *mr_inv;  // [nq*nq]  [j*nq+i] = q_j^-1 mod q_i (shoup)
    const u64 *mr_M;           // [nq*nq]  [i*nq+t] = (q_0...q_{i-1}) mod q_t
    const u64 *mr_H;           // [nq*nq]  [l*nq+i] mixed-radix digit i of (Q_l-1)/2
    const u64 *mr_Q;           // [nq*nq]  [l*nq+t] = Q_l mod q_t
    const double *mr_Mf;       // [nq] (q_0...q_{i-1}) as double
    int *status;               // device status word
};

// A set of limbs for batched per-limb kernels: limb (item, poly, j) lives at
// base + item*item_stride + poly*poly_stride + j*N and is taken modulo the
// prime of index prime_of[poly*nlimb + j].
struct LimbSet {
    u64 *base;
    long long item_stride, poly_stride;
    int nitem, npoly, nlimb;
    int8_t prime_of[SECPE_MAX_LIMBSET];
    int8_t aux[SECPE_MAX_LIMBSET];  // per-limb group (which base-conversion source)
};

// A batch of B ciphertexts laid out [B][2][cap][N] with `stride` words
// between items (stride >= 2*cap*N); limbs 0..level valid.
struct CtB {
    u64 *data = nullptr;
    int B = 0;
    long long stride = 0;
    int cap = 0;
    int level = 0;
    double scale = 0.0;
    int n = 0;
    u64 *poly(int b, int k) const { return data + b * stride + (long long)k * cap * n; }
    long long pstride() const { return (long long)cap * n; }
};

// event-based timing of selected kernel launches (secpe_kprof_*)
struct KProf {
    bool active = false;
    bool all = false;             // filter "*": every launch, by kernel name
    std::string filter;
    std::vector<cudaEvent_t> ev;  // pairs
    std::vector<const char *> names;  // kernel name of pair i (filter "*")
    std::vector<float> ms;        // duration of pair i, filled by secpe_kprof_end
    int used = 0;                 // pairs recorded
    int64_t launches = 0;
    double bytes = 0.0;        // algorithmic bytes (operands read once, results written once)
    double model_bytes = 0.0;  // bytes each launch itself reads and writes (intermediates included)
    double mul32 = 0.0;        // algorithmic 32-bit multiplies
};

// Launch configurations chosen by secpe_autotune: CTAs per SM (3 or 4, i.e.
// at most 80 or 64 registers per thread) of each tuned N = 2^16 kernel.
enum TuneSlot { TUNE_COLPASS = 0, TUNE_ROWPASS, TUNE_ICOLPASS, TUNE_IROWPASS, TUNE_BCONV, TUNE_NSLOTS };
struct Tuning {
    int ctas[TUNE_NSLOTS] = {3, 3, 3, 3, 3};
    bool tuned = false;
};

// Device buffers handed to the C ABI must start on a 16-byte boundary and
// item strides must be even (in words): the kernels read and write residues
// with 16-byte vector accesses and bulk copies.
static inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

struct secpe_ctx {
    secpe_params p;
    int n, log_n, nq, npsp, nprimes, L, dnum, alpha;
    std::vector<u64> primes;   // q_0..q_L, p_0..p_{k-1}
    std::vector<u64> psi;
    double scale;
    DevCtx dev;
    std::vector<void *> allocations;
    int *d_status;
    secpe_counters counters;
    // bootstrapping plan that replaces the refresh stand-in for the duration
    // of a call (secpe_argmax_batch_boot); null otherwise
    const secpe_boot *boot = nullptr;
    cudaStream_t stream;  // stream of the call in progress
    KProf kprof;
    Tuning tune;
    // host copies used by host-side constant encoding
    std::vector<u64> h_qinv_neg, h_r2, h_mu;
    std::vector<ulonglong2> h_mu_inv;  // host mirror of DevCtx::mu_inv
    std::vector<u64> h_mdr_pre_scaled; // [l*(k+1) + j] floor(M/2) * [(M/s_j)^-1] mod s_j
    // set for the duration of a precision-variant call: every NTT/INTT and
    // the key inner product run on the tensor pipe (ntt_tc.cu), and the
    // unfused key-switching kernels are used
    int tc_mode = 0;
};

struct secpe_keys {
    int seed_set;
    uint64_t seed;
    u64 *s_ntt;                        // [nprimes][N] plain residues
    u64 *rlk;                          // [dnum][2][nprimes][N] Montgomery form
    std::map<uint32_t, u64 *> gks;     // Galois element -> key
};

// ---------------------------------------------------------------------------
// host math (hostmath.cpp)
// ---------------------------------------------------------------------------
namespace hm {
u64 mulmod(u64 a, u64 b, u64 q);
u64 powmod(u64 a, u64 e, u64 q);
u64 invmod(u64 a, u64 q);
u64 shoup(u64 w, u64 q);      // floor(w * 2^64 / q)
u64 neg_inv64(u64 q);         // -q^-1 mod 2^64
bool is_prime(u64 n);
// Prime selection rule of secpe_params (see secpe.h); returns false when the
// parameters are out of range.
bool select_primes(const secpe_params &p, std::vector<u64> &q, std::vector<u64> &special);
u64 find_psi(u64 q, u64 n);
uint32_t bitrev(uint32_t x, int bits);
// Counter-based SplitMix64 stream (Steele, Lea, Flood 2014).
u64 sm_mix(u64 z);
// sparse ternary secret: h signs placed by the words of stream `key`
// (word w: position (w >> 1) mod n unless taken, sign w & 1 ? -1 : +1)
void sample_sparse_secret(u64 key, int n, int h, std::vector<long long> &s);
u64 sm_stream(u64 seed, u64 domain, u64 index);
long long round_half_away(double v);
}  // namespace hm

// stream domains of the counter-based sampler
enum { DOM_SECRET = 1, DOM_KSK_A = 2, DOM_KSK_E = 3, DOM_ENC_A = 4, DOM_ENC_E = 5,
       DOM_REFRESH = 6, DOM_PHOENIX = 7 };
