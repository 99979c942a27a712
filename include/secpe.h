/*
 * secpe.h - C ABI of a GB300 (sm_103a) library for SecPE's encrypted
 * prompt-ensemble aggregation and encrypted Argmax on RNS-CKKS
 * (Zhang et al., "SecPE: Secure Prompt Ensembling for Private and Robust
 * Large Language Models", arXiv 2502.00847).
 *
 * Conventions
 * -----------
 * - Every call returns an int status: SECPE_OK (0) or a negative SECPE_E*.
 *   Host-side validation errors are returned synchronously and nothing is
 *   launched.  Calls that take a cudaStream_t (passed as void*) are
 *   asynchronous on that stream; device-side failures (a bounded wait that
 *   gave up) are recorded in a per-context status word read by
 *   secpe_stream_status.
 * - Ciphertext data is caller-owned device memory laid out as
 *   [2][cap][N] uint64 words, cap >= level+1: polynomial c0 then c1, each a
 *   stack of cap RNS limbs of N residues in NTT (evaluation) form, limb i
 *   modulo q_i.  Only limbs 0..level are meaningful.  The library never
 *   frees caller buffers.  Batched calls take arrays of secpe_ct.
 * - Every device buffer passed in (ciphertext data, limb arrays, key-switch
 *   operands) must start on a 16-byte boundary and every item stride (in
 *   words) must be even; cudaMalloc and PyTorch allocations satisfy this.
 *   Other pointers or strides are rejected with SECPE_EINVAL before anything
 *   is launched (the kernels use 16-byte vector accesses and bulk copies).
 * - The context and key objects own their device memory (allocated with the
 *   CUDA stream-ordered allocator) and release it in *_destroy.
 * - There is no CPU fallback: without a usable CUDA device every call that
 *   needs one returns SECPE_ECUDA.
 * - A context serves one host thread at a time: every call that takes a
 *   stream records it in the context (its temporaries are allocated and
 *   freed on it, its launches and profiler events go to it) for the duration
 *   of the call, and the counters, profiler and device status word are
 *   per context.  Calls from several host threads on one context must be
 *   serialised by the caller; use one context per thread (or per stream) to
 *   run them concurrently.  Successive calls on different streams are fine
 *   when the caller orders the streams (events) wherever one call's outputs
 *   are another's inputs.
 */
#ifndef SECPE_H
#define SECPE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SECPE_OK 0
#define SECPE_EINVAL -1   /* bad argument (sizes, levels, pointers) */
#define SECPE_ENOMEM -2   /* device allocation failed */
#define SECPE_ELEVEL -3   /* not enough levels for the operation */
#define SECPE_ESCALE -4   /* operand scales differ */
#define SECPE_EKEY -5     /* a needed Galois / relinearisation key is missing */
#define SECPE_ECUDA -6    /* CUDA runtime error */
#define SECPE_ETIMEOUT -7 /* a bounded device-side wait gave up */
#define SECPE_EADMIT -8   /* request does not fit the admission budget */

/* Rotation "step" naming the complex conjugation of the slots (Galois
 * element 2N - 1) in secpe_keygen and secpe_rotate. */
#define SECPE_STEP_CONJ 0x40000000

/*
 * Parameter set.  Ring R_Q = Z_Q[X]/(X^N + 1), Q = q_0 ... q_L (SecPE
 * Sec. 2.2).  Primes (all = 1 mod 2N, all below 2^60):
 *   special primes: the n_p largest below 2^p_bits;
 *   q_0: the largest below 2^q0_bits not already taken when q0_bits differs
 *        from q_bits, otherwise the first prime of the sequence below;
 *   q_1..: alternately the nearest below and above 2^q_bits, below first;
 *   with boot_primes = b > 0, the top b primes q_(L-b+1)..q_L are instead
 *        the b largest below 2^boot_bits (taken after the special primes,
 *        before q_0), in decreasing order.
 * Key switching is hybrid with dnum digits of alpha = ceil(n_q/dnum) primes.
 * Sign = f^sign_df(g^sign_dg(x)) (SecPE Eq. comp); `reserve` levels are
 * kept below each depth-4 polynomial block before a refresh is forced.
 */
typedef struct {
    int32_t log_n;      /* 12..16 on the fast paths; 4..17 accepted */
    int32_t q0_bits;
    int32_t q_bits;
    int32_t n_q;        /* number of ciphertext primes, L + 1 (<= 48) */
    int32_t p_bits;
    int32_t n_p;        /* number of special primes (1..8) */
    int32_t dnum;       /* digits; dnum <= 15 and alpha <= 15 */
    int32_t log_scale;  /* scale Delta = 2^log_scale */
    int32_t sign_dg;    /* repetitions of g (paper: 2) */
    int32_t sign_df;    /* repetitions of f (paper: 2) */
    int32_t reserve;    /* levels kept in reserve (>= 1) */
    int32_t secret_hw;  /* 0: uniform ternary secret; h > 0: sparse ternary
                           secret with exactly h nonzero coefficients (the
                           bound on the ModRaise overflow that
                           bootstrapping's modular reduction needs) */
    int32_t boot_primes; /* 0, or the number of top ciphertext primes
                            (q_(L-boot_primes+1)..q_L) of boot_bits bits that
                            bootstrapping's levels use */
    int32_t boot_bits;
} secpe_params;

typedef struct secpe_ctx secpe_ctx;   /* primes, NTT tables, base-conversion tables */
typedef struct secpe_keys secpe_keys; /* secret key (device), relin + Galois keys */

typedef struct {
    uint64_t *data;   /* device, [2][cap][N] */
    int32_t level;    /* limbs 0..level valid */
    int32_t cap;      /* allocated limbs per polynomial */
    double scale;     /* CKKS scale of the encoded message */
} secpe_ct;

/* ---- context ---------------------------------------------------------- */
/* Builds primes/roots/tables on the host and uploads them to the current
 * device.  The prime values can be read back with secpe_ctx_primes. */
int secpe_ctx_create(const secpe_params *p, secpe_ctx **out);
void secpe_ctx_destroy(secpe_ctx *ctx);
/* Copies the n_q ciphertext primes then the n_p special primes to out
 * (host array of n_q + n_p words). */
int secpe_ctx_primes(const secpe_ctx *ctx, uint64_t *out);
/* Host-only (no device needed): runs the prime selection rule above and
 * writes n_q ciphertext primes then n_p special primes into out, which must
 * hold `capacity` >= n_q + n_p words.  Returns SECPE_EINVAL for parameters
 * outside the supported ranges. */
int secpe_select_primes(const secpe_params *p, uint64_t *out, int capacity);
int secpe_ctx_n(const secpe_ctx *ctx);
/* Device-side status word (0 = ok, else a SECPE_E* recorded by a kernel);
 * synchronises `stream` first, then clears the word. */
int secpe_stream_status(secpe_ctx *ctx, void *stream, int *device_status);
/* Self-test of the bounded device-side wait that the kernels with bulk
 * copies use: a one-CTA kernel arms a shared-memory mbarrier for one arrival,
 * performs that arrival only when `arrive` is non-zero, and waits for it with
 * at most `polls` polls (1 .. 4194304).  Without the arrival the wait runs
 * out, the kernel records SECPE_ETIMEOUT in the status word (read it with
 * secpe_stream_status) and returns; the context stays usable.  Nothing
 * faults, traps or hangs. */
int secpe_device_wait_selftest(secpe_ctx *ctx, int arrive, int64_t polls, void *stream);
const char *secpe_strerror(int code);

/* ---- keys ------------------------------------------------------------- */
/* Key generation of the RNS-CKKS scheme (SecPE Sec. 2.2; the user holds the
 * secret key, Sec. 3.1 step 1, the server the evaluation keys, step 3).
 * Secret key s (ternary; with secret_hw = h > 0, sparse: word c = 0, 1, ..
 * of the secret's stream puts sign (w & 1 ? -1 : +1) at position
 * (w >> 1) mod N unless that position is taken, until h are placed),
 * relinearisation key (s^2 -> s) and one Galois key per rotation step in
 * rot_steps (r > 0: RotL by r; r < 0: RotR by -r; SECPE_STEP_CONJ: the
 * complex conjugation of the slots, X -> X^(2N-1)), all drawn from the
 * counter-based SplitMix64 streams of `seed` (same streams as the CPU
 * oracle).  The keys object owns its device memory (about
 * dnum * 2 * (n_q + n_p) * N words per key); steps are taken modulo N/2.
 * Synchronous; SECPE_EINVAL for null pointers or n_rot < 0, SECPE_ENOMEM or
 * SECPE_ECUDA when the keys cannot be allocated. */
int secpe_keygen(secpe_ctx *ctx, uint64_t seed, const int32_t *rot_steps, int n_rot,
                 secpe_keys **out);
void secpe_keys_destroy(secpe_keys *keys);
/* Copies key material to host, converted to plain residues: which = 0
 * secret key NTT form [n_q+n_p][N]; which = 1 relinearisation key
 * [dnum][2][n_q+n_p][N]; which = 2 Galois key of rotation step `step`. */
int secpe_keys_export(const secpe_ctx *ctx, const secpe_keys *keys, int which, int32_t step,
                      uint64_t *host_out, size_t words);

/* ---- client side: encode + encrypt, decrypt + decode ------------------- */
/* Secret-key encryption (reading of SecPE Sec. 3.1 step 1) of integer
 * coefficients m[N] (host int64) at `level` with metadata `scale`:
 * c1 = a, c0 = -a*s + m + e, randomness from the streams of `seed`. */
int secpe_encrypt_coeffs(secpe_ctx *ctx, const secpe_keys *keys, const int64_t *m, int level,
                         double scale, uint64_t seed, secpe_ct *out, void *stream);
/* Encodes n real values into slots 0..n-1 (canonical embedding, slot j at
 * zeta^(5^j); host FP64) and encrypts them at the top level, scale Delta. */
int secpe_encrypt(secpe_ctx *ctx, const secpe_keys *keys, const double *v, int n, uint64_t seed,
                  secpe_ct *out, void *stream);
/* One prompt's logits (SecPE Sec. 3.1 step 1 / Eq. argmax layout): slots
 * 0..C-1 hold v, slots C..C'-1 hold d_min (C' = next power of two), zeros
 * beyond.  SECPE_EINVAL for C < 1 or C' > N/2. */
int secpe_encrypt_logits(secpe_ctx *ctx, const secpe_keys *keys, const double *v, int C,
                         double d_min, uint64_t seed, secpe_ct *out, void *stream);
/* Slot packing (SecPE Sec. 3.2, the paragraph after Alg. 1: one ciphertext
 * of N/2 slots carries the inputs of several queries that share the task,
 * i.e. the class count C and the prompt ensemble, and Alg. 1 runs on all of
 * them at once).  Query b of P occupies the block of 2C' slots starting at
 * slot 2C'b (C' = next power of two >= C): its C logits, then d_min up to
 * C', then C' zeros, the room the duplication y + RotR(y, C') fills.
 * Rotations by C' and by 2^i < C' keep every window Alg. 1 reads inside the
 * block, so after secpe_argmax_batch / secpe_encrypted_argmax (with C, one
 * query per packed ciphertext set) block b's first C slots hold query b's
 * z.  The K prompts of a packed query are K packed ciphertexts (prompt i of
 * every packed input in ciphertext i); K, d_min, d_max are shared.
 *
 * secpe_packed_capacity: inputs per ciphertext, N / (4 C') (0 when one block
 * does not fit); host only.  SECPE_EINVAL for log_n outside 4..17 or C < 1. */
int secpe_packed_capacity(int log_n, int C);
/* Host only: the integer coefficients m[N] of the packed slot vector of
 * v[P][C] (row-major) at scale `scale`: the canonical embedding of
 * secpe_encrypt computed in O(N log N) by a length-N complex DFT over the
 * odd powers of zeta (equal to the direct sums up to floating-point
 * rounding), rounded half away from zero.  SECPE_EINVAL for P outside
 * 1..capacity or a coefficient beyond 2^62. */
int secpe_encode_packed(int log_n, double scale, const double *v, int P, int C, double d_min, int64_t *m_out);
/* Host only: the first C slots of each of the P blocks, out[P][C], from
 * centred coefficients (secpe_decrypt_coeffs) divided by `scale`. */
int secpe_decode_packed(int log_n, double scale, const double *coeffs, int P, int C, double *out);
/* secpe_encode_packed + secpe_encrypt_coeffs at the top level, scale Delta. */
int secpe_encrypt_logits_packed(secpe_ctx *ctx, const secpe_keys *keys, const double *v, int P, int C,
                                double d_min, uint64_t seed, secpe_ct *out, void *stream);
/* Decrypts a packed result: out[P][C] (host) = the first C slots of every
 * block.  Synchronous. */
int secpe_decrypt_packed(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ct *ct, int P, int C, double *out,
                         void *stream);
/* Seeded ciphertexts (a transport form of the user's encryption, Sec. 3.1
 * step 1): c1 of a fresh encryption is the uniform polynomial
 * drawn from the stream of its encryption seed, so a client can send c0 and
 * the 8-byte seed only.  This regenerates c1 (limbs 0..level) on the device
 * for `batch` ciphertexts at base + i*ct_stride words ([2][cap][N] each),
 * seeds[i] being ciphertext i's encryption seed; the result is bit-identical
 * to the ciphertext secpe_encrypt* produced. */
int secpe_expand_seeded(secpe_ctx *ctx, uint64_t *base, int batch, size_t ct_stride, int cap, int level,
                        const uint64_t *seeds, void *stream);
/* Decryption and decoding by the user (SecPE Sec. 3.1 step 4; Sec. 2.2 Dec
 * and the canonical-embedding decoding): m = c0 + c1 s over the ciphertext's
 * limbs, exact CRT to centred integers, slots 0..n-1 (slot j at
 * zeta^(5^j)) divided by the ciphertext's scale, to host doubles (v_out[n]).
 * Synchronous; SECPE_EINVAL for n outside 0..N/2. */
int secpe_decrypt(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ct *ct, double *v_out,
                  int n, void *stream);
/* Centred coefficients of c0 + c1*s as doubles (host, N values). */
int secpe_decrypt_coeffs(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ct *ct,
                         double *coeffs_out, void *stream);

/* ---- primitives (SecPE Sec. 2.2 operation list) ------------------------ */
/* Forward (inverse = 0) or inverse negacyclic NTT, in place, of `count`
 * limbs: limb k is at limbs + k*N, taken modulo the prime of index
 * prime_idx[k] (host array; 0..n_q-1 ciphertext primes, n_q.. special).
 * Forward: out[j] = sum_k a[k] psi^((2 brv(j) + 1) k), bit-reversed order. */
int secpe_ntt(secpe_ctx *ctx, uint64_t *limbs, const int32_t *prime_idx, int count, int inverse,
              void *stream);
/* Same transform on `batch` ciphertexts laid out contiguously with a stride
 * of `ct_stride` words: both polynomials, limbs 0..level. */
int secpe_ntt_cts(secpe_ctx *ctx, uint64_t *base, int batch, size_t ct_stride, int cap, int level,
                  int inverse, void *stream);
/* Precision variant (N = 2^16 only): the same transforms, bit-identical,
 * computed as exact dense contractions on the tensor pipe.  The transform of
 * the ring R_Q (Sec. 2.2) factors into a fixed 256 x 256 matrix per prime on
 * every column, an element-wise twist, and a fixed 256 x 256 matrix per
 * prime on every row (the inverse in reverse order).  Each matrix product
 * splits residues and matrix entries into 8-bit limbs, forms u8 x u8 -> s32
 * products and recombines the diagonal sums modulo q.  The first call on a
 * context builds the matrices and twists (3 MiB per prime).  Scratch (the
 * byte planes, 512 KiB per limb, at most 1 GiB) comes from the stream-ordered
 * allocator. */
int secpe_ntt_tc(secpe_ctx *ctx, uint64_t *limbs, const int32_t *prime_idx, int count, int inverse,
                 void *stream);
/* secpe_ntt_cts on the tensor pipe: same layout and arguments, bit-identical. */
int secpe_ntt_cts_tc(secpe_ctx *ctx, uint64_t *base, int batch, size_t ct_stride, int cap, int level,
                     int inverse, void *stream);
/* Homomorphic addition and subtraction (SecPE Sec. 2.2, the slot-wise sum of
 * the aggregation, Sec. 3.1 step 3): out = a + b or a - b limb by limb at
 * level min(level_a, level_b), scale of a; out may be a or b.  SECPE_ESCALE
 * when the scales differ by more than 2^-40 relative. */
int secpe_add(secpe_ctx *ctx, const secpe_ct *a, const secpe_ct *b, secpe_ct *out, void *stream);
int secpe_sub(secpe_ctx *ctx, const secpe_ct *a, const secpe_ct *b, secpe_ct *out, void *stream);
/* out = a * c landing at out_level with scale exactly `target_scale`
 * (constant round(c * target/scale_a * q_{out_level+1}), then rescale). */
int secpe_mul_const(secpe_ctx *ctx, const secpe_ct *a, double c, double target_scale,
                    int out_level, secpe_ct *out, void *stream);
/* out = a + c in every slot (Sec. 2.2 addition of a plaintext constant, as in
 * Alg. 1's final + 1): c encodes as the constant polynomial round(c * scale)
 * added to c0; level and scale of a.  SECPE_EINVAL if |c * scale| >= 4e18. */
int secpe_add_const(secpe_ctx *ctx, const secpe_ct *a, double c, secpe_ct *out, void *stream);
/* Homomorphic product (SecPE Sec. 2.2 Mult): tensor, relinearise by hybrid
 * key switching with the relinearisation key, rescale; out at level
 * min(level_a, level_b) - 1 with scale s_a s_b / q_l.  SECPE_ELEVEL when
 * the inputs' level is below 1 + reserve, SECPE_EKEY without a key. */
int secpe_mul_relin(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ct *a, const secpe_ct *b,
                    secpe_ct *out, void *stream);
/* Rescale (SecPE Sec. 2.2: after a product the scale is divided by the last
 * prime q_l): rounded division (c + floor(q_l/2) - [c + floor(q_l/2)]_{q_l})
 * / q_l of every coefficient, out at level l - 1 with scale s / q_l; out
 * may alias in.  SECPE_ELEVEL at level 0. */
int secpe_rescale(secpe_ctx *ctx, const secpe_ct *in, secpe_ct *out, void *stream);
/* Same result as secpe_rescale (bit for bit), for callers that may not
 * allocate device memory during a call: serving loops that must keep a
 * fixed device-memory footprint and keep the allocator off their critical
 * path, and host frameworks that own all device memory and forbid hidden
 * allocations.  The paper has no counterpart: this is a deployment
 * variant.  Its scratch is a fixed file-scope device array of
 * 2 * 65536 * 24 words (24 MiB) that every GPU loading the library keeps
 * until exit; a call needs 2 * N * (level + 1) words and returns
 * SECPE_EINVAL beyond that (N = 2^16: level <= 23).  Under CUDA's default
 * lazy module loading the array is reserved on a device by the first call
 * there (its set-up looks up the array's device address and loads the
 * module), so that call can fail with SECPE_ECUDA on a full device: make one
 * warm-up call per device at start-up, before admitting requests and before
 * any stream capture.  After it, no cudaMalloc/cudaFree or other allocating
 * call is made.  All calls share the array: calls that may overlap on the
 * GPU race and must not be issued.  Errors as secpe_rescale (SECPE_ELEVEL
 * at level 0).  out may be in itself (same data and cap); any other overlap
 * of the two buffers returns SECPE_EINVAL. */
int secpe_rescale_noalloc(secpe_ctx *ctx, const secpe_ct *in, secpe_ct *out, void *stream);
/* Rotation of the slot vector (SecPE Sec. 2.2 RotL / RotR, used by Alg. 1):
 * RotL(in, steps) for steps > 0, RotR(in, -steps) for steps < 0, as the
 * automorphism X -> X^(5^steps) followed by hybrid key switching with the
 * Galois key of that step; out at in's level and scale (out may alias in).
 * SECPE_EKEY when the key was not generated. */
int secpe_rotate(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ct *in, int steps,
                 secpe_ct *out, void *stream);
/* Rotations of one ciphertext by every steps[i] (i < count, count <= 64)
 * into outs[i] (caller buffers, cap >= in's level + 1, none aliasing in),
 * sharing one ModUp of in's second polynomial (hoisting, as bootstrapping's
 * baby steps use it): per step the automorphism goes onto both polynomials
 * and onto every extended limb, then the key inner product and ModDown.  Each
 * result decrypts like secpe_rotate's with the same noise bound (its
 * residues differ: the extended limbs carry FastBConv's multiple of the
 * digit modulus, permuted).  SECPE_EKEY for a missing Galois key. */
int secpe_rotate_hoisted(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ct *in, const int32_t *steps,
                         int count, secpe_ct *outs, void *stream);
/* Hybrid key switching of one polynomial d ([cap][N], limbs 0..level, NTT
 * form) with the relinearisation key (galois_step = 0) or the Galois key of
 * a rotation step: writes ks0, ks1 ([cap][N] each). */
int secpe_keyswitch(secpe_ctx *ctx, const secpe_keys *keys, int galois_step, const uint64_t *d,
                    int level, int cap, uint64_t *ks0, uint64_t *ks1, void *stream);
/* Test-only, INSECURE stand-in for bootstrapping (SecPE Sec. 2.2 and Sec. 4.1
 * rely on bootstrapping to restore levels without describing it): decrypt
 * with the secret key held by the keys object, exact CRT lift, re-encrypt at
 * the top level with the same scale; randomness from the stream (qseed,
 * refresh_index).  It makes the evaluation interactive and must not be used
 * where the server may not see plaintexts. */
int secpe_refresh_testonly(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ct *in,
                           uint64_t qseed, uint64_t refresh_index, secpe_ct *out, void *stream);

/* ---- batched primitives -------------------------------------------------- */
/* The primitives of SecPE Sec. 2.2 (key switching, product + relinearisation
 * + rescale, rotation, rescale) on `batch` ciphertexts at once, each launch
 * serving all of them: batch ciphertexts at data + i*stride (words), each
 * [2][cap][N], all at the same level and scale.  Outputs are written to
 * caller memory with the same conventions; the output level/scale fields
 * are set by the call. */
typedef struct {
    uint64_t *data;
    int32_t batch;
    int32_t cap;
    int32_t level;
    double scale;
    uint64_t stride;  /* words between items, >= 2*cap*N */
} secpe_ctbatch;
/* Hybrid key switching (the ModUp, key inner product and ModDown behind
 * Sec. 2.2's relinearisation and rotations) of polynomial 0 of every item
 * of d (limbs 0..level); item i of out receives (ks0, ks1) in its
 * polynomials 0 and 1 at d's level.  galois_step 0 selects the
 * relinearisation key, any other value the Galois key of that rotation
 * (SECPE_EKEY if it was not generated).  SECPE_EINVAL for batch outside
 * 1..1024, a bad layout, or out->batch != d->batch. */
int secpe_keyswitch_batch(secpe_ctx *ctx, const secpe_keys *keys, int galois_step, const secpe_ctbatch *d,
                          secpe_ctbatch *out, void *stream);
/* Precision variant of secpe_keyswitch_batch (N = 2^16, dnum <= 8): every
 * NTT/INTT of the key switch runs as the exact tensor-pipe contraction of
 * secpe_ntt_tc, and the key inner product sum_j x_j k_{j,s} over the digits
 * as exact 8-bit-limb u8 x u8 -> s32 products on the tensor pipe (one
 * product per coefficient: rows = (output polynomial, diagonal), columns =
 * items); the base conversions of ModUp and ModDown stay on CUDA cores.
 * The result is bit-identical to secpe_keyswitch_batch.  Same arguments,
 * layout and errors; SECPE_EINVAL for other ring sizes or dnum > 8. */
int secpe_keyswitch_batch_tc(secpe_ctx *ctx, const secpe_keys *keys, int galois_step, const secpe_ctbatch *d,
                             secpe_ctbatch *out, void *stream);
/* secpe_mul_relin on item i of a and item i of b for every i, one launch
 * per step for the whole batch; errors as secpe_mul_relin, plus
 * SECPE_EINVAL for batch outside 1..1024 or a bad layout. */
int secpe_mul_relin_batch(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ctbatch *a,
                          const secpe_ctbatch *b, secpe_ctbatch *out, void *stream);
/* secpe_rotate (RotL for steps > 0, RotR for steps < 0) of every item. */
int secpe_rotate_batch(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ctbatch *in, int steps,
                       secpe_ctbatch *out, void *stream);
/* secpe_rescale of every item (SECPE_ELEVEL at level 0). */
int secpe_rescale_batch(secpe_ctx *ctx, const secpe_ctbatch *in, secpe_ctbatch *out, void *stream);

/* ---- bootstrapping --------------------------------------------------------- */
/* SecPE Sec. 2.2 and Sec. 4.1 rely on bootstrapping to restore a
 * ciphertext's levels (depth 14 at N = 2^16) without describing it; this is
 * the sparse-slot CKKS bootstrapping of Cheon, Han, Kim, Kim and Song (2018)
 * with the sub-sum of Chen, Chillotti and Song (2019), for a block of n
 * slots (n a power of two, 2n <= N/2):
 *   ModRaise of limb 0 to the top level; SubSum (rotations by n .. N/4);
 *   CoeffToSlot (baby-step giant-step plaintext diagonals of the slots and
 *   their conjugate: u = coefficient / q0 in slots [0, 2n) of every block);
 *   EvalMod (sin(2 pi u) from the degree-12 Taylor polynomial of
 *   cos(2 pi (u - 1/4) / 256) and 8 double angles); SlotToCoeff.
 * It needs a context with secret_hw in 1..32 (the ModRaise overflow bound)
 * and boot_primes >= 16 (its levels: 1 + 14 + 1, at the top), and the
 * Galois keys of secpe_boot_rotation_steps (conjugation included).  The
 * result is at level L - 16 with the input's label and decrypts to the
 * n-periodic block average of the input's slots: an n-periodic input (a
 * block of n slots repeated over the N/2 slots, e.g. a query packed into
 * every block by secpe_encrypt_logits_packed) comes back unchanged.
 * Non-interactive: no secret key is used.
 *
 * secpe_boot_rotation_steps: the rotation steps the keys need (host only);
 * with steps null only *count is written. */
typedef struct secpe_boot secpe_boot;
int secpe_boot_rotation_steps(const secpe_ctx *ctx, int n, int32_t *steps, int capacity, int *count);
/* Builds the plaintext diagonals with the library's encoder (2n for
 * CoeffToSlot at scale q_L, 2n for SlotToCoeff) and uploads them (device
 * memory owned by the plan: 2n (L + 1) + 2n (L - 14) limbs of N words). */
int secpe_boot_create(secpe_ctx *ctx, int n, secpe_boot **out);
/* The same from integer coefficients chosen by the caller: c2s_m[2][n][N]
 * (the diagonals of the slots then of their conjugate, diagonal g bs + b
 * rotated right by g bs, at scale q_L) and s2c_m[2n][N] (at scale
 * q_(L-15) / label of the EvalMod output). */
int secpe_boot_create_coeffs(secpe_ctx *ctx, int n, const int64_t *c2s_m, const int64_t *s2c_m,
                             secpe_boot **out);
void secpe_boot_destroy(secpe_boot *bt);
/* Bootstraps `batch` ciphertexts (any level; limb 0 is used) as one batch:
 * every evaluator launch serves the whole batch.  out->level/scale/batch
 * are set.  SECPE_EKEY for a missing rotation key. */
int secpe_bootstrap_batch(secpe_ctx *ctx, const secpe_keys *keys, const secpe_boot *bt, const secpe_ctbatch *in,
                          secpe_ctbatch *out, void *stream);
int secpe_bootstrap(secpe_ctx *ctx, const secpe_keys *keys, const secpe_boot *bt, const secpe_ct *in,
                    secpe_ct *out, void *stream);

/* ---- word-size probe: 32-bit residues ----------------------------------- */
/* The negacyclic NTT and the fast base conversion (the RNS primitives of
 * SecPE Sec. 2.2's CKKS) on 32-bit words, for primes q < 2^30 with
 * q = 1 mod 2N: a measurement of the word size against the 64-bit path,
 * with up to 128 primes per table (the circuit itself runs on 64-bit
 * residues).  N = 2^16 only (log_n = 16).  The table holds the twiddles
 * (device memory owned by it, 1 MiB per prime).  SECPE_EINVAL for another
 * N or a prime that is not NTT-friendly, SECPE_ECUDA if allocation fails. */
typedef struct secpe_ntt32_table secpe_ntt32_table;
int secpe_ntt32_create(int log_n, const uint32_t *primes, int n_primes, secpe_ntt32_table **out);
void secpe_ntt32_destroy(secpe_ntt32_table *t);
/* In place on `count` limbs of N words at limbs + i N (device, 16-byte
 * aligned), limb i under prime prime_idx[i] (host array, indices into the
 * table).  Forward: natural order in, bit-reversed order out (psi^brv
 * twiddles, as secpe_ntt); inverse: the exact inverse.  Values in [0, q). */
int secpe_ntt32(const secpe_ntt32_table *t, uint32_t *limbs, const int32_t *prime_idx, int count, int inverse,
                void *stream);
/* FastBConv of coefficient-form limbs: for each of `batch` items, in
 * [batch][n_in][N] under the distinct primes in_idx[n_in] (Q their product)
 * to out [batch][n_out][N] under out_idx[n_out]:
 * out_j = sum_i [x_i Qhat_i^-1]_{q_i} [Qhat_i]_{p_j} mod p_j, Qhat_i = Q/q_i
 * (no correction of the multiple of Q it may add).  n_in <= 16,
 * n_out <= 64; device buffers, 16-byte aligned. */
int secpe_bconv32(const secpe_ntt32_table *t, const uint32_t *in, const int32_t *in_idx, int n_in, uint32_t *out,
                  const int32_t *out_idx, int n_out, int batch, void *stream);
/* Hybrid key switching on 32-bit residues (the steps of secpe_keyswitch):
 * for `batch` polynomials d [batch][nq][N] (NTT form, primes q_idx), the
 * key [dnum][2][nq + np][N] (plain residues, limbs in the order q_idx then
 * p_idx; digit j = the q primes [j alpha, (j+1) alpha), dnum = ceil(nq /
 * alpha)), out [batch][2][nq][N] = ModDown(sum_j ModUp_j(d) * key_j) with
 * ModDown the rounded division by P = prod of the p_idx primes.  nq + np <=
 * 64, alpha <= 16, np <= 16, primes distinct; device buffers 16-byte
 * aligned; temporary device memory from the stream-ordered allocator.
 * fused = 0: one launch per step (INTT, FastBConv per digit, NTT, inner
 * product); fused = 1: the conversion inside the NTT's column pass and the
 * inner product inside its row pass, as on the 64-bit path (at most 256
 * extended limbs per item).  Both give the same residues. */
int secpe_keyswitch32(const secpe_ntt32_table *t, const uint32_t *d, const int32_t *q_idx, int nq,
                      const int32_t *p_idx, int np, int alpha, const uint32_t *key, uint32_t *out, int batch,
                      int fused, void *stream);

/* ---- SecPE circuit ----------------------------------------------------- */
/* Sign(x) = f^df(g^dg(x)) (SecPE Eq. comp), each degree-9 polynomial by a
 * depth-4 baby-step giant-step DAG; refreshes (counter from *refresh_index,
 * advanced) when fewer than 4 (+ out_levels for the last) levels remain. */
int secpe_sign(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ct *x, int out_levels,
               uint64_t qseed, uint64_t *refresh_index, secpe_ct *out, void *stream);
/* Max(a, y) = (a+y)/2 + (a-y)/2 * Sign(a-y) (SecPE Eq. max). */
int secpe_max(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ct *a, const secpe_ct *y,
              uint64_t qseed, uint64_t *refresh_index, secpe_ct *out, void *stream);
/* Ensemble aggregation (SecPE Sec. 3.1 step 3, Eq. norm scale):
 * out = (sum of the K cts) * 1/(K (d_max - d_min)) at level L-1, scale Delta. */
int secpe_ensemble_aggregate(secpe_ctx *ctx, const secpe_ct *cts, int K, double d_min,
                             double d_max, secpe_ct *out, void *stream);
/* SecPE Alg. 1 on a normalised ciphertext y with C >= 2 classes: returns z
 * with z ~ 1 at the argmax slot and ~ 0 at the other slots 0..C-1.
 * Needs Galois keys for RotR(C') and RotL(2^i), i < log2 C' (SECPE_EKEY
 * otherwise).  Levels follow secpe_level_plan (refresh level L).
 * SECPE_EINVAL for C < 2 or 2 C' > N/2 (no room for the duplicated copy). */
int secpe_encrypted_argmax(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ct *y, int C,
                           uint64_t qseed, secpe_ct *z_out, void *stream);

/* ---- upstream encrypted linear step (CLIP-style prompt ensembling) ------- */
/* SecPE Sec. 2.3 scores an image embedding x = I(x_in) (d values) against
 * the text embedding T_i[c] of prompt template i and class c, y_i[c] =
 * <T_i[c], x>, and aggregates the K logit vectors before the Argmax
 * (Sec. 3.1 step 3); here x is encrypted and the T_i are the server's
 * plaintext weights.  Layout (d a power of two, C' = next power of two >= C,
 * d C' <= N/2): the user encrypts x with x[j] repeated in the C' slots
 * [j C', (j+1) C') (secpe_encrypt_replicated); for each prompt the server
 * multiplies by the plaintext with T_i[c][j] at slot j C' + c (encoded at
 * scale q_L), adds log2(d) rotations by C' 2^t, multiplies by a plaintext
 * mask (1 on slots [0, C), scale q_(L-1)) and adds a plaintext with d_min on
 * [C, C') (scale Delta).  Each output is the layout secpe_encrypt_logits
 * produces, at level L - 2 with x's scale, ready for secpe_argmax_batch.
 * Needs Galois keys for C' 2^t, t < log2 d. */
typedef struct secpe_linear secpe_linear;
/* Encodes T[K][C][d] (host, row-major) with the packed encoder and uploads
 * the K weight plaintexts, the mask and the pad (device memory owned by the
 * object, about (K (L+1) + 2L) N words).  SECPE_EINVAL for d not a power of
 * two or d C' > N/2. */
int secpe_linear_create(secpe_ctx *ctx, const double *T, int K, int C, int d, double d_min, secpe_linear **out);
/* The same from integer coefficients chosen by the caller: W_m[K][N] at
 * scale q_L, mask_m[N] at scale q_(L-1), pad_m[N] at scale Delta. */
int secpe_linear_create_coeffs(secpe_ctx *ctx, const int64_t *W_m, const int64_t *mask_m, const int64_t *pad_m,
                               int K, int C, int d, secpe_linear **out);
void secpe_linear_destroy(secpe_linear *lin);
/* outs[K] (caller device buffers, cap >= L - 1) = the K prompts' logit
 * ciphertexts of x (level L, scale Delta); the K prompts run as one batch.
 * SECPE_ELEVEL / SECPE_ESCALE for other inputs, SECPE_EKEY for a missing
 * rotation key. */
int secpe_linear_apply(secpe_ctx *ctx, const secpe_keys *keys, const secpe_linear *lin, const secpe_ct *x,
                       secpe_ct *outs, void *stream);
/* Client: encrypts x[d] with x[j] in the C' slots [j C', (j+1) C'), top
 * level, scale Delta (packed encoder). */
int secpe_encrypt_replicated(secpe_ctx *ctx, const secpe_keys *keys, const double *x, int d, int C, uint64_t seed,
                             secpe_ct *out, void *stream);

/* Level plan of Alg. 1 (host only; level-aware QuickMax, a reading: SecPE
 * does not discuss levels).  Alg. 1 for C >= 2 classes on y at entry_level
 * (the aggregation's output level), evaluated greedily with refreshes that
 * return refresh_level (a refresh comes before a step that lacks its levels:
 * a QuickMax round needs 1 + reserve, each Sign polynomial 4 + reserve, the
 * last of Max's Sign 5 + reserve), falls into ranges: the first starts at
 * y, each refresh starts the next.  Range by range, in order, each range's
 * first ciphertext is dropped to the lowest level at which every refresh
 * still comes at the same step and the refreshed step keeps its levels (a
 * lower start never raises a later level, so one level at a time finds
 * it): the refresh count is unchanged and every step runs on at most as
 * many limbs.
 * targets[capacity] receives the levels of y entering round 0 (j = 0) and
 * of the ciphertext right after refresh j; *count = refreshes + 1 (with
 * targets null only *count is written).  secpe_encrypted_argmax,
 * secpe_argmax_batch and the server follow it with refresh_level = L, and
 * secpe_argmax_batch_boot with L - 16.  SECPE_EINVAL for bad arguments
 * (log_n outside 4..17, C above N/4, which leaves no room for the 2 C'
 * slots of Alg. 1) or capacity < *count, SECPE_ELEVEL if a refresh leaves
 * too few levels. */
int secpe_level_plan(const secpe_params *p, int C, int entry_level, int refresh_level, int32_t *targets,
                     int capacity, int *count);

/* One ensemble query for the batched driver. */
typedef struct {
    const secpe_ct *cts;  /* K input ciphertexts (top level, scale Delta) */
    int32_t K;
    int32_t C;
    double d_min, d_max;
    uint64_t qseed;       /* refresh randomness */
    secpe_ct *z_out;      /* output ciphertext (cap >= top level + 1) */
    const secpe_keys *keys; /* the query's tenant key set; null = the call's (or server's) keys */
} secpe_query;

/* Aggregation + Argmax of n_queries independent queries, batched: every
 * homomorphic operation runs once for all queries that take it at that
 * point of the circuit.  Queries of different tenants (q[i].keys) are
 * evaluated as one batch per key set, in order of first appearance.
 * Results equal the one-query calls with the query's keys bit for bit. */
int secpe_argmax_batch(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q,
                       int n_queries, void *stream);
/* SecPE Alg. 1 without the interactive stand-in: secpe_argmax_batch where
 * every refresh is a bootstrap of the refreshed batch with plan `bt` (its
 * block n must be a multiple of 2C' of every query).  Each query's inputs
 * must be 2C'-periodic (its logits packed into every block of 2C' slots,
 * secpe_encrypt_logits_packed with N/(4C') copies), so every intermediate
 * is periodic and each bootstrap returns it unchanged.  For a context with
 * bootstrapping primes the inputs sit at the top computation level L - 16 or
 * below (the bootstrap returns there); errors as secpe_argmax_batch and
 * secpe_bootstrap_batch. */
int secpe_argmax_batch_boot(secpe_ctx *ctx, const secpe_keys *keys, const secpe_boot *bt, const secpe_query *q,
                            int n_queries, void *stream);

/* The baseline SecPE compares its Argmax with (Sec. 3.2, Phoenix): after the
 * same duplication y + RotR(y, C'), every slot is compared with its
 * m = C' - 1 cyclic neighbours, s = sum_{i=1..m} Sign(y - RotL(y, i)); the
 * max slot has s = m and every other s <= m - 2, so
 * z = (Sign((s - (m - 1)) / (2m)) + 1) / 2: m + 1 Signs and m + 1 rotations
 * against SecPE's log2 C' + 1 of each.  The m comparisons start from the
 * same ciphertext and run as one batch.  Comparison i draws its refresh
 * randomness from the seed stream(qseed, 7, i), the final Sign from
 * stream(qseed, 7, 0).  Needs Galois keys for RotR(C') and RotL(i),
 * i = 1..C'-1 (SECPE_EKEY otherwise).  Same conventions as
 * secpe_encrypted_argmax; z ends at the reserve level. */
int secpe_phoenix_argmax(secpe_ctx *ctx, const secpe_keys *keys, const secpe_ct *y, int C, uint64_t qseed,
                         secpe_ct *z_out, void *stream);
/* Aggregation + the Phoenix Argmax of n_queries queries, batched like
 * secpe_argmax_batch (one batch per key set and C'); results equal
 * secpe_ensemble_aggregate + secpe_phoenix_argmax per query bit for bit. */
int secpe_phoenix_argmax_batch(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q, int n_queries,
                               void *stream);

/* Graph-captured batched Argmax.  secpe_argmax_batch_capture records the
 * whole evaluation of secpe_argmax_batch for these queries (every launch,
 * stream-ordered allocation and copy) into one CUDA graph, on a stream of its
 * own, without running it, and instantiates it; the z_out level/scale fields
 * are set as a run would set them.  The graph keeps the device addresses of
 * the queries' ciphertexts, z_out buffers and keys: the caller keeps them
 * alive and may rewrite the input ciphertexts in place (same level, scale,
 * layout) between launches.  secpe_graph_launch replays it on `stream` (one
 * launch for the whole batch) and adds the captured operation and kernel
 * counts to the context counters.  *n_nodes (if not null) receives the
 * graph's node count.  Errors: those of secpe_argmax_batch, SECPE_ECUDA when
 * capture or instantiation fails. */
typedef struct secpe_graph secpe_graph;
int secpe_argmax_batch_capture(secpe_ctx *ctx, const secpe_keys *keys, const secpe_query *q, int n_queries,
                               secpe_graph **out, int64_t *n_nodes);
int secpe_graph_launch(secpe_graph *g, void *stream);
/* Synchronises the device, destroys the graph and returns its memory. */
void secpe_graph_destroy(secpe_graph *g);

/* ---- continuous-batching server ---------------------------------------- */
/* A server keeps the state of admitted queries on the device and advances
 * them phase by phase through SecPE's circuit (Sec. 3.1 step 3 and Alg. 1:
 * aggregation + duplication, QuickMax rounds, final Sign).  Each
 * secpe_server_step admits what fits, then enqueues one phase of every query
 * in flight: queries at the same point of the circuit (same tenant, phase
 * and class-count power) form a group evaluated as one batch of at most
 * max_batch queries, groups in the order of their oldest member.  A query
 * submitted while others are mid-circuit therefore starts in the next step,
 * its launches interleaved on the stream with theirs.  Queries of different tenants (secpe_query.keys; null = the
 * server's keys) are batched only with queries of the same tenant.  Every
 * key set seen is counted as resident; a query is admitted when those keys +
 * in-flight states + one step's scratch + its state fit hbm_budget_bytes;
 * until then it waits (a submit whose new key set alone cannot fit returns
 * SECPE_EADMIT).  Results are bit-identical to secpe_encrypted_argmax with
 * the query's keys on the aggregated input.
 * The query's cts and z_out must stay valid until it completes. */
typedef struct secpe_server secpe_server;
typedef struct {
    int32_t waiting, active, done;
    uint64_t in_flight_bytes, keys_bytes, scratch_bytes;
} secpe_server_stats_t;
/* SECPE_EADMIT if the budget cannot hold even one query. */
int secpe_server_create(secpe_ctx *ctx, const secpe_keys *keys, uint64_t hbm_budget_bytes, int max_batch,
                        secpe_server **out);
void secpe_server_destroy(secpe_server *srv);
/* Validates the query (levels, scales, keys: SECPE_EKEY if a needed Galois
 * key is missing) and queues it; returns its ticket. */
int secpe_server_submit(secpe_server *srv, const secpe_query *q, int64_t *ticket);
/* Drops a query that has not completed (its state is released). */
int secpe_server_cancel(secpe_server *srv, int64_t ticket);
/* Admits what fits, then enqueues one phase of every query in flight on
 * `stream`; *launched = number of queries advanced (0 when idle). */
int secpe_server_step(secpe_server *srv, void *stream, int *launched);
/* *done = 1 when the query's result is ready on the device, 0 if not yet,
 * -1 if cancelled. */
int secpe_server_poll(secpe_server *srv, int64_t ticket, int *done);
/* Steps until the query completes; SECPE_ETIMEOUT after timeout_s seconds. */
int secpe_server_wait(secpe_server *srv, int64_t ticket, double timeout_s);
/* Releases the bookkeeping of a completed or cancelled query. */
int secpe_server_forget(secpe_server *srv, int64_t ticket);
int secpe_server_stats(const secpe_server *srv, secpe_server_stats_t *out);

/* Counters of the last circuit call on this context (rotations, Sign
 * calls, relinearisations, refreshes, key switches, kernel launches). */
typedef struct {
    int64_t rotations, signs, relins, refreshes, keyswitches, launches;
    int64_t bootstraps;  /* refreshes done by bootstrapping (secpe_argmax_batch_boot) */
} secpe_counters;
int secpe_get_counters(const secpe_ctx *ctx, secpe_counters *out);
int secpe_reset_counters(secpe_ctx *ctx);

/* ---- autotuning ---------------------------------------------------------- */
/* Launch configurations of the N = 2^16 kernels: for each tuned kernel (the
 * four transform passes and the base-conversion pass) the candidates are 3
 * and 4 CTAs per SM (at most 80 or 64 registers per thread).
 * secpe_autotune times the candidates alternately with CUDA events on a
 * zero-filled scratch batch of 64 x 32 limbs (1 GiB, larger than L2; the data
 * does not change the work), takes the median of 5 launches each, keeps 4
 * CTAs per SM only where it is more than 3% faster, and reports the choice in
 * *out (host, may be null); it needs 1 GiB of free device memory.  It synchronises `stream` (it cannot be captured).  For other ring
 * sizes there is nothing to tune and n_kernels = 0.  Untuned contexts use 3
 * CTAs per SM.  Every configuration computes identical results. */
typedef struct {
    int32_t n_kernels;
    char name[8][32];
    int32_t ctas_per_sm[8];  /* chosen */
    float ms[8][2];          /* per launch with 3 and with 4 CTAs per SM */
} secpe_tuning;
int secpe_autotune(secpe_ctx *ctx, secpe_tuning *out, void *stream);
/* Fixes kernel `kernel` (index as in secpe_tuning) to ctas_per_sm (3 or 4). */
int secpe_tuning_set(secpe_ctx *ctx, int kernel, int ctas_per_sm);

/* ---- instrumentation --------------------------------------------------- */
/* Device memory of the stream-ordered allocator on the current device (the
 * default memory pool, from which the library takes its temporaries and
 * which keeps freed blocks cached): *used = bytes in live allocations,
 * *reserved = bytes the pool holds from the driver.  With trim != 0 the
 * device is synchronised and the pool's unused blocks are returned to the
 * driver first.  Either output may be null.  SECPE_ECUDA without a device. */
int secpe_pool_usage(int trim, uint64_t *used, uint64_t *reserved);
/* Times, with CUDA events recorded on the launching stream around each
 * launch, every launch of the library kernels whose name contains
 * name_filter ("ntt", "ksk_ip", "modup", "moddown", ...), up to
 * max_launches launches, until secpe_kprof_end.  `bytes` accumulates each
 * recorded launch's share of its operation's algorithmic bytes (the minimal
 * DRAM traffic of the operation: its operands read once, its results
 * written once, its intermediates not at all; a standalone NTT/INTT is 16 N
 * bytes per limb, a key switch of B items at level l is B (l + 1) limbs in +
 * the key's 2 dnum(l) (l + 1 + n_p) limbs + B 2 (l + 1) limbs out, 8 N bytes
 * each).  `model_bytes` accumulates what the recorded launches themselves
 * read and write (each transform pass a read and a write of every residue,
 * intermediates included).  `mul32` accumulates their algorithmic 32-bit
 * multiplies: the 32 x 32-bit partial-product halves (mul.lo / mul.hi) of
 * the 64-bit modular products the kernels form (15 per Shoup product, 19
 * per Montgomery product, 8 per 128-bit multiply-accumulate, 11 per
 * Montgomery reduction; 60 per residue per 8-stage transform pass). */
typedef struct {
    int64_t launches;
    double total_ms;
    double bytes;
    double model_bytes;
    double mul32;
} secpe_kprof;
int secpe_kprof_begin(secpe_ctx *ctx, const char *name_filter, int max_launches);
/* Synchronises the device, sums the recorded durations, stops recording. */
int secpe_kprof_end(secpe_ctx *ctx, secpe_kprof *out);
/* With name_filter "*", every launch is recorded under its kernel's name
 * (and no operation-level range is).  After secpe_kprof_end, writes one
 * line per kernel, "name<TAB>launches<TAB>total ms", sorted by time, into
 * buf (host, len bytes, truncated and NUL-terminated; len may be 0 with buf
 * null) and the full text's size + 1 into *needed.  SECPE_EINVAL while the
 * profiler is still recording. */
int secpe_kprof_report(const secpe_ctx *ctx, char *buf, size_t len, size_t *needed);
/* Throughput probe of the integer multiply pipe (the roofline of the
 * transform and base-conversion kernels): one launch of
 * (SMs x ctas_per_sm) CTAs of 256 threads, each thread running 4
 * independent 128-bit multiply-accumulate chains (8 32-bit multiplies each,
 * the form the kernels use) for `iters` iterations on register data,
 * timed with CUDA events on `stream` after one untimed launch.  Writes the
 * achieved 32-bit multiplies per second to *mul32_per_s (host).  Scratch:
 * one 8-byte word per thread from the stream-ordered allocator.  iters in
 * 1 .. 2^20, ctas_per_sm in 1 .. 32. */
int secpe_mul32_probe(secpe_ctx *ctx, int ctas_per_sm, int iters, double *mul32_per_s, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SECPE_H */
