"""Plain CPU oracle of SecPE's encrypted ensemble Argmax on RNS-CKKS.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, the smoke check and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA library; the ring arithmetic is the plain C in ring.c, the rest is
numpy / Python integers in the order the paper (or the stated reading) gives.

Parity status per function:
  ring ops, NTT, basis conversion, rescale, key switching (plain and
  hoisted), encode/decode, Sign/Max/QuickMax/Argmax, the level plan, the
  Phoenix baseline, slot packing, the CLIP-style linear step and
  bootstrapping (boot.py): pinned (see tests/test_oracle_*.py and
  tests/test_level_plan.py; tests/test_oracle_pins_catch_mistakes.py plants
  mistakes that those pins catch).
  Residue-level intermediate values of the encrypted circuit: parity
  unpinned at that layer.  The paper prints none (its worked example is a
  missing figure), so residues are defined by this oracle; the decoded
  values and the returned index are pinned by mathematics (plaintext
  simulation, exact argmax).

Scheme summary (SecPE Sec. 2.2 and Sec. 3.2, readings where the paper is
silent are marked READING):
  * ciphertext (c0, c1) in NTT form over q_0..q_l, decrypting to c0 + c1*s;
  * READING: secret-key encryption, ternary secret, centred-binomial (eta=21)
    errors, randomness from counter-based SplitMix64 streams;
  * hybrid key switching with dnum digits and n_p special primes;
  * rescale by the last prime with rounding;
  * Sign = f^df o g^dg (Eq. comp) with the degree-9 f_4, g_4 of Cheon et al.
    (Asiacrypt 2020), each evaluated by the fixed depth-4 baby-step
    giant-step DAG in `poly9`;
  * Max(a, b) = (a+b)/2 + (a-b)/2 * Sign(a-b) (Eq. max);
  * Argmax = Alg. 1 (duplicate, QuickMax over rotations by 2^i, subtract the
    max, Sign, add 1).
"""
import math

import numpy as np

from . import _lib
from .params import Context
from .signpoly import sign_coeffs_float

U64 = np.uint64

# stream domains of the counter-based sampler (shared convention)
DOM_SECRET, DOM_KSK_A, DOM_KSK_E, DOM_ENC_A, DOM_ENC_E, DOM_REFRESH = 1, 2, 3, 4, 5, 6
DOM_PHOENIX = 7  # refresh seeds of the comparison Signs of the Phoenix baseline
STEP_CONJ = 0x40000000  # the rotation "step" naming the conjugation X -> X^(2N-1)


def round_half_away(v):
    """Round a double to the nearest integer, halves away from zero (exact)."""
    a = abs(v)
    f = math.floor(a)
    r = f + (1 if a - f >= 0.5 else 0)
    return int(r) if v >= 0 else -int(r)


class Ct:
    """Ciphertext: c[2][level+1][N] uint64 (NTT form), level, scale."""

    def __init__(self, c, level, scale):
        self.c = c
        self.level = level
        self.scale = scale

    def copy(self):
        return Ct(self.c.copy(), self.level, self.scale)


class Oracle:
    """RNS-CKKS scheme + SecPE circuit on the CPU."""

    def __init__(self, params):
        self.ctx = Context(params)
        self.p = params
        self.n = self.ctx.n
        self.log_n = self.ctx.log_n
        self.lib = _lib.lib()
        self.primes = self.ctx.all_primes
        self.nq = len(self.ctx.q)
        self.counters = {}
        self.ridx = 0
        self.qseed = 0
        self.boot_plan = None   # a boot.BootPlan: refreshes become bootstraps (non-interactive)
        self.plan = None        # level plan of the Argmax being evaluated (level_plan)
        self.reset_counters()

    def reset_counters(self):
        self.counters = dict(rotations=0, signs=0, relins=0, refreshes=0,
                             keyswitches=0, bootstraps=0)

    # ------------------------------------------------------------ ring layer
    def ntt(self, a, pi):
        """In-place forward NTT of one limb (prime index pi)."""
        self.lib.or_ntt_fwd(_lib.ptr(a), self.log_n, self.primes[pi], self.ctx.psi[pi])

    def intt(self, a, pi):
        self.lib.or_ntt_inv(_lib.ptr(a), self.log_n, self.primes[pi], self.ctx.psi[pi])

    def _binop(self, fn, a, b, pi):
        out = np.empty(self.n, dtype=U64)
        fn(_lib.ptr(a), _lib.ptr(b), _lib.ptr(out), self.n, self.primes[pi])
        return out

    def vmul(self, a, b, pi):
        return self._binop(self.lib.or_vmul, a, b, pi)

    def vadd(self, a, b, pi):
        return self._binop(self.lib.or_vadd, a, b, pi)

    def vsub(self, a, b, pi):
        return self._binop(self.lib.or_vsub, a, b, pi)

    def vscale(self, a, c, pi):
        out = np.empty(self.n, dtype=U64)
        self.lib.or_vscale(_lib.ptr(a), int(c) % self.primes[pi], _lib.ptr(out),
                           self.n, self.primes[pi])
        return out

    def vaddc(self, a, c, pi):
        out = np.empty(self.n, dtype=U64)
        self.lib.or_vaddc(_lib.ptr(a), int(c) % self.primes[pi], _lib.ptr(out),
                          self.n, self.primes[pi])
        return out

    def vreduce(self, a, pi):
        out = np.empty(self.n, dtype=U64)
        self.lib.or_vreduce(_lib.ptr(a), _lib.ptr(out), self.n, self.primes[pi])
        return out

    def from_signed(self, coeffs, pi):
        """int64 coefficients -> residues mod prime pi."""
        c = np.ascontiguousarray(coeffs, dtype=np.int64)
        out = np.empty(self.n, dtype=U64)
        self.lib.or_vfrom_signed(_lib.ptr(c), _lib.ptr(out), self.n, self.primes[pi])
        return out

    def fast_bconv(self, x, src_idx, dst_idx):
        """FastBConv of coefficient-form limbs x[len(src)][N] to dst primes."""
        qin = _lib.u64arr([self.primes[i] for i in src_idx])
        qout = _lib.u64arr([self.primes[i] for i in dst_idx])
        xin = np.ascontiguousarray(x, dtype=U64)
        out = np.empty((len(dst_idx), self.n), dtype=U64)
        self.lib.or_fast_bconv(_lib.ptr(xin), _lib.ptr(qin), len(src_idx),
                               _lib.ptr(qout), len(dst_idx), _lib.ptr(out), self.n)
        return out

    def automorph_ntt(self, a, pi, g):
        """X -> X^g on an NTT-form limb, done in the coefficient domain."""
        x = a.copy()
        self.intt(x, pi)
        out = np.empty(self.n, dtype=U64)
        self.lib.or_automorph_coeff(_lib.ptr(x), _lib.ptr(out), self.log_n,
                                    self.primes[pi], g)
        self.ntt(out, pi)
        return out

    # --------------------------------------------------------------- sampling
    def stream(self, seed, domain, index):
        return int(self.lib.or_sm_stream(seed & (2**64 - 1), domain, index))

    def sample_ternary(self, key):
        out = np.empty(self.n, dtype=np.int64)
        self.lib.or_sample_ternary(key, _lib.ptr(out), self.n)
        return out

    def sample_sparse(self, key, h):
        """Sparse ternary vector with exactly h nonzero coefficients."""
        out = np.empty(self.n, dtype=np.int64)
        self.lib.or_sample_sparse(key, _lib.ptr(out), self.n, h)
        return out

    def sample_cbd(self, key):
        out = np.empty(self.n, dtype=np.int64)
        self.lib.or_sample_cbd21(key, _lib.ptr(out), self.n)
        return out

    def sample_uniform(self, key, pi):
        """Uniform NTT-form limb for prime index pi (stream offset pi*N)."""
        out = np.empty(self.n, dtype=U64)
        self.lib.or_sample_uniform(key, pi * self.n, self.primes[pi], _lib.ptr(out), self.n)
        return out

    def ntt_of_signed(self, coeffs, idx):
        """NTT over the prime indices idx of an int64 coefficient vector."""
        out = np.empty((len(idx), self.n), dtype=U64)
        for r, pi in enumerate(idx):
            out[r] = self.from_signed(coeffs, pi)
            self.ntt(out[r], pi)
        return out

    # ------------------------------------------------------------- encoding
    def _pow5(self, count):
        two_n = 2 * self.n
        out = np.empty(count, dtype=np.int64)
        e = 1
        for j in range(count):
            out[j] = e
            e = e * 5 % two_n
        return out

    def encode_coeffs(self, v, scale):
        """Canonical-embedding encoding of a real vector into slots 0..len(v)-1
        (zeros beyond): m_k = round(scale * (2/N) * sum_j v_j cos(pi 5^j k / N)),
        i.e. the inverse of m -> (m(zeta^(5^j)))_j, zeta = exp(i pi / N),
        taking the real coefficients (SecPE Sec. 2.2 SIMD packing)."""
        v = np.asarray(v, dtype=np.float64)
        n_s = len(v)
        assert n_s <= self.n // 2
        two_n = 2 * self.n
        p5 = self._pow5(n_s)
        ks = np.arange(self.n, dtype=np.int64)
        acc = np.zeros(self.n, dtype=np.float64)
        for j in range(n_s):
            e = (p5[j] * ks) % two_n
            acc += v[j] * np.cos(np.pi * e.astype(np.float64) / self.n)
        vals = acc * (2.0 / self.n) * scale
        return np.array([round_half_away(float(x)) for x in vals], dtype=object)

    def encode_complex(self, z, scale):
        """Canonical-embedding encoding of a complex slot vector z (slots
        0..len(z)-1, zeros beyond): the real coefficients
        m_k = round(scale * (2/N) * Re(sum_j z_j zeta^(-5^j k)))
            = round(scale * (2/N) * sum_j (Re z_j cos(pi e/N) + Im z_j sin(pi e/N))),
        e = 5^j k mod 2N (the conjugate slots hold conj(z_j))."""
        z = np.asarray(z, dtype=np.complex128)
        n_s = len(z)
        assert n_s <= self.n // 2
        two_n = 2 * self.n
        p5 = self._pow5(n_s)
        ks = np.arange(self.n, dtype=np.int64)
        acc = np.zeros(self.n, dtype=np.float64)
        for j in range(n_s):
            th = np.pi * ((p5[j] * ks) % two_n).astype(np.float64) / self.n
            acc += z[j].real * np.cos(th) + z[j].imag * np.sin(th)
        vals = acc * (2.0 / self.n) * scale
        return np.array([round_half_away(float(x)) for x in vals], dtype=object)

    def decode_complex(self, m, scale, n_slots):
        """Slots 0..n_slots-1 of m(zeta^(5^j)) / scale, complex."""
        mf = np.array([float(x) for x in m], dtype=np.float64)
        two_n = 2 * self.n
        p5 = self._pow5(n_slots)
        ks = np.arange(self.n, dtype=np.int64)
        out = np.empty(n_slots, dtype=np.complex128)
        for j in range(n_slots):
            th = np.pi * ((p5[j] * ks) % two_n).astype(np.float64) / self.n
            out[j] = complex(np.dot(mf, np.cos(th)), np.dot(mf, np.sin(th)))
        return out / scale

    def decode_coeffs(self, m, scale, n_slots):
        """Slots 0..n_slots-1 of the real part of m(zeta^(5^j)) / scale."""
        mf = np.array([float(x) for x in m], dtype=np.float64)
        two_n = 2 * self.n
        p5 = self._pow5(n_slots)
        ks = np.arange(self.n, dtype=np.int64)
        out = np.empty(n_slots, dtype=np.float64)
        for j in range(n_slots):
            e = (p5[j] * ks) % two_n
            out[j] = np.dot(mf, np.cos(np.pi * e.astype(np.float64) / self.n))
        return out / scale

    # ------------------------------------------------------------------ keys
    def keygen(self, seed, rot_steps=()):
        """Secret key, relinearisation key and Galois keys for RotL(r), r in
        rot_steps (negative r means RotR(-r))."""
        all_idx = list(range(len(self.primes)))
        key = self.stream(seed, DOM_SECRET, 0)
        s = self.sample_sparse(key, self.p.secret_hw) if self.p.secret_hw else self.sample_ternary(key)
        self.s_coeffs = s
        self.s_ntt = self.ntt_of_signed(s, all_idx)
        self.seed = seed
        s2 = np.stack([self.vmul(self.s_ntt[pi], self.s_ntt[pi], pi) for pi in all_idx])
        self.rlk = self.make_ksk(s2, 0)
        self.gks = {}
        for r in rot_steps:
            g = self.galois(r)
            if g in self.gks:
                continue
            sg = np.stack([self.automorph_ntt(self.s_ntt[pi], pi, g) for pi in all_idx])
            self.gks[g] = self.make_ksk(sg, g)

    def make_ksk(self, s_new, kid):
        """Hybrid key-switching key from s_new to s: per digit j,
        b_j = -a_j s + e_j + [P]_{q_i} s_new on primes of digit j (0 on the
        other primes, where the CRT gadget vanishes, and on the special primes,
        where P vanishes), a_j uniform.  Returns array [dnum][2][nprimes][N]."""
        nprimes = len(self.primes)
        full_digits = self.ctx.digits(self.ctx.L)
        out = np.empty((len(full_digits), 2, nprimes, self.n), dtype=U64)
        for j, dig in enumerate(full_digits):
            ka = self.stream(self.seed, DOM_KSK_A, kid * 64 + j)
            ke = self.stream(self.seed, DOM_KSK_E, kid * 64 + j)
            e = self.sample_cbd(ke)
            e_ntt = self.ntt_of_signed(e, list(range(nprimes)))
            for pi in range(nprimes):
                a = self.sample_uniform(ka, pi)
                b = self.vsub(e_ntt[pi], self.vmul(a, self.s_ntt[pi], pi), pi)
                if pi in dig:
                    pm = self.ctx.P % self.primes[pi]
                    b = self.vadd(b, self.vscale(s_new[pi], pm, pi), pi)
                out[j, 0, pi] = b
                out[j, 1, pi] = a
        return out

    def galois(self, r):
        """Galois element of RotL(r) (RotR(r') = RotL(N/2 - r')); 2N - 1 for
        the conjugation (r = STEP_CONJ)."""
        two_n = 2 * self.n
        if r == STEP_CONJ:
            return two_n - 1
        if r < 0:
            r = self.n // 2 + r
        return pow(5, r % (self.n // 2), two_n)

    # ---------------------------------------------------- encrypt / decrypt
    def encrypt_coeffs(self, m, level, scale, seed):
        """Secret-key encryption of integer coefficients m (list/array of
        Python ints, |m| < q_0/2 not required): c1 = a, c0 = -a s + m + e."""
        idx = list(range(level + 1))
        ka = self.stream(seed, DOM_ENC_A, 0)
        e = self.sample_cbd(self.stream(seed, DOM_ENC_E, 0))
        c = np.empty((2, level + 1, self.n), dtype=U64)
        mm = [int(x) for x in m]
        for pi in idx:
            q = self.primes[pi]
            mres = np.array([(x + int(ei)) % q for x, ei in zip(mm, e)], dtype=U64)
            self.ntt(mres, pi)
            a = self.sample_uniform(ka, pi)
            c[0, pi] = self.vsub(mres, self.vmul(a, self.s_ntt[pi], pi), pi)
            c[1, pi] = a
        return Ct(c, level, scale)

    def encrypt(self, v, seed, level=None, scale=None):
        level = self.ctx.L if level is None else level
        scale = self.p.scale if scale is None else scale
        return self.encrypt_coeffs(self.encode_coeffs(v, scale), level, scale, seed)

    def encrypt_logits(self, v, n_classes, d_min, seed):
        """Client-side encryption of one prompt's logit vector (SecPE Sec. 3.1
        step 1, Eq. argmax layout): slots 0..C-1 hold the logits; READING for
        C not a power of two: slots C..C'-1 hold d_min, so that after the
        normalisation they sit at the bottom of the range; zeros beyond C'."""
        cp = 1 << (n_classes - 1).bit_length()
        v = np.asarray(v, dtype=np.float64)
        assert len(v) == n_classes
        full = np.concatenate([v, np.full(cp - n_classes, float(d_min))])
        return self.encrypt(full, seed)

    # ------------------------------------------------------- slot packing
    def packed_capacity(self, n_classes):
        """Inputs per ciphertext under slot packing (SecPE Sec. 3.2, after
        Alg. 1): each input needs a block of 2C' slots, C' values and the C'
        slots its duplication fills, so N/2 slots hold N/(4C') inputs."""
        cp = 1 << (n_classes - 1).bit_length()
        return (self.n // 2) // (2 * cp)

    def pack_slots(self, V, d_min):
        """Slot vector of the inputs V[P][C] (READING of the slot-batching
        paragraph: input b in the block of 2C' slots starting at 2C'b, its C
        logits, then d_min up to C' as for one query, then C' zeros)."""
        V = np.asarray(V, dtype=np.float64)
        P, C = V.shape
        cp = 1 << (C - 1).bit_length()
        assert P <= self.packed_capacity(C)
        out = np.zeros(P * 2 * cp, dtype=np.float64)
        for b in range(P):
            out[b * 2 * cp: b * 2 * cp + C] = V[b]
            out[b * 2 * cp + C: b * 2 * cp + cp] = d_min
        return out

    def encrypt_logits_packed(self, V, d_min, seed):
        """One prompt's logit vectors of P inputs in one ciphertext."""
        return self.encrypt(self.pack_slots(V, d_min), seed)

    def decrypt_packed(self, ct, P, n_classes):
        """The first C slots of each of the P blocks, [P][C]."""
        cp = 1 << (n_classes - 1).bit_length()
        s = self.decrypt(ct, P * 2 * cp)
        return np.stack([s[b * 2 * cp: b * 2 * cp + n_classes] for b in range(P)])

    def decrypt_coeffs(self, ct):
        """Centred integer coefficients of c0 + c1*s by exact CRT."""
        lv = ct.level
        res = []
        for pi in range(lv + 1):
            x = self.vadd(ct.c[0, pi], self.vmul(ct.c[1, pi], self.s_ntt[pi], pi), pi)
            self.intt(x, pi)
            res.append(x)
        return self.crt_centred(res, lv)

    def crt_centred(self, res, lv):
        qs = self.ctx.q[: lv + 1]
        Q = 1
        for q in qs:
            Q *= q
        acc = np.zeros(self.n, dtype=object)
        for pi, q in enumerate(qs):
            Mi = Q // q
            coef = Mi * pow(Mi % q, -1, q)
            acc = acc + res[pi].astype(object) * coef
        acc = acc % Q
        half = Q // 2
        return np.where(acc > half, acc - Q, acc)

    def decrypt(self, ct, n_slots):
        return self.decode_coeffs(self.decrypt_coeffs(ct), ct.scale, n_slots)

    # ------------------------------------------------------ key switching
    def keyswitch_acc(self, d, level, ksk):
        """ModUp and key inner product of hybrid key switching (before the
        division by P): d (NTT form, limbs 0..level) -> (acc0, acc1) over
        Q_l u P.  ModUp per digit: INTT, FastBConv to the other primes, NTT."""
        self.counters["keyswitches"] += 1
        q_idx = list(range(level + 1))
        sp_idx = self.ctx.special_idx()
        tgt = q_idx + sp_idx
        coef = d.copy()
        for pi in q_idx:
            self.intt(coef[pi], pi)
        acc0 = {t: np.zeros(self.n, dtype=U64) for t in tgt}
        acc1 = {t: np.zeros(self.n, dtype=U64) for t in tgt}
        for j, dig in enumerate(self.ctx.digits(level)):
            others = [t for t in tgt if t not in dig]
            conv = self.fast_bconv(np.stack([coef[pi] for pi in dig]), dig, others)
            ext = {}
            for r, t in enumerate(others):
                x = conv[r].copy()
                self.ntt(x, t)
                ext[t] = x
            for pi in dig:
                ext[pi] = d[pi]
            for t in tgt:
                acc0[t] = self.vadd(acc0[t], self.vmul(ext[t], ksk[j, 0, t], t), t)
                acc1[t] = self.vadd(acc1[t], self.vmul(ext[t], ksk[j, 1, t], t), t)
        return acc0, acc1

    def modup_ext(self, d, level):
        """ModUp of d (NTT form, limbs 0..level) as keyswitch_acc computes
        it: per digit j, ext[j][t] (NTT form) for every prime t of Q_l u P
        outside the digit, by FastBConv of the digit's INTT (no correction)."""
        q_idx = list(range(level + 1))
        tgt = q_idx + self.ctx.special_idx()
        coef = d.copy()
        for pi in q_idx:
            self.intt(coef[pi], pi)
        exts = []
        for dig in self.ctx.digits(level):
            others = [t for t in tgt if t not in dig]
            conv = self.fast_bconv(np.stack([coef[pi] for pi in dig]), dig, others)
            ext = {}
            for r, t in enumerate(others):
                x = conv[r].copy()
                self.ntt(x, t)
                ext[t] = x
            exts.append(ext)
        return exts

    def rotate_hoisted(self, ct, rs):
        """READING (hoisting; the paper does not describe bootstrapping, whose
        linear transforms rotate one ciphertext by many steps): RotL(ct, r)
        for every r in rs from one ModUp of c1.  For each r the automorphism
        X -> X^g goes onto c0, onto c1 (each digit's own limbs) and onto every
        extended limb, then come the inner product with the Galois key and
        ModDown.  The automorphism of an extended limb differs from the ModUp
        of the automorphism only by the multiple of the digit modulus that
        FastBConv leaves, permuted (same size), so each result is a key
        switching of sigma_g(c1) with the same noise bound as rotate's."""
        lv = ct.level
        exts = self.modup_ext(ct.c[1], lv)
        tgt = list(range(lv + 1)) + self.ctx.special_idx()
        outs = []
        for r in rs:
            g = self.galois(r)
            if g not in self.gks:
                raise KeyError("missing Galois key for rotation %d" % r)
            self.counters["rotations"] += 1
            self.counters["keyswitches"] += 1
            ksk = self.gks[g]
            t0 = np.stack([self.automorph_ntt(ct.c[0, pi], pi, g) for pi in range(lv + 1)])
            t1 = np.stack([self.automorph_ntt(ct.c[1, pi], pi, g) for pi in range(lv + 1)])
            acc0 = {t: np.zeros(self.n, dtype=U64) for t in tgt}
            acc1 = {t: np.zeros(self.n, dtype=U64) for t in tgt}
            for j, dig in enumerate(self.ctx.digits(lv)):
                for t in tgt:
                    x = t1[t] if t in dig else self.automorph_ntt(exts[j][t], t, g)
                    acc0[t] = self.vadd(acc0[t], self.vmul(x, ksk[j, 0, t], t), t)
                    acc1[t] = self.vadd(acc1[t], self.vmul(x, ksk[j, 1, t], t), t)
            k0, k1 = self.moddown(acc0, lv), self.moddown(acc1, lv)
            c = np.empty((2, lv + 1, self.n), dtype=U64)
            for pi in range(lv + 1):
                c[0, pi] = self.vadd(t0[pi], k0[pi], pi)
                c[1, pi] = k1[pi]
            outs.append(Ct(c, lv, ct.scale))
        return outs

    def keyswitch(self, d, level, ksk):
        """Hybrid key switching of d with key ksk: ModUp, inner product, then
        ModDown (rounded division by P)."""
        acc0, acc1 = self.keyswitch_acc(d, level, ksk)
        return self.moddown(acc0, level), self.moddown(acc1, level)

    def moddown_rescale(self, acc, dk, level):
        """Relinearisation's ModDown fused with the rescale (READING: one
        rounded division instead of two): x = P*dk + acc over Q_l u P,
        out = round(x / (P q_l)) over q_0..q_{l-1}, computed as
        (x - (FastBConv([x + h]_M) - h)) * M^-1 with M = P q_l, h = floor(M/2),
        the FastBConv from the primes of M (the special primes and q_l)."""
        sp_idx = self.ctx.special_idx()
        ql = self.primes[level]
        M = self.ctx.P * ql
        h = M // 2
        src = sp_idx + [level]
        xs = np.stack([acc[t].copy() for t in sp_idx] +
                      [self.vadd(self.vscale(dk[level], self.ctx.P % ql, level), acc[level], level)])
        for r, t in enumerate(src):
            self.intt(xs[r], t)
            xs[r] = self.vaddc(xs[r], h % self.primes[t], t)
        conv = self.fast_bconv(xs, src, list(range(level)))
        out = np.empty((level, self.n), dtype=U64)
        for pi in range(level):
            q = self.primes[pi]
            c = self.vaddc(conv[pi], -h % q, pi)
            self.ntt(c, pi)
            x = self.vadd(self.vscale(dk[pi], self.ctx.P % q, pi), acc[pi], pi)
            out[pi] = self.vscale(self.vsub(x, c, pi), pow(M % q, -1, q), pi)
        return out

    def moddown(self, acc, level):
        """Rounded division by P of x given over Q_l u P (READING: rounding,
        like the rescale): y = [x + h]_P with h = floor(P/2) on the special
        limbs (coefficient form), conv_i = FastBConv(y -> q_i) - h,
        out_i = (x_i - conv_i) * P^-1 mod q_i."""
        sp_idx = self.ctx.special_idx()
        hP = self.ctx.P // 2
        pc = np.stack([acc[t].copy() for t in sp_idx])
        for r, t in enumerate(sp_idx):
            self.intt(pc[r], t)
            pc[r] = self.vaddc(pc[r], hP % self.primes[t], t)
        q_idx = list(range(level + 1))
        conv = self.fast_bconv(pc, sp_idx, q_idx)
        out = np.empty((level + 1, self.n), dtype=U64)
        for pi in q_idx:
            q = self.primes[pi]
            x = self.vaddc(conv[pi], -hP % q, pi)
            self.ntt(x, pi)
            pinv = pow(self.ctx.P % q, -1, q)
            out[pi] = self.vscale(self.vsub(acc[pi], x, pi), pinv, pi)
        return out

    # --------------------------------------------------------- evaluator
    def drop(self, ct, level):
        """Modulus drop: keep limbs 0..level (scale unchanged)."""
        assert level <= ct.level
        return Ct(np.ascontiguousarray(ct.c[:, : level + 1]), level, ct.scale)

    def _check_scales(self, a, b):
        if abs(a.scale - b.scale) > a.scale * 2.0 ** -40:
            raise ValueError("scale mismatch %r vs %r" % (a.scale, b.scale))

    def add(self, a, b):
        lv = min(a.level, b.level)
        a, b = self.drop(a, lv), self.drop(b, lv)
        self._check_scales(a, b)
        c = np.empty_like(a.c)
        for k in range(2):
            for pi in range(lv + 1):
                c[k, pi] = self.vadd(a.c[k, pi], b.c[k, pi], pi)
        return Ct(c, lv, a.scale)

    def sub(self, a, b):
        lv = min(a.level, b.level)
        a, b = self.drop(a, lv), self.drop(b, lv)
        self._check_scales(a, b)
        c = np.empty_like(a.c)
        for k in range(2):
            for pi in range(lv + 1):
                c[k, pi] = self.vsub(a.c[k, pi], b.c[k, pi], pi)
        return Ct(c, lv, a.scale)

    def rescale(self, ct):
        """Divide by q_l with rounding: c' = (c + h - [c + h]_{q_l}) / q_l,
        h = floor(q_l / 2), [.] the remainder in [0, q_l)."""
        lv = ct.level
        ql = self.primes[lv]
        h = ql // 2
        out = np.empty((2, lv, self.n), dtype=U64)
        for k in range(2):
            y = ct.c[k, lv].copy()
            self.intt(y, lv)
            y = self.vaddc(y, h, lv)
            for pi in range(lv):
                # z = [c + h]_{q_l} - h, per coefficient, reduced mod q_i
                z = self.vaddc(self.vreduce(y, pi), -h % self.primes[pi], pi)
                self.ntt(z, pi)
                t = self.vsub(ct.c[k, pi], z, pi)
                out[k, pi] = self.vscale(t, pow(ql % self.primes[pi], -1, self.primes[pi]), pi)
        return Ct(out, lv - 1, ct.scale / float(ql))

    def tensor(self, a, b):
        """(a0 b0, a0 b1 + a1 b0, a1 b1) at the lower level, scale s_a s_b:
        a 3-component ciphertext (decrypts with (1, s, s^2))."""
        lv = min(a.level, b.level)
        a, b = self.drop(a, lv), self.drop(b, lv)
        d = np.empty((3, lv + 1, self.n), dtype=U64)
        for pi in range(lv + 1):
            d[0, pi] = self.vmul(a.c[0, pi], b.c[0, pi], pi)
            d[1, pi] = self.vadd(self.vmul(a.c[0, pi], b.c[1, pi], pi),
                                 self.vmul(a.c[1, pi], b.c[0, pi], pi), pi)
            d[2, pi] = self.vmul(a.c[1, pi], b.c[1, pi], pi)
        return Ct(d, lv, a.scale * b.scale)

    def relin_rescale(self, d):
        """Relinearise a 3-component ciphertext and divide by its last prime:
        key switching of d2 (ModUp, inner product) and one rounded division of
        (P d_k + acc_k) by P q_l for k = 0, 1."""
        lv = d.level
        if lv < 1 + self.p.reserve:
            raise ValueError("not enough levels")
        self.counters["relins"] += 1
        acc0, acc1 = self.keyswitch_acc(d.c[2], lv, self.rlk)
        c = np.stack([self.moddown_rescale(acc0, d.c[0], lv), self.moddown_rescale(acc1, d.c[1], lv)])
        return Ct(c, lv - 1, d.scale / float(self.primes[lv]))

    def add3(self, a, b):
        """Sum of two 3-component ciphertexts at the same level and scale."""
        assert a.level == b.level
        self._check_scales(a, b)
        c = np.empty_like(a.c)
        for k in range(3):
            for pi in range(a.level + 1):
                c[k, pi] = self.vadd(a.c[k, pi], b.c[k, pi], pi)
        return Ct(c, a.level, a.scale)

    def mul(self, a, b):
        """Slot-wise product (SecPE Sec. 2.2): tensor, relinearise, rescale."""
        lv = min(a.level, b.level)
        if lv < 1 + self.p.reserve:
            raise ValueError("not enough levels")
        return self.relin_rescale(self.tensor(a, b))

    def mul_const(self, x, c, target, out_level):
        """x * c landing at out_level with scale exactly `target`: drop x to
        out_level+1, multiply by the integer k = round(c * target / s_x * q),
        q = q_{out_level+1}, rescale."""
        return self.lincomb([(x, c)], target, out_level)

    def lincomb(self, terms, target, out_level):
        """sum_i c_i x_i landing at out_level with scale exactly `target`:
        each x_i is dropped to out_level+1 and multiplied by the integer
        k_i = round(c_i * target / s_i * q), q = q_{out_level+1}, so that
        every product has scale ~ target * q; the products are added and the
        sum is rescaled once (READING: a linear combination of constant
        multiples costs one rescale, not one per term)."""
        if out_level < self.p.reserve:
            raise ValueError("not enough levels")
        qf = float(self.primes[out_level + 1])
        cc = np.zeros((2, out_level + 2, self.n), dtype=U64)
        for x, c in terms:
            if x.level < out_level + 1:
                raise ValueError("not enough levels for mul_const")
            xd = self.drop(x, out_level + 1)
            k = round_half_away(c * (target / xd.scale * qf))
            for kk in range(2):
                for pi in range(out_level + 2):
                    cc[kk, pi] = self.vadd(cc[kk, pi], self.vscale(xd.c[kk, pi], k % self.primes[pi], pi), pi)
        r = self.rescale(Ct(cc, out_level + 1, target * qf))
        r.scale = target
        return r

    def add_const(self, x, c):
        """x + c: the constant polynomial round(c * s_x) added to c0."""
        k = round_half_away(c * x.scale)
        out = x.copy()
        for pi in range(x.level + 1):
            out.c[0, pi] = self.vaddc(x.c[0, pi], k % self.primes[pi], pi)
        return out

    def rotate(self, ct, r):
        """RotL(ct, r) for r > 0, RotR(ct, -r) for r < 0 (SecPE Sec. 2.2):
        automorphism X -> X^g, g = 5^r mod 2N, then key switching of c1."""
        g = self.galois(r)
        if g not in self.gks:
            raise KeyError("missing Galois key for rotation %d" % r)
        self.counters["rotations"] += 1
        lv = ct.level
        t0 = np.stack([self.automorph_ntt(ct.c[0, pi], pi, g) for pi in range(lv + 1)])
        t1 = np.stack([self.automorph_ntt(ct.c[1, pi], pi, g) for pi in range(lv + 1)])
        k0, k1 = self.keyswitch(t1, lv, self.gks[g])
        c = np.empty((2, lv + 1, self.n), dtype=U64)
        for pi in range(lv + 1):
            c[0, pi] = self.vadd(t0[pi], k0[pi], pi)
            c[1, pi] = k1[pi]
        return Ct(c, lv, ct.scale)

    def refresh(self, ct, qseed):
        """Test-only, insecure stand-in for bootstrapping (READING of SecPE
        Sec. 2.2/4.1, which rely on bootstrapping without describing it):
        decrypt, lift exactly by CRT to centred integers, re-encrypt at the top
        level with the same scale, randomness from stream (qseed, refresh#)."""
        if self.boot_plan is not None:
            # non-interactive: a bootstrap (boot.py) instead of the stand-in
            self.ridx += 1
            self.counters["refreshes"] += 1
            self.counters["bootstraps"] += 1
            return self.boot_plan.bootstrap(ct)
        m = self.decrypt_coeffs(ct)
        idx = self.ridx
        self.ridx += 1
        self.counters["refreshes"] += 1
        seed = self.stream(qseed, DOM_REFRESH, idx)
        return self.encrypt_coeffs(m, self.ctx.L, ct.scale, seed)

    # ------------------------------------------------------ SecPE circuit
    def ensure(self, ct, k):
        """Refresh ct if fewer than k + reserve levels remain.  Inside an
        Argmax with a level plan, the refreshed ciphertext is then dropped
        to the plan's level for the range the refresh starts."""
        if ct.level < k + self.p.reserve:
            ct = self.refresh(ct, self.qseed)
            if self.plan is not None and self.ridx < len(self.plan) and ct.level > self.plan[self.ridx]:
                ct = self.drop(ct, self.plan[self.ridx])
        return ct

    def refresh_level(self):
        """Level of a refreshed ciphertext: the top level for the stand-in,
        L - 16 for a bootstrap."""
        return self.ctx.L if self.boot_plan is None else self.boot_plan.out_level

    def level_plan(self, r, entry):
        """READING (level-aware QuickMax; the paper does not discuss levels).
        Alg. 1 with r QuickMax rounds on y at level `entry`, refreshing before
        a step that lacks its levels (as ensure does), falls into ranges: the
        first starts at y, each refresh starts the next.  Range by range, in
        order, the plan lowers the range's first ciphertext by as many levels
        as keep every refresh at the same step and leave the refreshed step
        its levels.  A lower start never raises a later level, so the levels
        that keep the refreshes in place form an interval, found by lowering
        one level at a time.  (A range's ciphertexts can reach later ranges:
        Max multiplies d, computed before a refresh inside Sign(d), by the
        refreshed Sign, so the whole circuit is walked for every trial.)
        Returns the level of each range's first ciphertext: [y after the
        duplication, after refresh 1, 2, ...]."""
        res, top = self.p.reserve, self.refresh_level()
        n_poly = self.p.sign_dg + self.p.sign_df

        def walk(plan):
            """Indices of the level tests that refresh under `plan` (None if a
            refreshed step lacks its levels)."""
            points, count, ok = [], [0], [True]

            def test(lv, k):
                count[0] += 1
                if lv >= k + res:
                    return lv
                points.append(count[0])
                j = len(points)
                out = min(top, plan[j]) if j < len(plan) else top
                ok[0] = ok[0] and out >= k + res
                return out

            lv = min(entry, plan[0])
            for _ in range(r):                  # QuickMax rounds: y <- Max(RotL(y, 2^i), y)
                lv = test(lv, 1)
                ld = lv                         # d = a - y stays at this level
                for i in range(n_poly):         # Sign(d), one more level for the last
                    lv = test(lv, 5 if i == n_poly - 1 else 4) - 4
                lv = min(ld, lv) - 1            # t = d * Sign(d)/2; Max = t + u at t's level
            for i in range(n_poly):             # final Sign, evaluated lowest
                lv = min(test(lv, 4), 4 * (n_poly - i) + res) - 4
            return points if ok[0] else None

        points = walk([entry])
        if points is None:
            raise ValueError("not enough levels after a refresh")
        plan = [entry] + [top] * len(points)
        for j in range(len(plan)):
            while plan[j] > 0 and walk(plan[:j] + [plan[j] - 1] + plan[j + 1:]) == points:
                plan[j] -= 1
        return plan

    def poly9(self, x, c, s_out):
        """Odd degree-9 p(x) = c1 x + c3 x^3 + c5 x^5 + c7 x^7 + c9 x^9 (SecPE
        Eq. comp: degree-9 f and g, evaluated baby-step giant-step).  READING
        of the schedule: baby steps in y = x^2, giant step x^4,
            p = x (c1 + c3 y) + x^5 (c5 + c7 y + c9 y^2),
        by the depth-4 DAG
          x2 = x*x, x4 = x2*x2, x5 = x4*x,
          P1 = c7 x2 + c9 x4 + c5, P0 = c3 x2 + c1   (one rescale each),
          p = relin_rescale(x5 (x) P1 + x (x) P0),
        the two 3-component products being added before their single
        relinearisation: 4 key switches per polynomial.  P1 lands at the
        scale that gives p the scale s_out, P0 at the scale that makes both
        products' scales equal."""
        c1, c3, c5, c7, c9 = c
        lv = x.level
        q3 = float(self.primes[lv - 3])
        x2 = self.mul(x, x)
        x4 = self.mul(x2, x2)
        x5 = self.mul(x4, x)
        s1 = s_out * q3 / x5.scale
        P1 = self.add_const(self.lincomb([(x2, c7), (x4, c9)], s1, lv - 3), c5)
        s0 = x5.scale * s1 / x.scale
        P0 = self.add_const(self.lincomb([(x2, c3)], s0, lv - 3), c1)
        return self.relin_rescale(self.add3(self.tensor(x5, P1), self.tensor(x, P0)))

    def sign(self, x, out_levels, last_factor=1.0, lowest=False):
        """Sign(x) = f^df(g^dg(x)) (SecPE Eq. comp); before each polynomial,
        refresh if fewer than 4 (+ out_levels for the last) levels remain.
        The last polynomial's coefficients are multiplied by last_factor
        (last_factor * Sign(x) at no extra level).  READING (level-aware
        evaluation; the paper does not discuss levels): with `lowest`, used
        for the final Sign of Alg. 1, which nothing follows, each
        polynomial's input is dropped to the levels the rest of the Sign
        needs, 4 (polynomials left) + out_levels + reserve; refreshes are
        the same as without it."""
        self.counters["signs"] += 1
        g, f = sign_coeffs_float()
        polys = [g] * self.p.sign_dg + [f] * self.p.sign_df
        for i, c in enumerate(polys):
            last = i == len(polys) - 1
            need = 4 + (out_levels if last else 0)
            x = self.ensure(x, need)
            keep = 4 * (len(polys) - i) + out_levels + self.p.reserve
            if lowest and x.level > keep:
                x = self.drop(x, keep)
            x = self.poly9(x, [last_factor * ci for ci in c] if last else c, self.p.scale)
        return x

    def max(self, a, y):
        """Max(a, y) = (a+y)/2 + (a-y)/2 * Sign(a-y) (SecPE Eq. max),
        computed as (a+y)*1/2 + d * (Sign(d)/2) with d = a - y: the 1/2 of the
        second term is folded into the coefficients of Sign's last
        polynomial, so t = d * (Sign(d)/2) keeps d's scale (READING: no level
        is spent on it, and the scale does not grow from round to round);
        u = (a+y) * 1/2 is brought to t's level and scale, max = t + u."""
        d = self.sub(a, y)
        s = self.sign(d, 1, last_factor=0.5)
        t = self.mul(d, s)
        u = self.mul_const(self.add(a, y), 0.5, t.scale, t.level)
        return self.add(t, u)

    def argmax(self, y, n_classes, qseed):
        """SecPE Alg. 1 on a normalised ciphertext y with n_classes valid
        slots (padded to C' = 2^ceil(log2 C)): y <- y + RotR(y, C');
        QuickMax: for i < log2 C': y <- Max(RotL(y, 2^i), y); then
        z = Sign(y_dup - y_max) + 1; levels as level_plan sets them."""
        if n_classes < 2:
            raise ValueError("argmax needs at least 2 classes")
        self.qseed = qseed
        self.ridx = 0
        cp = 1 << (n_classes - 1).bit_length()
        r = cp.bit_length() - 1
        if 2 * cp > self.n // 2:
            raise ValueError("2*C' exceeds the slot count")
        y = self.add(y, self.rotate(y, -cp))
        y_dup = y
        self.plan = self.level_plan(r, y.level)
        try:
            if y.level > self.plan[0]:
                y = self.drop(y, self.plan[0])
            for i in range(r):
                y = self.ensure(y, 1)
                a = self.rotate(y, 1 << i)
                y = self.max(a, y)
            al = self.mul_const(y_dup, 1.0, y.scale, y.level)
            d = self.sub(al, y)
            s = self.sign(d, 0, lowest=True)
        finally:
            self.plan = None
        return self.add_const(s, 1.0)

    def phoenix_argmax(self, y, n_classes, qseed):
        """The Phoenix Argmax the paper compares against (SecPE Sec. 3.2):
        every slot compared with its m = C' - 1 cyclic neighbours,
        s = sum_i Sign(y - RotL(y, i)), i = 1..m, then z from s by a linear
        map and one more Sign: m + 1 Signs and m + 1 rotations.  READINGS
        (the paper defers the details to Phoenix): the comparisons wrap
        around the C' slots of y, padded as for Alg. 1, through the same
        duplication y + RotR(y, C'); the max slot has s = m and every other
        slot s <= m - 2, so z = (Sign((s - (m - 1)) / (2m)) + 1) / 2, the 1/2
        folded into the last polynomial of that Sign; comparison i draws its
        refresh randomness from the seed stream(qseed, 7, i) and the final
        Sign from stream(qseed, 7, 0), each counting refreshes from 0."""
        if n_classes < 2:
            raise ValueError("argmax needs at least 2 classes")
        cp = 1 << (n_classes - 1).bit_length()
        if 2 * cp > self.n // 2:
            raise ValueError("2*C' exceeds the slot count")
        m = cp - 1
        y = self.add(y, self.rotate(y, -cp))
        s = None
        for i in range(1, m + 1):
            self.qseed, self.ridx = self.stream(qseed, DOM_PHOENIX, i), 0
            si = self.sign(self.sub(y, self.rotate(y, i)), 1)
            s = si if s is None else self.add(s, si)
        t = self.mul_const(self.add_const(s, -(m - 1.0)), 1.0 / (2 * m), self.p.scale, s.level - 1)
        self.qseed, self.ridx = self.stream(qseed, DOM_PHOENIX, 0), 0
        z = self.sign(t, 0, last_factor=0.5, lowest=True)
        return self.add_const(z, 0.5)

    # ---------------------------------------- upstream encrypted linear step
    def mul_plain(self, ct, m, pt_scale):
        """Slot-wise product with the plaintext of integer coefficients m
        encoded at scale pt_scale, then the rescale: scale s * pt_scale / q_l."""
        lv = ct.level
        P = self.ntt_of_signed(np.array([int(v) for v in m], dtype=np.int64), list(range(lv + 1)))
        c = np.empty_like(ct.c)
        for k in range(2):
            for pi in range(lv + 1):
                c[k, pi] = self.vmul(ct.c[k, pi], P[pi], pi)
        return self.rescale(Ct(c, lv, ct.scale * pt_scale))

    def add_plain(self, ct, m):
        """ct + (plaintext of integer coefficients m, 0): m must be encoded at
        ct's scale."""
        P = self.ntt_of_signed(np.array([int(v) for v in m], dtype=np.int64), list(range(ct.level + 1)))
        out = ct.copy()
        for pi in range(ct.level + 1):
            out.c[0, pi] = self.vadd(ct.c[0, pi], P[pi], pi)
        return out

    def replicated_slots(self, x, n_classes):
        """x[d] with x[j] repeated in the C' slots [j C', (j+1) C') (READING of
        the layout of the CLIP-style linear step, Sec. 2.3)."""
        cp = 1 << (n_classes - 1).bit_length()
        return np.repeat(np.asarray(x, dtype=np.float64), cp)

    def encrypt_replicated(self, x, n_classes, seed):
        return self.encrypt(self.replicated_slots(x, n_classes), seed)

    def linear_plaintexts(self, T, d_min, level=None):
        """Integer coefficients of the linear step's plaintexts for weights
        T[K][C][d]: W_i (T_i[c][j] at slot j C' + c) at scale q_level, the
        mask (1 on slots [0, C)) at scale q_(level-1), the pad (d_min on
        [C, C')) at scale Delta."""
        level = self.ctx.L if level is None else level
        T = np.asarray(T, dtype=np.float64)
        K, C, d = T.shape
        cp = 1 << (C - 1).bit_length()
        Wm = []
        for i in range(K):
            v = np.zeros(d * cp)
            for j in range(d):
                v[j * cp: j * cp + C] = T[i, :, j]
            Wm.append(self.encode_coeffs(v, float(self.primes[level])))
        mask = np.zeros(cp)
        mask[:C] = 1.0
        pad = np.zeros(cp)
        pad[C:] = d_min
        return Wm, self.encode_coeffs(mask, float(self.primes[level - 1])), self.encode_coeffs(pad, self.p.scale)

    def linear_logits(self, x, plaintexts, n_classes, d):
        """The K prompts' logit ciphertexts y_i = mask (.) sum_t RotL(W_i (.)
        x, C' 2^t) (accumulated) + pad, each product rescaled: for prompt i,
        slot c < C holds <T_i[c], x> (SecPE Sec. 2.3, CLIP ensembling)."""
        Wm, mask_m, pad_m = plaintexts
        cp = 1 << (n_classes - 1).bit_length()
        outs = []
        for m in Wm:
            p = self.mul_plain(x, m, float(self.primes[x.level]))
            s = cp
            while s < cp * d:
                p = self.add(p, self.rotate(p, s))
                s <<= 1
            p = self.mul_plain(p, mask_m, float(self.primes[p.level]))
            outs.append(self.add_plain(p, pad_m))
        return outs

    def aggregate(self, cts, d_min, d_max):
        """Ensemble aggregation (SecPE Sec. 3.1 step 3) with the normalisation
        of Eq. norm folded into one constant: y = (sum_i ct_i) * w,
        w = 1 / (K (D_max - D_min)), landing at level L-1 with scale Delta.
        The shift -D_min/(D_max-D_min) of Eq. norm is dropped: Alg. 1's output
        is invariant under a common shift, and an unmasked shift would break
        the zero padding that Alg. 1's duplication step relies on."""
        K = len(cts)
        y = cts[0]
        for c in cts[1:]:
            y = self.add(y, c)
        w = 1.0 / (K * (d_max - d_min))
        return self.mul_const(y, w, self.p.scale, y.level - 1)
