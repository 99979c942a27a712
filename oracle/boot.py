"""CKKS bootstrapping in the oracle.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only tests/, the smoke check and the
benchmark's CPU legs may import the oracle.

SecPE evaluates its Argmax with bootstrapping (Sec. 2.2: it refreshes a
ciphertext's levels; Sec. 4.1: N = 2^16, L = 35, bootstrapping depth 14)
but does not describe the procedure.  READING: the sparse-slot
bootstrapping of Cheon, Han, Kim, Kim and Song ("Bootstrapping for
approximate homomorphic encryption", Eurocrypt 2018) with the sub-sum of
Chen, Chillotti and Song ("Improved bootstrapping for approximate
homomorphic encryption", Eurocrypt 2019), for a sparse secret of Hamming
weight h and a block of n slots (2n <= N/2):

1. ModRaise: the level-0 ciphertext (c0, c1) mod q0, lifted to centred
   integers and reduced modulo q_0..q_L, decrypts to t = m + q0 I with
   |I_k| <= (h + 1)/2.
2. SubSum: y <- y + RotL(y, 2^j) for 2^j = n .. N/4: the slot vector becomes
   the n-periodic block sum, the polynomial (N/2n) Pi(t), Pi keeping the
   coefficients at multiples of N/(2n) (the subring in Y = X^(N/2n)).
3. CoeffToSlot: with p the 2n subring coefficients of Pi(t) and w the slots
   under the label q0 (N/2) / n, (p_lo + i p_hi) / q0 = (1/n) V^H w,
   V[j][a] = omega^(a 5^j), omega = exp(i pi / 2n); a plaintext linear
   transform of w and of its conjugate puts u = p / q0 (real) into slots
   [0, n) (low half) and [n, 2n) (high half) of every 2n-block.
4. EvalMod: u = m'/q0 + I', and sin(2 pi u) / (2 pi) = m'/q0 up to O(u^3):
   cos(2 pi (u - 1/4) / 2^r) by its Taylor polynomial (degree 12), then r
   double angles cos 2x = 2 cos^2 x - 1.
5. SlotToCoeff: the inverse transform, z = (q0 / 2 pi) V (f_lo + i f_hi) /
   label, back to the slot layout of the input.

The result decrypts to the n-periodic block average of the input's slots
(READING: the convention under which bootstrapping is the identity on the
inputs it is meant for): an n-periodic input (a block of n slots repeated,
which the client produces by packing its query into every block) comes
back unchanged; data in slots [0, n) with zeros beyond come back divided by
N/(2n) and replicated.  Every linear transform is a baby-step giant-step sum of
plaintext diagonals; every plaintext is encoded by the direct
canonical-embedding sums of ckks.Oracle.encode_complex.
"""
import math

import numpy as np

from .ckks import Ct, STEP_CONJ

R_DOUBLINGS = 8      # double angles after the Taylor polynomial
TAYLOR_TERMS = 7     # cos(x) = sum_{k < 7} (-1)^k x^(2k) / (2k)!


def bsgs_split(n_diag):
    """(baby, giant) with baby * giant = n_diag, baby = 2^ceil(log2(n)/2)."""
    lg = n_diag.bit_length() - 1
    bs = 1 << ((lg + 1) // 2)
    return bs, n_diag // bs


def subring_vandermonde(n):
    """V[j][a] = omega^(a 5^j mod 4n), omega = exp(i pi / 2n): the slot
    values of a subring polynomial sum_a p_a Y^a with Y = X^(N/2n), for the
    first n coefficients (the other n enter multiplied by i)."""
    e = np.array([pow(5, j, 4 * n) for j in range(n)], dtype=np.int64)
    a = np.arange(n, dtype=np.int64)
    return np.exp(1j * np.pi * ((np.outer(e, a) % (4 * n)).astype(np.float64)) / (2 * n))


class BootPlan:
    """Matrices, diagonals and plaintexts of the bootstrapping of one
    parameter set and block size n (the rotation steps it needs are in
    `rotation_steps`)."""

    def __init__(self, o, n):
        S = o.n // 2
        assert n & (n - 1) == 0 and 2 * n <= S
        self.o, self.n, self.S = o, n, S
        self.q0 = o.primes[0]
        L = o.ctx.L
        self.level_c2s = L
        self.out_level = L - 16    # the circuit's 16 levels (checked in bootstrap)
        V = subring_vandermonde(n)
        G = V.conj().T / n                                      # n x n
        A = np.zeros((2 * n, n), dtype=np.complex128)
        B = np.zeros((2 * n, n), dtype=np.complex128)
        A[:n], A[n:] = G / 2, G / 2j
        B[:n], B[n:] = G.conj() / 2, -G.conj() / 2j
        # CoeffToSlot: input period n, output period 2n: n diagonals each
        self.c2s_bs, self.c2s_gs = bsgs_split(n)
        j = np.arange(S)
        self.c2s_A = [A[j % (2 * n), (j + k) % n] for k in range(n)]
        self.c2s_B = [B[j % (2 * n), (j + k) % n] for k in range(n)]
        # SlotToCoeff: input period 2n (real), output period n: 2n diagonals
        H = (self.q0 / (2 * math.pi)) * V                         # n x n, before the output label
        M = np.zeros((n, 2 * n), dtype=np.complex128)
        M[:, :n], M[:, n:] = H, 1j * H
        self.s2c_bs, self.s2c_gs = bsgs_split(2 * n)
        self.s2c_M = [M[j % n, (j + k) % (2 * n)] for k in range(2 * n)]
        self._pt = {}

    def rotation_steps(self):
        steps = {STEP_CONJ}
        s = self.n
        while s < self.S:
            steps.add(s)
            s <<= 1
        for bs, gs in ((self.c2s_bs, self.c2s_gs), (self.s2c_bs, self.s2c_gs)):
            steps.update(range(1, bs))
            steps.update(g * bs for g in range(1, gs))
        return sorted(steps)

    # ------------------------------------------------------------ plaintexts
    def plaintext(self, key, values, scale):
        """Integer coefficients of a complex slot vector at `scale` (cached
        by key)."""
        if key not in self._pt:
            self._pt[key] = self.o.encode_complex(values, scale)
        return self._pt[key]

    @staticmethod
    def shifted(diag, s):
        """RotR of a slot vector by s: out[j] = diag[(j - s) mod len]."""
        return np.roll(diag, s)

    # ------------------------------------------------------------ steps
    def mod_raise(self, ct):
        """Level-0 ciphertext -> the same coefficients, centred mod q0, at the
        top level; label q0 (N/2) / n (the CoeffToSlot convention)."""
        o = self.o
        assert ct.level == 0
        q0 = self.q0
        L = o.ctx.L
        out = np.empty((2, L + 1, o.n), dtype=np.uint64)
        for k in range(2):
            c = ct.c[k, 0].copy()
            o.intt(c, 0)
            cen = np.where(c > q0 // 2, c.astype(object) - q0, c.astype(object))
            cen = np.array([int(v) for v in cen], dtype=np.int64)
            out[k] = o.ntt_of_signed(cen, list(range(L + 1)))
        return Ct(out, L, float(q0) * self.S / self.n)

    def sub_sum(self, ct):
        """y <- y + RotL(y, s) for s = n, 2n, .., N/4."""
        s = self.n
        while s < self.S:
            ct = self.o.add(ct, self.o.rotate(ct, s))
            s <<= 1
        return ct

    def _bsgs(self, inputs, diags, bs, gs, key, pt_scale, out_scale=None):
        """sum_k diag_k (.) RotL(x, k) over the inputs (x, diagonals) as
        sum_g RotL(sum_b RotR(diag_{g bs + b}, g bs) (.) RotL(x, b), g bs),
        every inner sum rescaled once; plaintexts at pt_scale; the baby steps
        RotL(x, b) of one input by rotate_hoisted."""
        o = self.o
        lv = inputs[0][0].level
        # the baby steps of one input share one ModUp (hoisting)
        baby = [[x] + o.rotate_hoisted(x, list(range(1, bs))) for x, _ in inputs]
        total = None
        for g in range(gs):
            acc = np.zeros((2, lv + 1, o.n), dtype=np.uint64)
            for t, (x, dg) in enumerate(inputs):
                for b in range(bs):
                    m = self.plaintext((key, t, g, b), self.shifted(dg[g * bs + b], g * bs), pt_scale)
                    P = o.ntt_of_signed(np.array([int(v) for v in m], dtype=np.int64), list(range(lv + 1)))
                    for k in range(2):
                        for pi in range(lv + 1):
                            acc[k, pi] = o.vadd(acc[k, pi], o.vmul(baby[t][b].c[k, pi], P[pi], pi), pi)
            inner = o.rescale(Ct(acc, lv, inputs[0][0].scale * pt_scale))
            if out_scale is not None:
                inner.scale = out_scale
            if g:
                inner = o.rotate(inner, g * bs)
            total = inner if total is None else o.add(total, inner)
        return total

    def coeff_to_slot(self, w):
        """u = p / q0 into slots [0, n) (low coefficients) and [n, 2n) (high)
        of every 2n-block, from w and its conjugate; plaintexts at scale
        q_level, so the label is kept."""
        o = self.o
        wc = o.rotate(w, STEP_CONJ)
        return self._bsgs([(w, self.c2s_A), (wc, self.c2s_B)], None, self.c2s_bs, self.c2s_gs, "c2s",
                          float(o.primes[w.level]))

    def eval_mod(self, u):
        """sin(2 pi u): cos(2 pi (u - 1/4) / 2^r) by the Taylor polynomial
        sum_{k<7} (-1)^k x^(2k) / (2k)!, evaluated as P0(y) + y^3 P1(y) in
        y = x^2 (P0 = c0 + c1 y + c2 y^2, P1 = c3 + c4 y + c5 y^2 + c6 y^3),
        then r double angles c <- 2c^2 - 1.  Working label: the top prime q_L
        (the label of a product of two such values stays near it)."""
        o = self.o
        wl = float(o.primes[o.ctx.L])
        a = 2 * math.pi / (1 << R_DOUBLINGS)
        c = [(-1) ** k / math.factorial(2 * k) for k in range(TAYLOR_TERMS)]
        x = o.add_const(o.mul_const(u, a, wl, u.level - 1), -a / 4)
        y = o.mul(x, x)
        y2 = o.mul(y, y)
        y3 = o.mul(y2, y)
        lp1 = y3.level - 1
        t1 = wl * float(o.primes[lp1]) / y3.scale
        p1 = o.add_const(o.add(o.lincomb([(y, c[4]), (y2, c[5])], t1, lp1), o.lincomb([(y3, c[6])], t1, lp1)), c[3])
        prod = o.relin_rescale(o.tensor(y3, p1))
        p0 = o.add_const(o.lincomb([(y, c[1]), (y2, c[2])], prod.scale, prod.level), c[0])
        cs = o.add(prod, p0)
        for _ in range(R_DOUBLINGS):
            d = o.mul(cs, cs)
            cs = o.add_const(o.add(d, d), -1.0)
        return cs

    def slot_to_coeff(self, f, out_scale):
        """The block average of the original slots, label out_scale: slots
        (q0 / 2 pi) V (f_lo + i f_hi) / out_scale, as plaintexts at scale
        q_level out_scale / label(f) carrying (q0 / 2 pi) V."""
        pt_scale = float(self.o.primes[f.level]) / f.scale
        return self._bsgs([(f, self.s2c_M)], None, self.s2c_bs, self.s2c_gs, "s2c", pt_scale,
                          out_scale=out_scale)

    def bootstrap(self, ct):
        """Level-0 (or any-level, dropped to 0) ciphertext -> the n-periodic
        block average of its slots at level L - 16, with ct's label."""
        o = self.o
        lab = ct.scale
        x = self.mod_raise(o.drop(ct, 0))
        x = self.sub_sum(x)
        u = self.coeff_to_slot(x)
        f = self.eval_mod(u)
        z = self.slot_to_coeff(f, lab)
        assert z.level == self.out_level
        return z
