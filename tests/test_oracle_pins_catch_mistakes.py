"""Planted mistakes: the pins are sensitive, not only passed.

Each case plants one plausible slip in a copy of the oracle, on the CPU, and
runs the pin that covers that step, which must fail:

* the rescale and the ModDown without their rounding term (floor division)
  against the big-integer rounded-division pins;
* rotations in the wrong direction (5^-r for 5^r) against np.roll;
* the tensor product without one cross term against the plaintext product;
* the transform without its psi^k twist (a cyclic instead of a negacyclic
  NTT, self-consistent: encryption and decryption still work) against the
  plaintext product;
* the slot order on powers of 3 instead of 5 (self-consistent: the
  encode/decode round trip still passes) against the monomial's closed form;
* a digit typo in the f_4 and g_4 coefficient tables against the closed form
  and g_4's pinned values;
* a rescale that does not divide the scale, against the rounded-division pin
  (which also checks the scale and the decoded values);
* the aggregation without its 1/K, Alg. 1 without its final + 1, and Max
  without the 1/2 folded into Sign's last polynomial, against the toy
  circuit's plaintext simulation and Max's plaintext values;
* bootstrapping's CoeffToSlot built on powers of 3 instead of 5 against the
  raised plaintext's subring coefficients (big-integer decryption);
* slot packing in blocks of C' slots (no room for Alg. 1's duplication),
  packed and read back consistently, against the packed plaintext
  pipeline."""
import numpy as np
import pytest

import test_oracle_boot as boot_pins
import test_oracle_ckks as ckks_pins
import test_oracle_packing as packing_pins
import test_oracle_sign as sign_pins
from oracle import BOOT_TOY, TOY, Oracle
from oracle import boot as oboot
from oracle import signpoly
from oracle.ckks import Ct

KEY_SEED = 20250201
ROT = [1, 2, 3, -2, -4, -8]


class FloorRescale(Oracle):
    def rescale(self, ct):
        lv, ql = ct.level, self.primes[ct.level]
        out = np.empty((2, lv, self.n), dtype=np.uint64)
        for k in range(2):
            y = ct.c[k, lv].copy()
            self.intt(y, lv)
            for pi in range(lv):
                z = self.vreduce(y, pi)          # [c]_{q_l}: no + q_l/2
                self.ntt(z, pi)
                t = self.vsub(ct.c[k, pi], z, pi)
                out[k, pi] = self.vscale(t, pow(ql % self.primes[pi], -1, self.primes[pi]), pi)
        return Ct(out, lv - 1, ct.scale / float(ql))


class FloorModDown(Oracle):
    def moddown(self, acc, level):
        sp = self.ctx.special_idx()
        pc = np.stack([acc[t].copy() for t in sp])
        for r, t in enumerate(sp):
            self.intt(pc[r], t)                  # no + P/2
        conv = self.fast_bconv(pc, sp, list(range(level + 1)))
        out = np.empty((level + 1, self.n), dtype=np.uint64)
        for pi in range(level + 1):
            q = self.primes[pi]
            x = conv[pi].copy()
            self.ntt(x, pi)
            out[pi] = self.vscale(self.vsub(acc[pi], x, pi), pow(self.ctx.P % q, -1, q), pi)
        return out


class ScaleKept(Oracle):
    def rescale(self, ct):
        r = super().rescale(ct)
        r.scale = ct.scale                       # forgot to divide by q_l
        return r


class MaxUnhalved(Oracle):
    def max(self, a, y):
        d = self.sub(a, y)
        s = self.sign(d, 1, last_factor=1.0)     # the 1/2 of (a-y)/2 Sign(a-y) dropped
        t = self.mul(d, s)
        u = self.mul_const(self.add(a, y), 0.5, t.scale, t.level)
        return self.add(t, u)


class TightBlocks(Oracle):
    def pack_slots(self, V, d_min):
        V = np.asarray(V, dtype=np.float64)
        P, C = V.shape
        cp = 1 << (C - 1).bit_length()
        out = np.zeros(P * 2 * cp, dtype=np.float64)
        for b in range(P):                       # stride C' instead of 2 C'
            out[b * cp: b * cp + C] = V[b]
            out[b * cp + C: (b + 1) * cp] = d_min
        return out

    def decrypt_packed(self, ct, P, n_classes):
        cp = 1 << (n_classes - 1).bit_length()
        s = self.decrypt(ct, P * 2 * cp)
        return np.stack([s[b * cp: b * cp + n_classes] for b in range(P)])


class WrongDirection(Oracle):
    def galois(self, r):
        return super().galois(-r)


class DroppedCrossTerm(Oracle):
    def tensor(self, a, b):
        d = super().tensor(a, b)
        lv = d.level
        a, b = self.drop(a, lv), self.drop(b, lv)
        for pi in range(lv + 1):
            d.c[1, pi] = self.vmul(a.c[0, pi], b.c[1, pi], pi)    # a1 b0 dropped
        return d


class DroppedTwist(Oracle):
    _tw = {}

    def _twist(self, a, pi, e):
        key = (self.primes[pi], e)
        if key not in self._tw:
            q = self.primes[pi]
            w = pow(self.ctx.psi[pi], e, q)
            t, x = np.empty(self.n, dtype=np.uint64), 1
            for k in range(self.n):
                t[k] = x
                x = x * w % q
            self._tw[key] = t
        a[:] = self.vmul(np.ascontiguousarray(a), self._tw[key], pi)

    def ntt(self, a, pi):
        self._twist(a, pi, -1)                   # undoes the twist the transform applies
        super().ntt(a, pi)

    def intt(self, a, pi):
        super().intt(a, pi)
        self._twist(a, pi, 1)


def _keyed(cls, rot=()):
    o = cls(TOY)
    o.keygen(KEY_SEED, rot_steps=list(rot))
    return o


def test_floor_rescale_fails_the_rounding_pin():
    with pytest.raises(AssertionError):
        ckks_pins.test_rescale_is_rounded_division(_keyed(FloorRescale))


def test_floor_moddown_fails_the_rounding_pin():
    with pytest.raises(AssertionError):
        ckks_pins.test_moddown_is_rounded_division_by_P(_keyed(FloorModDown))


def test_wrong_rotation_direction_fails_the_roll_pin():
    with pytest.raises(AssertionError):
        ckks_pins.test_rotation_direction(_keyed(WrongDirection, ROT))


def test_dropped_cross_term_fails_the_product_pin():
    with pytest.raises(AssertionError):
        ckks_pins.test_encrypt_decrypt_and_linear_ops(_keyed(DroppedCrossTerm))


def test_dropped_twist_fails_the_product_pin():
    o = _keyed(DroppedTwist)
    # self-consistent: a fresh ciphertext still decrypts
    v = np.random.default_rng(8).uniform(-1, 1, 8)
    assert np.max(np.abs(o.decrypt(o.encrypt(v, seed=3), 8) - v)) < 2.0 ** -20
    with pytest.raises(AssertionError):
        ckks_pins.test_keyswitch_noise_small(o)


def test_slot_order_on_powers_of_3_fails_the_monomial_pin(monkeypatch):
    def pow3(self, count):
        return np.array([pow(3, j, 2 * self.n) for j in range(count)], dtype=np.int64)

    monkeypatch.setattr(Oracle, "_pow5", pow3)
    # self-consistent: the round trip alone does not see it
    ckks_pins.test_encode_decode_roundtrip(Oracle(TOY))
    with pytest.raises(AssertionError):
        ckks_pins.test_decode_of_monomial_is_root_ordering()


def test_f4_digit_typo_fails_the_closed_form_pin(monkeypatch):
    monkeypatch.setattr(signpoly, "F4_NUM", (315, -420, 387, -180, 35))
    with pytest.raises(AssertionError):
        sign_pins.test_f4_table_equals_closed_form()


def test_g4_digit_typo_fails_its_pin(monkeypatch):
    monkeypatch.setattr(signpoly, "G4_NUM", (5850, -34974, 97051, -113492, 46623))
    with pytest.raises(AssertionError):
        sign_pins.test_g4_pinning_properties()


def test_rescale_keeping_the_scale_fails_the_rescale_pin():
    with pytest.raises(AssertionError):
        ckks_pins.test_rescale_is_rounded_division(_keyed(ScaleKept))


def test_aggregation_without_1_over_K_fails_the_circuit_pin(monkeypatch):
    agg = Oracle.aggregate

    def without_k(self, cts, d_min, d_max):
        # weight 1/(d_max - d_min) instead of 1/(K (d_max - d_min))
        return agg(self, cts, d_min, d_min + (d_max - d_min) / len(cts))

    monkeypatch.setattr(Oracle, "aggregate", without_k)
    with pytest.raises(AssertionError):
        ckks_pins.test_toy_argmax_circuit(2, 1)


def test_argmax_without_the_final_plus_one_fails_the_circuit_pin(monkeypatch):
    argmax = Oracle.argmax

    def without_plus_one(self, y, n_classes, qseed):
        return self.add_const(argmax(self, y, n_classes, qseed), -1.0)

    monkeypatch.setattr(Oracle, "argmax", without_plus_one)
    with pytest.raises(AssertionError):
        ckks_pins.test_toy_argmax_circuit(2, 1)


def test_max_without_its_half_fails_the_max_pin():
    with pytest.raises(AssertionError):
        ckks_pins.test_max_keeps_the_scale(_keyed(MaxUnhalved, ROT))


def test_coeff_to_slot_on_powers_of_3_fails_its_pin(monkeypatch):
    def vandermonde3(n):
        e = np.array([pow(3, j, 4 * n) for j in range(n)], dtype=np.int64)
        a = np.arange(n, dtype=np.int64)
        return np.exp(1j * np.pi * ((np.outer(e, a) % (4 * n)).astype(np.float64)) / (2 * n))

    monkeypatch.setattr(oboot, "subring_vandermonde", vandermonde3)
    n = boot_pins.N_BLOCK
    o = Oracle(BOOT_TOY)
    plan = oboot.BootPlan(o, n)
    o.keygen(99, rot_steps=plan.rotation_steps())
    v = np.random.default_rng(1).uniform(-1, 1, n)
    ct = o.drop(o.encrypt(np.tile(v, (o.n // 2) // n), seed=5, level=7), 0)
    x = plan.mod_raise(ct)
    xs = plan.sub_sum(x)
    with pytest.raises(AssertionError):
        boot_pins.test_coeff_to_slot_gives_subring_coefficients(dict(o=o, x=x, xs=xs, u=plan.coeff_to_slot(xs)))


def test_packing_without_room_for_the_duplication_fails_the_packed_pin():
    with pytest.raises(AssertionError):
        packing_pins.test_oracle_packed_argmax_every_input(_keyed(TightBlocks, ROT))
