"""Level-aware QuickMax (a reading: the paper does not discuss levels).

Range by range, the plan starts each refresh range as low as every refresh
staying at its step allows.  Pins:
* hand-derived plans of the argmax8 parameter set (walked below by hand);
* the library's host-side plan (secpe_level_plan) equals the oracle's for
  every preset, class count and both refresh levels;
* on the real toy circuit the refreshes happen at the same points as with
  the greedy levels, every relinearisation runs on at most as many limbs,
  the result is the same Argmax, and one level lower for any range moves or
  adds a refresh or runs out of levels (the plan is the largest drop)."""
import numpy as np
import pytest

from oracle import ARGMAX8, BOOT16, BOOT_TOY, TOY, Oracle
from paper_2502_00847_gb300 import build as pkg_build
from paper_2502_00847_gb300 import secpe


def test_argmax8_plans_by_hand():
    """argmax8: L = 23, reserve 1, 4 polynomials per Sign; a test of level l
    for a step that needs k passes when l >= k + 1; y enters at 22.
    r = 1: round 0 runs its polynomials at 22, 18, 14, 10 (needs 2, 5, 5, 5,
    6) and leaves t at min(22, 6) - 1 = 5.  The final Sign's first
    polynomial passes at 5 (y at 21 would leave t at 4 and refresh there, so
    22 stays); its second refreshes; after that the lowest-level clamp puts
    the input at 13 anyway, and 12 would leave the last polynomial at 4 and
    refresh again: [22, 13].
    r = 2: round 1 refreshes at its second polynomial; from p the rest of
    its polynomials need p - 4 >= 5 and p - 8 >= 6, so p = 14 (t =
    min(5, 2) - 1 = 1 and the final Sign refreshes at its first polynomial,
    as it does from 23); after that refresh the final Sign needs p - 12 >= 5:
    [22, 14, 17].
    r = 3: as for r = 2, but the first test of QuickMax round k = 2 must still pass:
    t = min(5, p - 12) - 1 >= 2 gives p = 15; round k = 2 refreshes at its first
    polynomial and from p needs p - 12 >= 6, p = 18: [22, 15, 18, 17]."""
    o = Oracle(ARGMAX8)
    assert o.level_plan(1, 22) == [22, 13]
    assert o.level_plan(2, 22) == [22, 14, 17]
    assert o.level_plan(3, 22) == [22, 15, 18, 17]


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return secpe.lib()


def _as_dict(p):
    return {k: getattr(p, k) for k in ("log_n", "q0_bits", "q_bits", "n_q", "p_bits", "n_p", "dnum",
                                       "log_scale", "sign_dg", "sign_df", "reserve", "secret_hw",
                                       "boot_primes", "boot_bits")}


@pytest.mark.parametrize("p", [TOY, ARGMAX8, BOOT_TOY, BOOT16], ids=["toy", "argmax8", "boot_toy", "boot16"])
def test_library_plan_equals_oracle(lib, p):
    o = Oracle(p)
    L = o.ctx.L
    tops = [L] + ([L - 16] if p.boot_primes else [])
    for top in tops:
        for C in (2, 3, 4, 6, 14, 64, 200):
            r = (C - 1).bit_length()
            for entry in sorted({L - 1, L - 17, 5, 1 + p.reserve} & set(range(1 + p.reserve, L))):
                o.boot_plan = None if top == L else _Top(top)
                want = o.level_plan(r, entry)
                assert secpe.level_plan(C, entry, top, **_as_dict(p)) == want, (top, C, entry)
    o.boot_plan = None


class _Top:
    """Stands in for a bootstrapping plan: only its output level is read."""

    def __init__(self, lv):
        self.out_level = lv


def test_library_plan_rejects_bad_arguments(lib):
    d = _as_dict(TOY)
    # C = 1; entry below 0; refresh level above L or 0; C above N/4 (no room
    # for 2 C' slots, and far beyond: C' would overflow 32 bits)
    for C, entry, top in ((1, 10, 11), (4, -1, 11), (4, 10, 12), (4, 10, 0), (1025, 10, 11),
                          (2 ** 30 + 1, 10, 11), (2 ** 31 - 1, 10, 11)):
        with pytest.raises(secpe.SecpeError):
            secpe.level_plan(C, entry, top, **d)


def _trace(o, y, C, qseed, plan_on, monkeypatch, plan=None):
    """Runs the oracle's Argmax; returns (z, relin levels, refresh points:
    the index of the level test (ensure call) that refreshed).  plan_on
    False: greedy levels; plan: a given plan."""
    levels, points, tests = [], [], [0]
    relin0, refresh0, ensure0 = Oracle.relin_rescale, Oracle.refresh, Oracle.ensure
    lp0 = Oracle.level_plan

    def relin(self, d):
        levels.append(d.level)
        return relin0(self, d)

    def ensure(self, ct, k):
        tests[0] += 1
        return ensure0(self, ct, k)

    def refresh(self, ct, qs):
        points.append(tests[0])
        return refresh0(self, ct, qs)

    def level_plan(self, r, entry):
        if plan is not None:
            return list(plan)
        if not plan_on:
            return [entry] + [self.refresh_level()] * 64
        return lp0(self, r, entry)

    with monkeypatch.context() as m:
        m.setattr(Oracle, "relin_rescale", relin)
        m.setattr(Oracle, "refresh", refresh)
        m.setattr(Oracle, "ensure", ensure)
        m.setattr(Oracle, "level_plan", level_plan)
        z = o.argmax(y, C, qseed=qseed)
    return z, levels, points


@pytest.mark.parametrize("C", [2, 3])
def test_toy_circuit_keeps_refreshes_and_is_maximal(C, monkeypatch):
    o = Oracle(TOY)
    cp = 1 << (C - 1).bit_length()
    r = cp.bit_length() - 1
    o.keygen(810 + C, rot_steps=[-cp] + [1 << i for i in range(r)])
    rng = np.random.default_rng(C)
    logits = rng.uniform(-1, 1, (2, C))
    logits[0, 1] += 0.5
    cts = [o.encrypt_logits(logits[i], C, -1.0, seed=3000 + i) for i in range(2)]
    y = o.aggregate(cts, -1.0, 1.0)
    plan = o.level_plan(r, y.level)
    zg, lg, pg = _trace(o, y, C, 21, False, monkeypatch)
    zp, lp, pp = _trace(o, y, C, 21, True, monkeypatch)
    assert pp == pg and len(lp) == len(lg)
    assert all(a <= b for a, b in zip(lp, lg)) and sum(lp) < sum(lg)
    dg, dp = o.decrypt(zg, C), o.decrypt(zp, C)
    assert int(np.argmax(dp)) == int(np.argmax(dg)) == int(np.argmax(logits.mean(0)))
    assert np.max(np.abs(dp - dg)) < 2.0 ** -10
    # one level lower anywhere: a refresh moves or is added, or levels run out
    for j in range(len(plan)):
        low = list(plan)
        low[j] -= 1
        try:
            _, ll, pl = _trace(o, y, C, 21, True, monkeypatch, plan=low)
        except ValueError:
            continue
        assert pl != pg, j
