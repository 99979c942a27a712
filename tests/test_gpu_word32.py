"""Word-size probe on the GPU (secpe_ntt32*, secpe_bconv32): 32-bit residues
under the about-29-bit primes of the WORD32 prime chain, N = 2^16.

* the forward transform of every limb equals the oracle's NTT residue for
  residue (same network and ordering as the 64-bit path), the inverse gives
  the input back exactly, and the inverse of the oracle's transform too;
* the fast base conversion of a 14-limb digit to 42 other primes equals the
  oracle's FastBConv, item by item;
* the hybrid key switching of 32-bit residues (ModUp, inner product with
  the oracle's relinearisation key, rounded ModDown), unfused and fused,
  equals the oracle's keyswitch residue for residue;
* bad tables and arguments are refused on the host."""
import numpy as np
import pytest

from oracle import Oracle
from oracle.params import WORD32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    pkg_build.build()
    torch.cuda.set_device(0)
    o = Oracle(WORD32)
    primes = [int(q) for q in o.primes]
    t = secpe.Ntt32(primes)
    yield o, primes, t, secpe, torch
    t.close()


def _to_dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _to_host(x):
    return x.cpu().numpy().view(np.uint32).astype(np.uint64)


def test_ntt32_matches_oracle(env):
    o, primes, t, secpe, torch = env
    rng = np.random.default_rng(31)
    idx = [0, 5, 17, 30, 47, 48, 55, 3]
    a = np.stack([rng.integers(0, primes[i], o.n, dtype=np.uint64) for i in idx])
    x = _to_dev(torch, a)
    t.ntt(x, idx)
    got = _to_host(x)
    for r, i in enumerate(idx):
        want = a[r].copy()
        o.ntt(want, i)
        assert np.array_equal(got[r], want), i
    t.ntt(x, idx, inverse=True)
    assert np.array_equal(_to_host(x), a)
    # the inverse of the oracle's forward transform
    f = a.copy()
    for r, i in enumerate(idx):
        o.ntt(f[r], i)
    y = _to_dev(torch, f)
    t.ntt(y, idx, inverse=True)
    assert np.array_equal(_to_host(y), a)


def test_bconv32_matches_oracle(env):
    o, primes, t, secpe, torch = env
    rng = np.random.default_rng(32)
    src = list(range(14))
    dst = list(range(14, 48)) + list(range(48, 56))
    B = 2
    x = np.stack([np.stack([rng.integers(0, primes[i], o.n, dtype=np.uint64) for i in src]) for _ in range(B)])
    xd = _to_dev(torch, x)
    out = torch.zeros((B, len(dst), o.n), dtype=torch.int32, device="cuda")
    t.bconv(xd, src, out, dst)
    got = _to_host(out).reshape(B, len(dst), o.n)
    for b in range(B):
        want = o.fast_bconv(x[b], src, dst)
        assert np.array_equal(got[b], want), b


def test_keyswitch32_matches_oracle(env):
    import torch
    from oracle import Params
    _, _, _, secpe, _ = env
    p = Params(log_n=16, q0_bits=29, q_bits=29, n_q=12, p_bits=29, n_p=4, dnum=3, log_scale=29)
    o = Oracle(p)
    o.keygen(33)
    nq, L = p.n_q, p.n_q - 1
    t = secpe.Ntt32([int(q) for q in o.primes])
    rng = np.random.default_rng(34)
    B = 2
    d = np.stack([np.stack([rng.integers(0, o.primes[i], o.n, dtype=np.uint64) for i in range(nq)])
                  for _ in range(B)])
    key = _to_dev(torch, o.rlk)
    want = [o.keyswitch(d[b], L, o.rlk) for b in range(B)]
    for fused in (False, True):
        out = torch.zeros((B, 2, nq, o.n), dtype=torch.int32, device="cuda")
        t.keyswitch(_to_dev(torch, d), list(range(nq)), list(range(nq, nq + p.n_p)), p.alpha, key, out, fused)
        got = _to_host(out).reshape(B, 2, nq, o.n)
        for b in range(B):
            assert np.array_equal(got[b, 0], want[b][0]) and np.array_equal(got[b, 1], want[b][1]), (fused, b)
    t.close()


def test_word32_rejects_bad_arguments(env):
    o, primes, t, secpe, torch = env
    with pytest.raises(secpe.SecpeError):
        secpe.Ntt32([primes[0]], log_n=12)                 # only N = 2^16
    with pytest.raises(secpe.SecpeError):
        secpe.Ntt32([(1 << 30) + 1])                        # not below 2^30
    with pytest.raises(secpe.SecpeError):
        secpe.Ntt32([primes[0] + 2])                        # not prime / not 1 mod 2N
    x = torch.zeros((2, o.n), dtype=torch.int32, device="cuda")
    with pytest.raises(secpe.SecpeError):
        t.ntt(x, [0, 56])                                   # index outside the table
    out = torch.zeros((1, 2, o.n), dtype=torch.int32, device="cuda")
    with pytest.raises(secpe.SecpeError):
        t.bconv(x.view(1, 2, o.n), [0, 0], out, [1, 2])     # repeated input prime
