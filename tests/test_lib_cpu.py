"""CPU-side checks of the CUDA library: it builds, loads, exports every
function include/secpe.h declares, and its host-side prime selection equals
the oracle's (no GPU needed)."""
import os
import re

import pytest

from oracle.params import ARGMAX, MICRO, TOY, Params, select_primes
from paper_2502_00847_gb300 import build as pkg_build
from paper_2502_00847_gb300 import secpe

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "secpe.h")


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return secpe.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(secpe_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert sorted(declared_functions()) == sorted(secpe.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_strerror(lib):
    assert lib.secpe_strerror(0) == b"ok"
    assert lib.secpe_strerror(-5) == b"missing key"
    assert lib.secpe_strerror(-99) == b"unknown error"


def _as_dict(p):
    return {k: getattr(p, k) for k in ("log_n", "q0_bits", "q_bits", "n_q", "p_bits", "n_p", "dnum",
                                       "log_scale", "sign_dg", "sign_df", "reserve")}


@pytest.mark.parametrize("p", [TOY, MICRO, ARGMAX,
                               Params(log_n=10, q0_bits=55, q_bits=36, n_q=7, p_bits=58, n_p=3, dnum=3,
                                      log_scale=36),
                               Params(log_n=13, q0_bits=45, q_bits=45, n_q=5, p_bits=50, n_p=2, dnum=2,
                                      log_scale=45)],
                         ids=["toy", "micro", "argmax", "odd1", "odd2"])
def test_prime_selection_matches_oracle(lib, p):
    q, sp = secpe.select_primes(**_as_dict(p))
    oq, osp = select_primes(p)
    assert q == oq and sp == osp


def test_prime_selection_rejects_bad_params(lib):
    bad = _as_dict(TOY)
    bad["log_n"] = 30
    with pytest.raises(secpe.SecpeError) as e:
        secpe.select_primes(**bad)
    assert e.value.code == -1


def test_context_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(secpe.SecpeError) as e:
        secpe.Context.from_params(TOY)
    assert e.value.code == -6


def test_package_presets_match_the_oracles():
    """The library's named parameter sets (numbers only) are the ones the
    oracle defines, field by field."""
    import dataclasses

    from oracle import params as oparams
    from paper_2502_00847_gb300 import presets
    assert set(presets.PRESETS) == set(oparams.PRESETS)
    for name, p in presets.PRESETS.items():
        for f in dataclasses.fields(p):
            assert getattr(p, f.name) == getattr(oparams.PRESETS[name], f.name), (name, f.name)
