"""Builds and loads the oracle's C core (ring.c) with gcc.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only tests, the smoke check and the
benchmark's CPU-baseline leg may import the oracle.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsecpe_oracle.so")
_SRC = os.path.join(_HERE, "ring.c")

_lib = None


def build(force=False):
    """Compile ring.c into a shared library (plain gcc, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, _SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        u64 = ctypes.c_uint64
        p = ctypes.c_void_p
        i32 = ctypes.c_int
        sigs = {
            "or_powmod": (u64, [u64, u64, u64]),
            "or_bitrev": (u64, [u64, i32]),
            "or_ntt_naive": (None, [p, p, i32, u64, u64]),
            "or_negacyclic_naive": (None, [p, p, p, i32, u64]),
            "or_ntt_fwd": (None, [p, i32, u64, u64]),
            "or_ntt_inv": (None, [p, i32, u64, u64]),
            "or_vmul": (None, [p, p, p, u64, u64]),
            "or_vadd": (None, [p, p, p, u64, u64]),
            "or_vsub": (None, [p, p, p, u64, u64]),
            "or_vscale": (None, [p, u64, p, u64, u64]),
            "or_vaddc": (None, [p, u64, p, u64, u64]),
            "or_vreduce": (None, [p, p, u64, u64]),
            "or_vfrom_signed": (None, [p, p, u64, u64]),
            "or_fast_bconv": (None, [p, p, i32, p, i32, p, u64]),
            "or_automorph_coeff": (None, [p, p, i32, u64, u64]),
            "or_sm_word": (u64, [u64, u64]),
            "or_sm_stream": (u64, [u64, u64, u64]),
            "or_sample_ternary": (None, [u64, p, u64]),
            "or_sample_cbd21": (None, [u64, p, u64]),
            "or_sample_sparse": (None, [u64, p, u64, u64]),
            "or_sample_uniform": (None, [u64, u64, u64, p, u64]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def ptr(a):
    """Address of a C-contiguous numpy array."""
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def u64arr(x):
    return np.ascontiguousarray(x, dtype=np.uint64)
