"""Oracle: a plain, slow, obviously correct CPU implementation of SecPE's
encrypted ensemble Argmax on RNS-CKKS (SecPE Sec. 2.2, Sec. 3.2, Alg. 1).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline / reference legs may import, call, link or run
anything in this package.  It shares no code with the CUDA library and does
not import it.
"""
from .params import Params, Context, PRESETS, TOY, MICRO, ARGMAX, ARGMAX8, BOOT_TOY, BOOT16, WORD32  # noqa: F401
from .ckks import Oracle, Ct  # noqa: F401
from ._lib import build  # noqa: F401
