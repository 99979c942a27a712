"""Host-side validation of the entry points added around the Argmax (slot
packing, Phoenix, the linear step, bootstrapping): each bad argument returns
its status code before anything is launched (no GPU fault is involved), and
the context keeps working afterwards."""
import numpy as np
import pytest

from oracle import BOOT_TOY, TOY
from paper_2502_00847_gb300 import workloads

pytestmark = pytest.mark.gpu

EINVAL, ELEVEL, EKEY = -1, -3, -5


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe
    pkg_build.build()
    torch.cuda.set_device(0)
    ctx = secpe.Context.from_params(TOY)
    keys = secpe.Keys(ctx, 41, [1, -2])
    return ctx, keys, secpe


def _code(fn):
    from paper_2502_00847_gb300 import secpe
    with pytest.raises(secpe.SecpeError) as e:
        fn()
    return e.value.code


def test_packing_errors(env):
    ctx, keys, secpe = env
    cap = secpe.packed_capacity(12, 3)
    assert cap == 256
    assert _code(lambda: secpe.encrypt_logits_packed(ctx, keys, np.zeros((cap + 1, 3)), -1.0, 1)) == EINVAL
    assert _code(lambda: secpe.encode_packed(12, 2.0 ** 40, np.zeros((0, 3)), -1.0)) == EINVAL
    assert secpe.packed_capacity(12, 2048) == 0 and _code(lambda: secpe.packed_capacity(3, 4)) == EINVAL


def test_phoenix_errors(env):
    ctx, keys, secpe = env
    ct = secpe.encrypt(ctx, keys, np.zeros(4), 2)
    before = ctx.counters()["launches"]
    assert _code(lambda: secpe.phoenix_argmax(ctx, keys, ct, 1, 0)) == EINVAL        # C = 1
    assert ctx.counters()["launches"] == before
    assert _code(lambda: secpe.phoenix_argmax(ctx, keys, ct, 4, 0)) == EKEY          # no RotR(4) key


def test_linear_errors(env):
    ctx, keys, secpe = env
    T = np.zeros((2, 3, 48))
    assert _code(lambda: secpe.Linear(ctx, T=T, d_min=-1.0)) == EINVAL              # d not a power of two
    assert _code(lambda: secpe.Linear(ctx, T=np.zeros((1, 3, 1024)), d_min=-1.0)) == EINVAL   # d C' > N/2
    lin = secpe.Linear(ctx, T=np.zeros((2, 3, 8)), d_min=-1.0)
    x = secpe.encrypt_replicated(ctx, keys, np.zeros(8), 3, 5)
    low = secpe.Ciphertext(x.data, ctx.L - 1, x.scale)
    assert _code(lambda: lin.apply(keys, low)) == ELEVEL
    assert _code(lambda: lin.apply(keys, x)) == EKEY                                 # rotations by C' 2^t
    lin.close()


def test_bootstrap_and_batch_errors(env):
    ctx, keys, secpe = env
    assert _code(lambda: secpe.Boot(ctx, 16)) == EINVAL          # dense secret, no bootstrapping primes
    bctx = secpe.Context.from_params(BOOT_TOY)
    assert _code(lambda: secpe.Boot(bctx, 12)) == EINVAL         # block not a power of two
    assert _code(lambda: secpe.Boot(bctx, 2048)) == EINVAL       # 2n > N/2
    assert _code(lambda: secpe.Boot(bctx, 1 << 30)) == EINVAL    # 2n beyond 32 bits
    bk = secpe.Keys(bctx, 3, [1, -2])
    bt = secpe.Boot(bctx, 16)
    ct = secpe.encrypt(bctx, bk, np.zeros(16), 4)
    assert _code(lambda: bt.bootstrap(bk, ct)) == EKEY             # no conjugation / sub-sum keys
    q = workloads.toy_query(seed=7, K=2, C=9)                      # 2C' = 32 > n = 16
    cts = [secpe.encrypt_logits(bctx, bk, q.logits[i], q.d_min, q.enc_seeds[i]) for i in range(q.K)]
    b = [dict(cts=cts, C=q.C, d_min=q.d_min, d_max=q.d_max, qseed=q.qseed, z_out=bctx.new_ct())]
    assert _code(lambda: secpe.argmax_batch_boot(bctx, bk, bt, b)) == EINVAL
    bt.close()
    # the batched driver wants one input level per call
    q2 = workloads.toy_query(seed=8, K=2, C=2)
    c2 = [secpe.encrypt_logits(ctx, keys, q2.logits[i], q2.d_min, q2.enc_seeds[i]) for i in range(2)]
    c2[1] = secpe.Ciphertext(c2[1].data, ctx.L - 1, c2[1].scale)
    b2 = [dict(cts=c2, C=2, d_min=q2.d_min, d_max=q2.d_max, qseed=1, z_out=ctx.new_ct())]
    assert _code(lambda: secpe.argmax_batch(ctx, keys, b2)) == EINVAL
    assert ctx.stream_status() == 0 and bctx.stream_status() == 0
