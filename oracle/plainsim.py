"""FP64 plaintext simulation of the SecPE circuit (slot values only).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.

The same op sequence as the encrypted circuit in ckks.py, applied to real
slot vectors: rotations are np.roll over N/2 slots, Sign is the composite
polynomial evaluated by the same BSGS DAG in exact real arithmetic.  Used to
pin decoded values (layer 2 of parity) and the returned index (layer 3).
"""
import numpy as np

from .signpoly import sign_coeffs_float


def poly9(x, c):
    c1, c3, c5, c7, c9 = c
    x2 = x * x
    x4 = x2 * x2
    x5 = x4 * x
    P1 = c7 * x2 + c9 * x4 + c5
    P0 = c3 * x2 + c1
    return x5 * P1 + x * P0


def sign(x, dg=2, df=2):
    g, f = sign_coeffs_float()
    for c in [g] * dg + [f] * df:
        x = poly9(x, c)
    return x


def rotl(v, r):
    return np.roll(v, -r)


def vmax(a, y, dg=2, df=2):
    d = a - y
    return (a + y) / 2 + (d / 2) * sign(d, dg, df)


def argmax_slots(y, n_classes, dg=2, df=2):
    """Alg. 1 on a slot vector y (normalised, zero beyond C')."""
    cp = 1 << (n_classes - 1).bit_length()
    r = cp.bit_length() - 1
    y = y + rotl(y, -cp)
    y_dup = y
    for i in range(r):
        y = vmax(rotl(y, 1 << i), y, dg, df)
    return sign(y_dup - y, dg, df) + 1.0


def pad_logits(v, n_classes, d_min):
    """Client-side layout (READING for C not a power of two): slots 0..C-1
    hold the logits, slots C..C'-1 hold d_min, zeros beyond."""
    cp = 1 << (n_classes - 1).bit_length()
    out = np.zeros(cp, dtype=np.float64)
    out[:n_classes] = v
    out[n_classes:cp] = d_min
    return out


def ensemble_argmax(logits, d_min, d_max, slots, dg=2, df=2):
    """logits[K][C] -> z over the first C slots (plaintext Alg. 1 pipeline)."""
    logits = np.asarray(logits, dtype=np.float64)
    K, C = logits.shape
    y = np.zeros(slots)
    for i in range(K):
        p = pad_logits(logits[i], C, d_min)
        y[: len(p)] += p
    y = y * (1.0 / (K * (d_max - d_min)))
    return argmax_slots(y, C, dg, df)[:C]


def ensemble_argmax_packed(logits, d_min, d_max, slots, dg=2, df=2):
    """logits[P][K][C] of P inputs packed in one slot vector (input b in the
    block of 2C' slots at 2C'b) -> z[P][C] (plaintext Alg. 1 pipeline on the
    packed vector, every block read back)."""
    logits = np.asarray(logits, dtype=np.float64)
    P, K, C = logits.shape
    cp = 1 << (C - 1).bit_length()
    y = np.zeros(slots)
    for b in range(P):
        for i in range(K):
            p = pad_logits(logits[b, i], C, d_min)
            y[b * 2 * cp: b * 2 * cp + cp] += p
    y = y * (1.0 / (K * (d_max - d_min)))
    z = argmax_slots(y, C, dg, df)
    return np.stack([z[b * 2 * cp: b * 2 * cp + C] for b in range(P)])


def phoenix_argmax_slots(y, n_classes, dg=2, df=2):
    """The Phoenix Argmax on a slot vector: s = sum_{i=1..m} Sign(y -
    RotL(y, i)) after the duplication, z = (Sign((s - (m-1)) / (2m)) + 1)/2."""
    cp = 1 << (n_classes - 1).bit_length()
    m = cp - 1
    y = y + rotl(y, -cp)
    s = np.zeros_like(y)
    for i in range(1, m + 1):
        s = s + sign(y - rotl(y, i), dg, df)
    t = (s - (m - 1.0)) * (1.0 / (2 * m))
    return 0.5 * sign(t, dg, df) + 0.5


def ensemble_phoenix_argmax(logits, d_min, d_max, slots, dg=2, df=2):
    """logits[K][C] -> z over the first C slots (plaintext Phoenix pipeline)."""
    logits = np.asarray(logits, dtype=np.float64)
    K, C = logits.shape
    y = np.zeros(slots)
    for i in range(K):
        p = pad_logits(logits[i], C, d_min)
        y[: len(p)] += p
    y = y * (1.0 / (K * (d_max - d_min)))
    return phoenix_argmax_slots(y, C, dg, df)[:C]

