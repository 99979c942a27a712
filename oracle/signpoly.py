"""The degree-9 polynomials f and g of SecPE's composite Sign (Eq. comp).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.

SecPE (Sec. 3.2) approximates Sign by f^df(g^dg(x)) with degree-9 f and g,
alpha = 12, df = dg = 2, but prints no coefficients.  READING: f and g are the
n = 4 members of the families of Cheon, Kim, Kim, Lee, Lee, "Efficient
homomorphic comparison methods with optimal complexity" (Asiacrypt 2020):

  f_n(x) = sum_{i=0}^{n} 4^-i * binom(2i, i) * x * (1 - x^2)^i   (closed form),
  g_4(x) = (5850 x - 34974 x^3 + 97015 x^5 - 113492 x^7 + 46623 x^9) / 2^10,

the latter taken from that paper's table; tests/test_oracle_sign.py checks
the properties that pin it (odd, g_4(1) = 1022/1024, g_4'(0) = 5850/1024,
sup on [0, 1] < 1, and the composite error table).
"""
from fractions import Fraction
from math import comb


def f_closed_form_coeffs(n=4):
    """Coefficients [a_0..a_{2n+1}] of f_n by expanding the closed form."""
    coeffs = [Fraction(0)] * (2 * n + 2)
    for i in range(n + 1):
        w = Fraction(comb(2 * i, i), 4 ** i)
        # x * (1 - x^2)^i = sum_k binom(i, k) (-1)^k x^(2k+1)
        for k in range(i + 1):
            coeffs[2 * k + 1] += w * comb(i, k) * (-1) ** k
    return coeffs


F4_NUM = (315, -420, 378, -180, 35)          # / 2^7, odd powers 1..9
F4_DEN = 2 ** 7
G4_NUM = (5850, -34974, 97015, -113492, 46623)  # / 2^10, odd powers 1..9
G4_DEN = 2 ** 10


def f4_exact():
    return [Fraction(c, F4_DEN) for c in F4_NUM]


def g4_exact():
    return [Fraction(c, G4_DEN) for c in G4_NUM]


def sign_coeffs_float():
    """(g, f) odd-power coefficients [c1, c3, c5, c7, c9] as doubles (exact:
    every one is an integer over a power of two)."""
    g = [float(c) for c in g4_exact()]
    f = [float(c) for c in f4_exact()]
    return g, f


def eval_odd(c, x):
    """c1 x + c3 x^3 + ... + c9 x^9 (works for floats, Fractions, arrays)."""
    x2 = x * x
    acc = c[4]
    for k in (3, 2, 1, 0):
        acc = acc * x2 + c[k]
    return acc * x


def composite(x, dg=2, df=2):
    g, f = sign_coeffs_float()
    for _ in range(dg):
        x = eval_odd(g, x)
    for _ in range(df):
        x = eval_odd(f, x)
    return x
