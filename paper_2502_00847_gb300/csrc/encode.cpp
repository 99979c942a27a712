// Host-side CKKS encoding of real vectors (canonical embedding, SecPE
// Sec. 2.2 SIMD packing).  Slot j corresponds to the root zeta^(5^j),
// zeta = exp(i pi / N); for a real vector v in slots 0..n-1 (zeros beyond)
// the real coefficient vector is
//   m_k = round(scale * (2/N) * sum_j v_j cos(pi (5^j k mod 2N) / N)),
// and decoding takes the real part of m(zeta^(5^j)) / scale.
#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>

namespace enc {

static std::vector<double> cos_table(int n) {
    std::vector<double> t(2 * (size_t)n);
    const double pi = 3.14159265358979323846;
    for (int e = 0; e < 2 * n; e++) t[e] = std::cos(pi * (double)e / (double)n);
    return t;
}

static std::vector<uint32_t> pow5(int count, int n) {
    std::vector<uint32_t> p(count);
    uint64_t e = 1;
    for (int j = 0; j < count; j++) {
        p[j] = (uint32_t)e;
        e = e * 5 % (2ull * n);
    }
    return p;
}

bool encode_real(int n, const double *v, int nv, double scale, std::vector<long long> &m) {
    if (nv < 0 || nv > n / 2) return false;
    const std::vector<double> ct = cos_table(n);
    const std::vector<uint32_t> p5 = pow5(nv, n);
    const uint64_t mask = 2ull * n - 1;
    m.assign(n, 0);
    for (int k = 0; k < n; k++) {
        double acc = 0.0;
        for (int j = 0; j < nv; j++) acc += v[j] * ct[((uint64_t)p5[j] * k) & mask];
        const double x = acc * (2.0 / n) * scale;
        if (!(std::fabs(x) < 4.0e18)) return false;
        m[k] = std::llround(x);
    }
    return true;
}

void decode_real(int n, const double *coeffs, double scale, int nslots, double *out) {
    const std::vector<double> ct = cos_table(n);
    const std::vector<uint32_t> p5 = pow5(nslots, n);
    const uint64_t mask = 2ull * n - 1;
    for (int j = 0; j < nslots; j++) {
        double acc = 0.0;
        for (int k = 0; k < n; k++) acc += coeffs[k] * ct[((uint64_t)p5[j] * k) & mask];
        out[j] = acc / scale;
    }
}

// ---------------------------------------------------------------------------
// The same embedding in O(N log N), for full slot vectors (slot packing).
// Writing the odd powers of zeta as zeta^(2t+1), t = 0..N-1, and
// omega = zeta^2 (an N-th root of unity):
//   encode: with u_t = v_j at 2t+1 = 5^j and at 2t+1 = -5^j (mod 2N) (the
//           conjugate slot of a real vector), zero elsewhere,
//           m_k = (1/N) Re(zeta^-k sum_t u_t omega^-tk)   (a length-N DFT),
//   decode: v_j = Re(sum_k m_k zeta^k omega^tk) / scale at 2t+1 = 5^j,
// which are the sums above regrouped; the results agree with them up to
// floating-point rounding.
using cplx = std::complex<double>;

bool encode_complex_fft(int n, const double *re, const double *im, int nv, double scale, std::vector<long long> &m);

// In-place iterative radix-2 DFT of length n = 2^k: a_k <- sum_t a_t
// e^(sign 2 pi i t k / n) (unscaled).
static void fft(std::vector<cplx> &a, int sign) {
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; i++) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    const double pi = 3.14159265358979323846;
    std::vector<cplx> w(n / 2);
    for (size_t k = 0; k < n / 2; k++) w[k] = cplx(std::cos(2 * pi * k / n), sign * std::sin(2 * pi * k / n));
    for (size_t len = 2; len <= n; len <<= 1) {
        const size_t step = n / len;
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; k++) {
                const cplx x = a[i + k], y = a[i + k + len / 2] * w[k * step];
                a[i + k] = x + y;
                a[i + k + len / 2] = x - y;
            }
    }
}

bool encode_real_fft(int n, const double *v, int nv, double scale, std::vector<long long> &m) {
    return encode_complex_fft(n, v, nullptr, nv, scale, m);
}

// Complex slots z_j = re_j + i im_j (im may be null): u_t = z_j at
// 2t+1 = 5^j and conj(z_j) at 2t+1 = -5^j, which keeps m real.
bool encode_complex_fft(int n, const double *re, const double *im, int nv, double scale, std::vector<long long> &m) {
    if (nv < 0 || nv > n / 2 || (n & (n - 1))) return false;
    const uint64_t two_n = 2ull * n;
    std::vector<cplx> u(n, cplx(0.0, 0.0));
    uint64_t e = 1;
    for (int j = 0; j < nv; j++) {
        const double b = im ? im[j] : 0.0;
        u[(e - 1) / 2] = cplx(re[j], b);
        u[(two_n - e - 1) / 2] = cplx(re[j], -b);
        e = e * 5 % two_n;
    }
    fft(u, -1);
    const double pi = 3.14159265358979323846;
    m.assign(n, 0);
    for (int k = 0; k < n; k++) {
        const double re = u[k].real() * std::cos(pi * k / n) + u[k].imag() * std::sin(pi * k / n);
        const double x = re / n * scale;
        if (!(std::fabs(x) < 4.0e18)) return false;
        m[k] = std::llround(x);
    }
    return true;
}

void decode_real_fft(int n, const double *coeffs, double scale, int nslots, double *out) {
    const double pi = 3.14159265358979323846;
    std::vector<cplx> a(n);
    for (int k = 0; k < n; k++) a[k] = coeffs[k] * cplx(std::cos(pi * k / n), std::sin(pi * k / n));
    fft(a, +1);
    const uint64_t two_n = 2ull * n;
    uint64_t e = 1;
    for (int j = 0; j < nslots; j++) {
        out[j] = a[(e - 1) / 2].real() / scale;
        e = e * 5 % two_n;
    }
}

}  // namespace enc
