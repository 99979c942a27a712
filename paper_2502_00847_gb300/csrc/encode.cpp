// Host-side CKKS encoding of real vectors (canonical embedding, SecPE
// Sec. 2.2 SIMD packing).  Slot j corresponds to the root zeta^(5^j),
// zeta = exp(i pi / N); for a real vector v in slots 0..n-1 (zeros beyond)
// the real coefficient vector is
//   m_k = round(scale * (2/N) * sum_j v_j cos(pi (5^j k mod 2N) / N)),
// and decoding takes the real part of m(zeta^(5^j)) / scale.
#include <cmath>
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

}  // namespace enc
