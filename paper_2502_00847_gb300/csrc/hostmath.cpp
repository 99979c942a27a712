// Host-side number theory for the SecPE GB300 library: primes, roots of
// unity, Shoup/Montgomery constants, the counter-based sampler keys and the
// rounding rule for encoded constants.
#include <cmath>
#include <set>

#include "internal.h"

namespace hm {

u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }

u64 powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

u64 invmod(u64 a, u64 q) { return powmod(a % q, q - 2, q); }

u64 shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

u64 neg_inv64(u64 q) {
    // Newton iteration for q^-1 mod 2^64 (q odd): x <- x (2 - q x)
    u64 x = q;  // correct to 3 bits
    for (int i = 0; i < 6; i++) x *= 2 - q * x;
    return (u64)0 - x;
}

bool is_prime(u64 n) {
    if (n < 2) return false;
    static const u64 bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 p : bases) {
        if (n % p == 0) return n == p;
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        s++;
    }
    for (u64 a : bases) {
        u64 x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; r++) {
            x = mulmod(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

static void below(u64 bound, u64 m, int count, const std::set<u64> &taken, std::vector<u64> &out) {
    u64 k = (bound - 2) / m;
    while ((int)out.size() < count && k > 0) {
        u64 c = k * m + 1;
        if (c < bound && !taken.count(c) && is_prime(c)) out.push_back(c);
        k--;
    }
}

static void above(u64 bound, u64 m, int count, const std::set<u64> &taken, std::vector<u64> &out) {
    u64 k = bound / m + 1;
    while ((int)out.size() < count) {
        u64 c = k * m + 1;
        if (c > bound && !taken.count(c) && is_prime(c)) out.push_back(c);
        k++;
    }
}

bool select_primes(const secpe_params &p, std::vector<u64> &q, std::vector<u64> &special) {
    if (p.log_n < 4 || p.log_n > 17) return false;
    if (p.n_q < 2 || p.n_q > 48 || p.n_p < 1 || p.n_p > 8) return false;
    if (p.p_bits < 20 || p.p_bits > 60 || p.q0_bits < 20 || p.q0_bits > 60) return false;
    if (p.q_bits < 20 || p.q_bits > 59) return false;
    const u64 m = 2ull << p.log_n;
    q.clear();
    special.clear();
    std::set<u64> taken;
    below(1ull << p.p_bits, m, p.n_p, taken, special);
    if ((int)special.size() != p.n_p) return false;
    for (u64 x : special) taken.insert(x);
    if (p.boot_primes < 0 || p.boot_primes > p.n_q - 2 || (p.boot_primes && (p.boot_bits < 20 || p.boot_bits > 60)))
        return false;
    std::vector<u64> boot;
    if (p.boot_primes > 0) {
        below(1ull << p.boot_bits, m, p.boot_primes, taken, boot);
        if ((int)boot.size() != p.boot_primes) return false;
        for (u64 x : boot) taken.insert(x);
    }
    if (p.q0_bits != p.q_bits) {
        std::vector<u64> q0;
        below(1ull << p.q0_bits, m, 1, taken, q0);
        if (q0.size() != 1) return false;
        q.push_back(q0[0]);
        taken.insert(q0[0]);
    }
    const int n_comp = p.n_q - p.boot_primes;
    int need = n_comp - (int)q.size();
    std::vector<u64> lo, hi;
    below(1ull << p.q_bits, m, need, taken, lo);
    above(1ull << p.q_bits, m, need, taken, hi);
    if ((int)lo.size() < need) return false;
    for (int i = 0; (int)q.size() < n_comp; i++) {
        q.push_back(lo[i]);
        if ((int)q.size() < n_comp) q.push_back(hi[i]);
    }
    for (u64 x : boot) q.push_back(x);
    for (u64 x : q)
        if (x >= (1ull << 60)) return false;
    return true;
}

u64 find_psi(u64 q, u64 n) {
    u64 e = (q - 1) / (2 * n);
    for (u64 x = 2;; x++) {
        u64 psi = powmod(x, e, q);
        if (powmod(psi, n, q) == q - 1) return psi;
    }
}

uint32_t bitrev(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; i++) {
        r = (r << 1) | (x & 1);
        x >>= 1;
    }
    return r;
}

static const u64 kGamma = 0x9E3779B97F4A7C15ull;

u64 sm_mix(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

u64 sm_stream(u64 seed, u64 domain, u64 index) {
    return sm_mix(sm_mix(seed + domain * kGamma) + index * kGamma);
}

long long round_half_away(double v) { return std::llround(v); }

void sample_sparse_secret(u64 key, int n, int h, std::vector<long long> &s) {
    s.assign(n, 0);
    int placed = 0;
    for (u64 c = 0; placed < h; c++) {
        const u64 w = sm_mix(key + (c + 1) * kGamma);
        const u64 pos = (w >> 1) & (u64)(n - 1);
        if (s[pos] != 0) continue;
        s[pos] = (w & 1) ? -1 : 1;
        placed++;
    }
}

}  // namespace hm
