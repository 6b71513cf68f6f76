// Host-side CKKS canonical-embedding encoder/decoder (Sec. 2: a ciphertext over
// Z_Q[X]/(X^{2N}+1) carries N real slots).  Slot i is the evaluation of the plaintext at
// zeta^{5^i mod 2n}, zeta = exp(i pi / n); a real slot vector z has the real coefficients
// m_j = (2S/n) sum_i z_i cos(pi g_i j / n), computed with one complex FFT of length 2n.
// Encoding is preprocessing: it runs on the host and never touches ciphertext arithmetic.
// Complex slot values (the diagonals of bootstrapping's linear maps) take the real polynomial
// with m(zeta^g_i) = S z_i and m(zeta^-g_i) = S conj(z_i): m_j = (2S/n) sum_i Re(z_i zeta^(-g_i j)).
#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <vector>

#include "internal.h"

namespace {

typedef std::complex<double> cd;

struct FftPlan {
    int n = 0, logn = 0;
    std::vector<cd> w;            // exp(-2 pi i k / n), k < n/2
    std::vector<int> rev;
};

std::mutex g_mu;
std::map<int, FftPlan *> g_plans;

const FftPlan *plan_for(int n) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find(n);
    if (it != g_plans.end()) return it->second;
    FftPlan *p = new FftPlan();
    p->n = n;
    while ((1 << p->logn) < n) p->logn++;
    p->w.resize(n / 2);
    for (int k = 0; k < n / 2; k++) {
        double a = -2.0 * M_PI * (double)k / (double)n;
        p->w[k] = cd(std::cos(a), std::sin(a));
    }
    p->rev.resize(n);
    for (int i = 0; i < n; i++) {
        int r = 0;
        for (int b = 0; b < p->logn; b++)
            if (i >> b & 1) r |= 1 << (p->logn - 1 - b);
        p->rev[i] = r;
    }
    g_plans[n] = p;
    return p;
}

// in-place forward DFT: X[k] = sum_j x[j] exp(-2 pi i j k / n)
void fft(std::vector<cd> &x) {
    const FftPlan *p = plan_for((int)x.size());
    const int n = p->n;
    for (int i = 0; i < n; i++)
        if (i < p->rev[i]) std::swap(x[i], x[p->rev[i]]);
    for (int len = 2; len <= n; len <<= 1) {
        const int step = n / len;
        for (int i = 0; i < n; i += len)
            for (int j = 0; j < len / 2; j++) {
                cd u = x[i + j], v = x[i + j + len / 2] * p->w[j * step];
                x[i + j] = u + v;
                x[i + j + len / 2] = u - v;
            }
    }
}

std::vector<int> slot_exponents(int n) {
    std::vector<int> g(n / 2);
    long long v = 1;
    for (int i = 0; i < n / 2; i++) {
        g[i] = (int)v;
        v = v * 5 % (2 * n);
    }
    return g;
}

}  // namespace

void encode_slots(const double *z, int n, double S, int64_t *m_out) {
    std::vector<int> g = slot_exponents(n);
    std::vector<cd> A(2 * (size_t)n, cd(0, 0));
    for (int i = 0; i < n / 2; i++) {
        A[g[i]] = cd(z[i], 0);
        A[2 * n - g[i]] = cd(z[i], 0);
    }
    fft(A);
    for (int j = 0; j < n; j++) {
        double v = S / n * A[j].real();
        double r = v >= 0 ? std::floor(v + 0.5) : std::ceil(v - 0.5);   // half away from zero
        m_out[j] = (int64_t)r;
    }
}

void encode_slots_complex(const double *re, const double *im, int n, double S, int64_t *m_out) {
    std::vector<int> g = slot_exponents(n);
    std::vector<cd> A(2 * (size_t)n, cd(0, 0));
    for (int i = 0; i < n / 2; i++) {
        A[g[i]] = cd(re[i], im[i]);
        A[2 * n - g[i]] = cd(re[i], -im[i]);
    }
    fft(A);
    for (int j = 0; j < n; j++) {
        double v = S / n * A[j].real();
        double r = v >= 0 ? std::floor(v + 0.5) : std::ceil(v - 0.5);
        m_out[j] = (int64_t)r;
    }
}

void decode_coeffs(const double *m, int n, double S, double *z_out) {
    std::vector<int> g = slot_exponents(n);
    std::vector<cd> a(2 * (size_t)n, cd(0, 0));
    for (int j = 0; j < n; j++) a[j] = cd(m[j], 0);
    fft(a);
    for (int i = 0; i < n / 2; i++) z_out[i] = a[g[i]].real() / S;
}
