// Host-side polynomial approximation of activation functions in the Chebyshev basis (Appendix
// "Polynomial Approximation"): interpolation at the Chebyshev nodes (Appendix "Chebyshev
// Basis") and the minimax (best uniform) polynomial by the Remez exchange algorithm.  The coefficients feed he_poly_eval / he_poly_eval_ps, which evaluate
// sum c_k T_k(t) on t in [-1, 1].
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace {

double activation(int fn, double x) {
    switch (fn) {
        case HE_FN_GELU: return 0.5 * x * (1.0 + erf(x / sqrt(2.0)));
        case HE_FN_RELU: return x > 0.0 ? x : 0.0;
        case HE_FN_SILU: return x / (1.0 + exp(-x));
        case HE_FN_SOFTPLUS: return (x > 0.0 ? x : 0.0) + log1p(exp(-fabs(x)));
        default: return NAN;
    }
}

// sum_{k<=deg} c_k T_k(t) by Clenshaw's recurrence
double clenshaw(const double *c, int deg, double t) {
    double b1 = 0.0, b2 = 0.0;
    for (int k = deg; k >= 1; k--) {
        const double b0 = 2.0 * t * b1 - b2 + c[k];
        b2 = b1;
        b1 = b0;
    }
    return t * b1 - b2 + c[0];
}

// Gaussian elimination with partial pivoting on an m x m system (row-major A, rhs b -> x)
bool solve(std::vector<double> A, std::vector<double> b, int m, std::vector<double> &x) {
    for (int col = 0; col < m; col++) {
        int piv = col;
        for (int r = col + 1; r < m; r++)
            if (fabs(A[(size_t)r * m + col]) > fabs(A[(size_t)piv * m + col])) piv = r;
        if (A[(size_t)piv * m + col] == 0.0) return false;
        if (piv != col) {
            for (int k = 0; k < m; k++) std::swap(A[(size_t)piv * m + k], A[(size_t)col * m + k]);
            std::swap(b[piv], b[col]);
        }
        for (int r = col + 1; r < m; r++) {
            const double f = A[(size_t)r * m + col] / A[(size_t)col * m + col];
            if (f == 0.0) continue;
            for (int k = col; k < m; k++) A[(size_t)r * m + k] -= f * A[(size_t)col * m + k];
            b[r] -= f * b[col];
        }
    }
    x.assign(m, 0.0);
    for (int r = m - 1; r >= 0; r--) {
        double s = b[r];
        for (int k = r + 1; k < m; k++) s -= A[(size_t)r * m + k] * x[k];
        x[r] = s / A[(size_t)r * m + r];
    }
    return true;
}

}  // namespace

extern "C" int he_cheb_interp(int fn, int deg, double lo, double hi, double *coeffs) {
    if (deg < 0 || deg > 1000 || !(hi > lo) || !coeffs || std::isnan(activation(fn, 0.5 * (lo + hi)))) {
        he_set_error("he_cheb_interp: bad argument");
        return HE_EINVAL;
    }
    // p interpolates f at the deg + 1 first-kind nodes t_j = cos(theta_j), theta_j =
    // pi (j + 1/2) / (deg + 1); discrete orthogonality of T_k over these nodes gives
    // c_k = (2 / (deg + 1)) sum_j f(t_j) cos(k theta_j), halved for k = 0
    const int K = deg + 1;
    const double half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
    std::vector<double> theta(K), fv(K);
    for (int j = 0; j < K; j++) {
        theta[j] = M_PI * (j + 0.5) / K;
        fv[j] = activation(fn, half * cos(theta[j]) + mid);
    }
    for (int k = 0; k < K; k++) {
        double sum = 0.0;
        for (int j = 0; j < K; j++) sum += fv[j] * cos(k * theta[j]);
        coeffs[k] = (2.0 / K) * sum;
    }
    coeffs[0] *= 0.5;
    return HE_OK;
}

extern "C" int he_cheb_minimax(int fn, int deg, double lo, double hi, double *coeffs, double *err) {
    if (deg < 0 || deg > 200 || !(hi > lo) || !coeffs || std::isnan(activation(fn, 0.5 * (lo + hi)))) {
        he_set_error("he_cheb_minimax: bad argument");
        return HE_EINVAL;
    }
    const int n = deg + 2;                                // reference points
    const double half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
    auto f = [&](double t) { return activation(fn, half * t + mid); };
    // scan grid: Chebyshev-spaced (dense near the ends, where the extrema crowd) plus t = 0
    const int G = 400 * n;
    std::vector<double> tg;
    tg.reserve(G + 2);
    for (int i = 0; i <= G; i++) tg.push_back(-cos(M_PI * i / G));
    tg.push_back(0.0);
    std::sort(tg.begin(), tg.end());
    tg.erase(std::unique(tg.begin(), tg.end()), tg.end());
    std::vector<double> fg(tg.size());
    for (size_t i = 0; i < tg.size(); i++) fg[i] = f(tg[i]);
    std::vector<double> ref(n), c(deg + 1, 0.0), sol;
    for (int i = 0; i < n; i++) ref[i] = -cos(M_PI * i / (n - 1));
    double E = 0.0;
    const double gr = (sqrt(5.0) - 1.0) / 2.0;
    for (int it = 0; it < 100; it++) {
        // p(ref_i) + (-1)^i E = f(ref_i)
        std::vector<double> A((size_t)n * n), rhs(n);
        for (int i = 0; i < n; i++) {
            double T0 = 1.0, T1 = ref[i];
            A[(size_t)i * n + 0] = 1.0;
            if (deg >= 1) A[(size_t)i * n + 1] = T1;
            for (int k = 2; k <= deg; k++) {
                const double T2 = 2.0 * ref[i] * T1 - T0;
                A[(size_t)i * n + k] = T2;
                T0 = T1;
                T1 = T2;
            }
            A[(size_t)i * n + deg + 1] = (i % 2) ? -1.0 : 1.0;
            rhs[i] = f(ref[i]);
        }
        if (!solve(A, rhs, n, sol)) { he_set_error("he_cheb_minimax: singular reference"); return HE_ESTATE; }
        std::copy(sol.begin(), sol.begin() + deg + 1, c.begin());
        E = sol[deg + 1];
        auto e = [&](double t) { return f(t) - clenshaw(c.data(), deg, t); };
        // the largest |error| of each run of one sign, refined by golden section
        std::vector<double> pts, vals;
        size_t i = 0;
        while (i < tg.size()) {
            const double r0 = fg[i] - clenshaw(c.data(), deg, tg[i]);
            const bool pos = r0 >= 0.0;
            size_t best = i;
            double bestv = fabs(r0);
            size_t j = i + 1;
            for (; j < tg.size(); j++) {
                const double r = fg[j] - clenshaw(c.data(), deg, tg[j]);
                if ((r >= 0.0) != pos) break;
                if (fabs(r) > bestv) { bestv = fabs(r); best = j; }
            }
            const double sg = pos ? 1.0 : -1.0;
            double a = tg[best > 0 ? best - 1 : 0], b = tg[std::min(best + 1, tg.size() - 1)];
            double x1 = b - gr * (b - a), x2 = a + gr * (b - a);
            double f1 = sg * e(x1), f2 = sg * e(x2);
            for (int g = 0; g < 60; g++) {
                if (f1 > f2) { b = x2; x2 = x1; f2 = f1; x1 = b - gr * (b - a); f1 = sg * e(x1); }
                else { a = x1; x1 = x2; f1 = f2; x2 = a + gr * (b - a); f2 = sg * e(x2); }
            }
            double bx = tg[best], bv = bestv;
            if (f1 > bv) { bx = x1; bv = f1; }
            if (f2 > bv) { bx = x2; bv = f2; }
            pts.push_back(bx);
            vals.push_back(sg * bv);
            i = j;
        }
        while ((int)pts.size() > n) {                     // keep n alternating extrema
            if ((int)pts.size() == n + 1) {
                const size_t d = fabs(vals.front()) < fabs(vals.back()) ? 0 : pts.size() - 1;
                pts.erase(pts.begin() + d);
                vals.erase(vals.begin() + d);
                continue;
            }
            size_t k = 0;
            for (size_t q = 1; q < vals.size(); q++)
                if (fabs(vals[q]) < fabs(vals[k])) k = q;
            if (k == 0 || k + 1 == vals.size()) {
                pts.erase(pts.begin() + k);
                vals.erase(vals.begin() + k);
            } else {
                const size_t kk = fabs(vals[k - 1]) < fabs(vals[k + 1]) ? k - 1 : k + 1;
                const size_t hi_i = std::max(k, kk), lo_i = std::min(k, kk);
                pts.erase(pts.begin() + hi_i);
                vals.erase(vals.begin() + hi_i);
                pts.erase(pts.begin() + lo_i);
                vals.erase(vals.begin() + lo_i);
            }
        }
        if ((int)pts.size() < n) { he_set_error("he_cheb_minimax: fewer than deg + 2 alternation points"); return HE_ESTATE; }
        double emax = 0.0;
        for (double v : vals) emax = std::max(emax, fabs(v));
        ref = pts;
        if (emax - fabs(E) <= 1e-10 * emax) break;
    }
    memcpy(coeffs, c.data(), (size_t)(deg + 1) * sizeof(double));
    if (err) *err = fabs(E);
    return HE_OK;
}
