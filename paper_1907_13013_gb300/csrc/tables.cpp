// Host-side S_N tables of the library (arXiv:1907.13013, Sec. 2.2).
//
// Gauss-Legendre nodes by Newton's method on P_N from the asymptotic
// initial guess cos(pi (i - 1/4) / (N + 1/2)), weights 2 / ((1 - x^2) P_N'(x)^2);
// Legendre values by the three-term recurrence; the moment operator
// D[l][n] = w_n P_l(mu_n) (Eq. phi-mom), the expansion operator
// M[n][l] = (2l+1)/2 P_l(mu_n) (Eq. treq), the MPD Laplacian F = M Lambda D
// (Eq. fp-mpd: V = D, and V^{-1} = M because Gauss-Legendre integrates the
// degree <= 2N-2 products P_l P_k exactly), and the WFD Laplacian
// (Eqs. fp-wdd, sph-weights, w_wfd with gamma_{n+1/2} = gamma_{n-1/2} - 2 mu_n w_n).
#include "fpsa_internal.h"

#include <cmath>

namespace fpsa {

static void legendre_and_derivative(int N, double x, double *pn, double *dpn) {
    double p0 = 1.0, p1 = x;
    for (int l = 1; l < N; ++l) {
        double p2 = ((2.0 * l + 1.0) * x * p1 - l * p0) / (l + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;                                          // P_N
    *dpn = N * (p0 - x * p1) / ((1.0 - x) * (1.0 + x));  // P_N' from P_N, P_{N-1}
}

void build_tables(int N, int L1, int laplacian, Tables &t) {
    t.N = N;
    t.L1 = L1;
    t.mu.assign(N, 0.0);
    t.w.assign(N, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < N / 2; ++i) {
        double x = std::cos(pi * (i + 0.75) / (N + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre_and_derivative(N, x, &p, &dp);
            double dx = p / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-17) break;
        }
        double p, dp;
        legendre_and_derivative(N, x, &p, &dp);
        // 1 - x^2 as (1 - x)(1 + x): no cancellation next to x = 1
        double wi = 2.0 / ((1.0 - x) * (1.0 + x) * dp * dp);
        // x > 0 is the (i+1)-th largest root; store ascending and mirrored
        t.mu[N - 1 - i] = x;
        t.mu[i] = -x;
        t.w[N - 1 - i] = wi;
        t.w[i] = wi;
    }
    // P[l][n], l < N
    std::vector<double> P((size_t)N * N);
    for (int n = 0; n < N; ++n) {
        double x = t.mu[n];
        P[n] = 1.0;
        if (N > 1) P[N + n] = x;
        for (int l = 1; l + 1 < N; ++l)
            P[(size_t)(l + 1) * N + n] = ((2.0 * l + 1.0) * x * P[(size_t)l * N + n] - l * P[(size_t)(l - 1) * N + n]) / (l + 1.0);
    }
    // D and M padded to N moments; rows / columns l >= L1 are kept for D (moments of
    // every order are computed) but M's columns l >= L1 are zero (truncated expansion).
    t.D.assign((size_t)N * N, 0.0);
    t.M.assign((size_t)N * N, 0.0);
    for (int l = 0; l < N; ++l)
        for (int n = 0; n < N; ++n) {
            t.D[(size_t)l * N + n] = t.w[n] * P[(size_t)l * N + n];
            t.M[(size_t)n * N + l] = (l < L1) ? 0.5 * (2.0 * l + 1.0) * P[(size_t)l * N + n] : 0.0;
        }
    // angular Laplacian A_FP (N x N)
    t.Afp.assign((size_t)N * N, 0.0);
    if (laplacian == FPSA_LAPLACIAN_MPD) {
        for (int a = 0; a < N; ++a)
            for (int b = 0; b < N; ++b) {
                double s = 0.0;
                for (int l = 0; l < N; ++l) {
                    double m_al = 0.5 * (2.0 * l + 1.0) * P[(size_t)l * N + a];
                    s += m_al * (-(double)l * (l + 1.0)) * t.D[(size_t)l * N + b];
                }
                t.Afp[(size_t)a * N + b] = s;
            }
    } else {
        std::vector<double> g(N + 1, 0.0);
        for (int n = 0; n < N; ++n) g[n + 1] = g[n] - 2.0 * t.mu[n] * t.w[n];
        g[N] = 0.0;  // exact value; the recurrence leaves rounding there
        for (int n = 0; n < N; ++n) {
            double lo = (n > 0) ? g[n] / (t.mu[n] - t.mu[n - 1]) / t.w[n] : 0.0;
            double hi = (n < N - 1) ? g[n + 1] / (t.mu[n + 1] - t.mu[n]) / t.w[n] : 0.0;
            if (n > 0) t.Afp[(size_t)n * N + n - 1] = lo;
            if (n < N - 1) t.Afp[(size_t)n * N + n + 1] = hi;
            t.Afp[(size_t)n * N + n] = -(lo + hi);
        }
    }
}

}  // namespace fpsa
