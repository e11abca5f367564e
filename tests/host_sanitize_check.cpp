// Host-side C++ of the library (S_N tables, batch geometry and the block cyclic
// reduction schedule) run under AddressSanitizer and UndefinedBehaviorSanitizer by
// tests/test_host_sanitizers.py, with the invariants each must satisfy:
//   tables (even N from 2 to 256, three truncations, both Laplacians): ordinates
//     ascending and mirrored, Gauss-Legendre exactness of the weights to degree 2N - 1,
//     D M = I on the kept moments (Eqs. phi-mom, treq), the MPD Laplacian's eigenrelation
//     D F M = diag(-l (l + 1)) (Eq. legendre), the WFD Laplacian's zero row sums,
//     w-symmetry, nonnegative off-diagonals and preserved first moment (Sec. 3.3);
//   geometry (seeded ragged batches): every cell but an instance's first eliminated
//     exactly once, at level ctz(local), between its neighbours local -/+ 2^l of the
//     same instance, and every coupling slot an item names inside the cell's own range.
// Prints "host check ok" and exits 0 when every check holds.
#include "../paper_1907_13013_gb300/csrc/fpsa_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

using fpsa::BcrItem;
using fpsa::Geometry;
using fpsa::Tables;

static int failures = 0;

static void check(bool ok, const char *what, int a, int b, double v) {
    if (!ok && failures++ < 20) std::printf("FAIL %s (%d, %d): %.3e\n", what, a, b, v);
}

static void check_tables(int N, int L1, int lap) {
    Tables t;
    fpsa::build_tables(N, L1, lap, t);
    check((int)t.mu.size() == N && (int)t.w.size() == N && (int)t.D.size() == N * N &&
              (int)t.M.size() == N * N && (int)t.Afp.size() == N * N,
          "table sizes", N, L1, 0.0);
    for (int n = 0; n < N; ++n) {
        check(std::fabs(t.mu[n]) < 1.0 && t.w[n] > 0.0, "ordinate range / positive weight", N, n, t.mu[n]);
        check(t.mu[n] == -t.mu[N - 1 - n] && t.w[n] == t.w[N - 1 - n], "mirrored ordinates", N, n, t.mu[n]);
        if (n > 0) check(t.mu[n] > t.mu[n - 1], "ascending ordinates", N, n, t.mu[n]);
    }
    // exactness: sum_n w_n mu_n^k = 2 / (k + 1) for even k, 0 for odd k, k <= 2N - 1
    for (int k = 0; k <= 2 * N - 1; ++k) {
        double s = 0.0;
        for (int n = 0; n < N; ++n) s += t.w[n] * std::pow(t.mu[n], k);
        const double exact = (k % 2) ? 0.0 : 2.0 / (k + 1);
        check(std::fabs(s - exact) <= 1e-13, "Gauss-Legendre exactness", N, k, s - exact);
    }
    // D M = I on the kept moments; M's columns beyond the truncation are zero
    for (int l = 0; l < N; ++l)
        for (int k = 0; k < N; ++k) {
            double s = 0.0;
            for (int n = 0; n < N; ++n) s += t.D[(size_t)l * N + n] * t.M[(size_t)n * N + k];
            const double want = (k < L1 && l == k) ? 1.0 : 0.0;
            if (k < L1) check(std::fabs(s - want) <= 1e-10, "D M = I", l, k, s - want);
            else check(s == 0.0, "truncated expansion", l, k, s);
        }
    if (lap == FPSA_LAPLACIAN_MPD) {
        // D F M = diag(-l (l + 1)) with the full expansion (M of L1 = N)
        Tables full;
        fpsa::build_tables(N, N, lap, full);
        std::vector<double> FM((size_t)N * N, 0.0);
        for (int a = 0; a < N; ++a)
            for (int k = 0; k < N; ++k) {
                double s = 0.0;
                for (int b = 0; b < N; ++b) s += t.Afp[(size_t)a * N + b] * full.M[(size_t)b * N + k];
                FM[(size_t)a * N + k] = s;
            }
        for (int l = 0; l < N; ++l)
            for (int k = 0; k < N; ++k) {
                double s = 0.0;
                for (int a = 0; a < N; ++a) s += t.D[(size_t)l * N + a] * FM[(size_t)a * N + k];
                const double want = (l == k) ? -(double)l * (l + 1.0) : 0.0;
                check(std::fabs(s - want) <= 1e-8 * (1.0 + (double)N * N), "MPD eigenrelation", l, k, s - want);
            }
    } else {
        for (int n = 0; n < N; ++n) {
            double rs = 0.0, mx = 0.0;
            for (int m = 0; m < N; ++m) mx = std::fmax(mx, std::fabs(t.Afp[(size_t)n * N + m]));
            for (int m = 0; m < N; ++m) {
                const double a = t.Afp[(size_t)n * N + m];
                rs += a;
                if (m != n) check(a >= 0.0, "WFD off-diagonal sign", n, m, a);
                if (std::abs(m - n) > 1) check(a == 0.0, "WFD tridiagonal", n, m, a);
                const double sym = t.w[n] * a - t.w[m] * t.Afp[(size_t)m * N + n];
                check(std::fabs(sym) <= 1e-12 * (1.0 + mx), "WFD w-symmetry", n, m, sym);
            }
            check(std::fabs(rs) <= 1e-12 * (1.0 + mx), "WFD zero row sum", N, n, rs);
        }
        // first moment: sum_n w_n mu_n (A_FP v)_n = -2 sum_n w_n mu_n v_n for every v
        for (int m = 0; m < N; ++m) {
            double s = 0.0, mx = 0.0;
            for (int n = 0; n < N; ++n) {
                s += t.w[n] * t.mu[n] * t.Afp[(size_t)n * N + m];
                mx = std::fmax(mx, std::fabs(t.w[n] * t.Afp[(size_t)n * N + m]));
            }
            const double want = -2.0 * t.w[m] * t.mu[m];
            check(std::fabs(s - want) <= 1e-12 * (1.0 + mx), "WFD first moment", N, m, s - want);
        }
    }
}

static int ctz(int x) {
    int t = 0;
    while (!(x & 1)) {
        x >>= 1;
        ++t;
    }
    return t;
}

static int levels_of(int K) {
    int l = 0;
    while ((1 << l) < K) ++l;
    return l;
}

static void check_geometry(const std::vector<int32_t> &K, int N) {
    Geometry g;
    const int B = (int)K.size();
    fpsa::build_geometry(K.data(), B, N, N, 1, g);
    int sumK = 0, nl = 0;
    for (int b = 0; b < B; ++b) {
        check(g.off[b] == sumK, "instance offset", b, g.off[b], 0.0);
        sumK += K[b];
        nl = std::max(nl, levels_of(K[b]));
    }
    check(g.sumK == sumK && g.n_levels == nl && (int)g.levels.size() == nl, "batch sizes", g.sumK, g.n_levels, 0.0);
    // slot ranges: cell i of an instance owns ctz(i) + 1 slots (the first cell one per level and a spare)
    std::vector<int> seen(sumK, 0), nslots(sumK, 0);
    int expect_base = 0;
    for (int b = 0; b < B; ++b)
        for (int i = 0; i < K[b]; ++i) {
            const int c = g.off[b] + i;
            check(g.cell_inst[c] == b, "cell instance", c, g.cell_inst[c], 0.0);
            check(g.slot_base[c] == expect_base, "slot base", c, g.slot_base[c], 0.0);
            nslots[c] = i == 0 ? levels_of(K[b]) + 1 : ctz(i) + 1;
            expect_base += nslots[c];
        }
    check(g.n_slots == expect_base, "slot count", g.n_slots, expect_base, 0.0);
    auto in_range = [&](int cell, int slot) {
        return cell >= 0 && slot >= g.slot_base[cell] && slot < g.slot_base[cell] + nslots[cell];
    };
    for (int l = 0; l < nl; ++l)
        for (const BcrItem &it : g.levels[l]) {
            const int b = g.cell_inst[it.cell], i = it.cell - g.off[b], st = 1 << l;
            ++seen[it.cell];
            check(it.level == l && i == it.local && it.K_inst == K[b], "item fields", it.cell, l, 0.0);
            check(i > 0 && ctz(i) == l, "eliminated at level ctz(local)", it.cell, l, 0.0);
            check(it.left == it.cell - st && g.cell_inst[it.left] == b, "left neighbour", it.cell, it.left, 0.0);
            if (i + st < K[b]) check(it.right == it.cell + st, "right neighbour", it.cell, it.right, 0.0);
            else check(it.right == -1, "no right neighbour", it.cell, it.right, 0.0);
            check(in_range(it.cell, it.s_cell) && it.s_cell == g.slot_base[it.cell] + l, "cell slot", it.cell, l, 0.0);
            check(in_range(it.left, it.s_left) && in_range(it.left, it.s_left_next) &&
                      it.s_left_next == it.s_left + 1,
                  "left slots", it.cell, l, 0.0);
            if (it.right >= 0)
                check(in_range(it.right, it.s_right) && in_range(it.right, it.s_right_next) &&
                          it.s_right_next == it.s_right + 1,
                      "right slots", it.cell, l, 0.0);
            else check(it.s_right == -1 && it.s_right_next == -1, "absent right slots", it.cell, l, 0.0);
        }
    check((int)g.roots.size() == B, "one root per instance", B, (int)g.roots.size(), 0.0);
    for (int b = 0; b < B; ++b) {
        const BcrItem &r = g.roots[b];
        check(r.cell == g.off[b] && r.local == 0 && r.left == -1 && r.right == -1 && r.level == levels_of(K[b]) &&
                  in_range(r.cell, r.s_cell),
              "root item", b, r.cell, 0.0);
        ++seen[r.cell];
    }
    for (int c = 0; c < sumK; ++c) check(seen[c] == 1, "every cell solved once", c, seen[c], 0.0);
}

int main() {
    std::vector<int> orders;
    for (int N = 2; N <= 32; N += 2) orders.push_back(N);
    for (int N : {40, 64, 98, 128, 130, 192, 254, 256}) orders.push_back(N);
    for (int N : orders) {
        const int l1s[3] = {1, N / 2, N};
        for (int j = 0; j < 3; ++j) {
            check_tables(N, l1s[j], FPSA_LAPLACIAN_WFD);
            if (N <= 64 || j == 2) check_tables(N, l1s[j], FPSA_LAPLACIAN_MPD);
        }
    }
    unsigned long long s = 13013;
    auto next = [&](int lo, int hi) {  // 64-bit LCG (Knuth's MMIX constants), uniform in [lo, hi]
        s = s * 6364136223846793005ULL + 1442695040888963407ULL;
        return lo + (int)((s >> 33) % (unsigned long long)(hi - lo + 1));
    };
    check_geometry({1}, 16);
    check_geometry({2}, 16);
    check_geometry({1, 1, 3, 4, 5, 8, 9}, 32);
    check_geometry({2000}, 64);
    for (int trial = 0; trial < 40; ++trial) {
        std::vector<int32_t> K(next(1, 40));
        for (int32_t &k : K) k = next(1, trial % 4 == 0 ? 5000 : 300);
        check_geometry(K, 2 * next(1, 64));
    }
    if (failures) {
        std::printf("%d failures\n", failures);
        return 1;
    }
    std::printf("host check ok\n");
    return 0;
}
