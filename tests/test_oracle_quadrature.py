"""Pins of the oracle's angular tables (P1, P2) against closed forms and the paper's identities."""
import numpy as np
import pytest

from oracle import quadrature as qd


@pytest.mark.parametrize("N", [2, 4, 16, 64, 256])
def test_gauss_legendre_exact_to_degree_2N_minus_1(N):
    # Sec. 2.2: S_N Gauss-Legendre integrates polynomials of degree <= 2N-1 exactly.
    mu, w = qd.gauss_legendre(N)
    assert np.all(np.diff(mu) > 0) and abs(w.sum() - 2.0) < 1e-13
    for k in range(0, 2 * N, max(1, N // 8)):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * mu ** k) - exact) < 1e-13 * max(1, N / 16)
    # one degree higher is not exact (rules out an accidentally larger rule)
    assert abs(np.sum(w * mu ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-8 * 2.0 ** (-N) or N > 32


def test_legendre_closed_forms_and_orthogonality():
    x = np.linspace(-1, 1, 7)
    P = qd.legendre_table(x, 4)
    assert np.allclose(P[2], (3 * x ** 2 - 1) / 2, atol=1e-15)
    assert np.allclose(P[3], (5 * x ** 3 - 3 * x) / 2, atol=1e-15)
    assert np.allclose(P[4], (35 * x ** 4 - 30 * x ** 2 + 3) / 8, atol=1e-15)
    mu, w = qd.gauss_legendre(16)
    P = qd.legendre_table(mu, 15)
    G = (P * w) @ P.T
    assert np.allclose(G, np.diag(2.0 / (2 * np.arange(16) + 1)), atol=1e-13)


@pytest.mark.parametrize("N", [4, 16, 64, 128])
def test_D_times_M_is_identity(N):
    # Gauss-Legendre exactness makes the expansion operator M the inverse of D (L = N-1),
    # i.e. V^{-1} = M for the MPD matrix V of Eq. fp-mpd.
    mu, w = qd.gauss_legendre(N)
    D = qd.moment_operator(mu, w, N - 1)
    M = qd.expansion_operator(mu, N - 1)
    # rounding of N-term sums with weights up to (2N-1)/2 grows roughly like N
    assert np.abs(D @ M - np.eye(N)).max() < 2e-14 * N
    assert np.abs(M @ D - np.eye(N)).max() < 2e-13 * N


@pytest.mark.parametrize("N", [4, 16, 32])
def test_mpd_legendre_eigenrelation(N):
    # Eq. legendre: L_FP P_l = -l(l+1) P_l; MPD (Eq. fp-mpd) preserves it for l <= N-1.
    mu, w = qd.gauss_legendre(N)
    F = qd.mpd_laplacian(mu, w)
    P = qd.legendre_table(mu, N - 1)
    for l in range(N):
        lhs = F @ P[l]
        assert np.abs(lhs + l * (l + 1) * P[l]).max() < 1e-10 * max(1, l * l)


@pytest.mark.parametrize("N", [4, 16, 64])
def test_wfd_structure(N):
    # Sec. 2.2: WFD gives a diagonally dominant M-matrix; gamma from Eq. sph-weights.
    mu, w = qd.gauss_legendre(N)
    g = qd.wfd_gamma(mu, w)
    assert g[0] == 0.0 and abs(g[-1]) < 1e-14 and np.all(g[1:-1] > 0)
    W = qd.wfd_laplacian(mu, w)
    assert np.abs(W.sum(axis=1)).max() < 1e-12                       # W 1 = 0
    off = W - np.diag(np.diag(W))
    assert np.all(off >= 0) and np.all(np.diag(W) < 0)
    assert np.count_nonzero(np.triu(W, 2)) == 0 and np.count_nonzero(np.tril(W, -2)) == 0
    S = np.diag(w) @ W
    assert np.abs(S - S.T).max() < 1e-12                              # self-adjoint in the w inner product


@pytest.mark.parametrize("N", [8, 16, 64])
def test_wfd_preserves_only_moments_0_and_1(N):
    # Sec. 3.3: WFD preserves the zeroth and first Legendre moments, not higher ones.
    mu, w = qd.gauss_legendre(N)
    W = qd.wfd_laplacian(mu, w)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(N)
    P = qd.legendre_table(mu, 2)
    for l in (0, 1):
        lhs = np.sum(w * P[l] * (W @ x))
        rhs = -l * (l + 1) * np.sum(w * P[l] * x)
        assert abs(lhs - rhs) < 1e-11 * np.abs(x).max() * N
    lhs2 = np.sum(w * P[2] * (W @ x))
    assert abs(lhs2 + 6 * np.sum(w * P[2] * x)) > 1e-6


def test_wfd_consistent_with_continuous_operator():
    # The three-point scheme approximates d/dmu (1-mu^2) d/dmu: applied to P_2 it
    # tends to -6 P_2 at interior ordinates as N grows (first-order in the spacing).
    errs = []
    for N in (32, 64, 128):
        mu, w = qd.gauss_legendre(N)
        W = qd.wfd_laplacian(mu, w)
        P2 = (3 * mu ** 2 - 1) / 2
        inner = np.abs(mu) < 0.8
        errs.append(np.abs((W @ P2 + 6 * P2)[inner]).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.05


@pytest.mark.parametrize("N", [2, 16, 64, 256])
def test_gauss_legendre_against_50_digit_roots(N):
    # P1: the S_N rule of Sec. 2.2 is the N-point Gauss-Legendre rule: nodes are the
    # roots of P_N, weights 2 / ((1 - x^2) P_N'(x)^2). Solved here independently by
    # Newton's method in 50-digit arithmetic (mpmath), from the cosine initial guess.
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50

    def p_and_dp(x):
        p0, p1 = mp.mpf(1), x
        for k in range(2, N + 1):
            p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
        return p1, N * (x * p1 - p0) / (x * x - 1)

    mu, w = qd.gauss_legendre(N)
    for i in range(N // 2):
        x = mp.cos(mp.pi * (i + mp.mpf(3) / 4) / (N + mp.mpf(1) / 2))  # (i+1)-th largest root
        for _ in range(60):
            p, dp = p_and_dp(x)
            dx = p / dp
            x -= dx
            if abs(dx) < mp.mpf(10) ** -45:
                break
        p, dp = p_and_dp(x)
        wx = 2 / ((1 - x * x) * dp * dp)
        j = N - 1 - i
        # nodes: the nearest doubles, to within an ulp
        dx = mp.mpf(mu[j]) - x
        assert abs(dx) <= 1.2e-16 and mu[i] == -mu[j], (i, float(x), mu[j])
        # weights: the exact weight, up to its first-order change at the rounded node
        # (|w'/w| = 2|x| / (1 - x^2) at a root of P_N) and the recurrence's rounding
        bound = abs(2 * x * dx / (1 - x * x)) + 4 * N * 2.2e-16
        assert abs(mp.mpf(w[j]) / wx - 1) <= bound and w[i] == w[j], (i, float(wx), w[j], float(bound))
