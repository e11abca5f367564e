"""Angular discretization for the oracle (test infrastructure only; see package header).

S_N Gauss-Legendre quadrature, Legendre tables and the N x N angular operators
of Sec. 2.2 of arXiv:1907.13013:

- D (moments from angular fluxes): phi_l = sum_n w_n P_l(mu_n) psi_n, the S_N
  quadrature form of Eq. phi-mom.
- M (angular values from moments): the Legendre expansion (2l+1)/2 P_l(mu_n)
  that appears in the scattering source of Eq. treq.
- MPD angular Laplacian F = V^{-1} Lambda V of Eq. fp-mpd, with
  V_ij = P_{i-1}(mu_j) w_j and Lambda_ii = -i(i-1).
- WFD angular Laplacian W of Eq. w_wfd, with the gamma recurrence of
  Eq. sph-weights.

Ordinates are sorted ascending (mu_1 < ... < mu_N), weights sum to 2.
"""

import numpy as np


def gauss_legendre(N):
    """S_N Gauss-Legendre nodes and weights, mu ascending, sum(w) = 2 (Sec. 2.2).

    Nodes: the roots of P_N from numpy's Gauss-Legendre routine (a library
    primitive). Weights: the closed form of the Gauss-Legendre rule at those nodes,
    w_n = 2 / ((1 - mu_n^2) P_N'(mu_n)^2), with P_N'(x) = N (P_{N-1} - x P_N) / (1 - x^2)
    from the recurrence below and 1 - x^2 formed as (1 - x)(1 + x), which keeps its
    relative accuracy next to x = +-1 (numpy's own weights are rescaled
    approximations, off by up to 2e-11 relative at N = 256).
    Pinned by: exactness for polynomials of degree <= 2N-1, and nodes and weights
    against a 50-digit Newton solution of P_N = 0 (tests P1).
    """
    if N < 2 or N % 2:
        raise ValueError("N must be even and >= 2")
    mu, _ = np.polynomial.legendre.leggauss(N)
    mu = np.sort(mu).astype(np.float64)
    P = legendre_table(mu, N)
    one_minus_x2 = (1.0 - mu) * (1.0 + mu)
    dP = N * (P[N - 1] - mu * P[N]) / one_minus_x2
    w = 2.0 / (one_minus_x2 * dP * dP)
    return mu, w


def legendre_table(x, lmax):
    """P[l, j] = P_l(x_j) for l = 0..lmax by the three-term (Bonnet) recurrence.

    (l+1) P_{l+1} = (2l+1) x P_l - l P_{l-1}.
    Pinned by: closed forms of P_2, P_3 and orthogonality under Gauss-Legendre.
    """
    x = np.asarray(x, dtype=np.float64)
    P = np.zeros((lmax + 1, x.size))
    P[0] = 1.0
    if lmax >= 1:
        P[1] = x
    for l in range(1, lmax):
        P[l + 1] = ((2 * l + 1) * x * P[l] - l * P[l - 1]) / (l + 1)
    return P


def moment_operator(mu, w, L):
    """D[l, n] = w_n P_l(mu_n), l = 0..L: phi_l = D psi (Eq. phi-mom by quadrature)."""
    return legendre_table(mu, L) * w[None, :]


def expansion_operator(mu, L):
    """M[n, l] = (2l+1)/2 P_l(mu_n), l = 0..L: the Legendre sum of Eq. treq.

    The scattering source at ordinate n is sum_l M[n,l] sigma_{s,l} phi_l.
    """
    l = np.arange(L + 1)
    return (legendre_table(mu, L) * ((2 * l + 1) / 2.0)[:, None]).T


def mpd_laplacian(mu, w):
    """MPD discrete angular Laplacian F = V^{-1} Lambda V (Eq. fp-mpd).

    V_ij = P_{i-1}(mu_j) w_j, Lambda_ii = -i(i-1), i, j = 1..N. V^{-1} is taken
    with a dense inverse exactly as the equation is written (no use of the
    Gauss-Legendre identity V^{-1} = M), so that the identity itself is a pin.
    Pinned by: F P_l(mu) = -l(l+1) P_l(mu) for l <= N-1 (Eq. legendre, P2).
    """
    N = mu.size
    V = legendre_table(mu, N - 1) * w[None, :]
    lam = -np.arange(N) * (np.arange(N) + 1.0)
    return np.linalg.solve(V, lam[:, None] * V)


def wfd_gamma(mu, w):
    """gamma_{n+1/2}, n = 0..N (gamma[0] = gamma_{1/2}), Eq. sph-weights.

    Reading of the paper's undefined normalization nu: with mu ascending and
    sum(w) = 2 the recurrence is gamma_{n+1/2} = gamma_{n-1/2} - 2 mu_n w_n from
    gamma_{1/2} = 0, which approximates 1 - mu^2 at the cell edges and returns
    gamma_{N+1/2} = 0 (sum_n w_n mu_n = 0).
    """
    g = np.zeros(mu.size + 1)
    for n in range(mu.size):
        g[n + 1] = g[n] - 2.0 * mu[n] * w[n]
    return g


def wfd_laplacian(mu, w):
    """WFD tridiagonal angular Laplacian W of Eq. w_wfd (row n carries 1/w_n).

    (W psi)_n = [gamma_{n+1/2} (psi_{n+1}-psi_n)/(mu_{n+1}-mu_n)
                 - gamma_{n-1/2} (psi_n-psi_{n-1})/(mu_n-mu_{n-1})] / w_n   (Eq. fp-wdd)
    Pinned by: zeroth and first moments preserved (l = 0, 1; Sec. 3.3), row sums 0,
    diag(w) W symmetric, M-matrix sign pattern (Sec. 2.2).
    """
    N = mu.size
    g = wfd_gamma(mu, w)
    W = np.zeros((N, N))
    for n in range(N):
        if n > 0:
            W[n, n - 1] = g[n] / (mu[n] - mu[n - 1]) / w[n]
        if n < N - 1:
            W[n, n + 1] = g[n + 1] / (mu[n + 1] - mu[n]) / w[n]
        W[n, n] = -(W[n, n - 1] if n > 0 else 0.0) - (W[n, n + 1] if n < N - 1 else 0.0)
    return W


def angular_laplacian(mu, w, kind):
    """The discrete L_FP used by the FP operator: 'mpd' (Eq. fp-mpd) or 'wfd' (Eq. w_wfd)."""
    if kind == "mpd":
        return mpd_laplacian(mu, w)
    if kind == "wfd":
        return wfd_laplacian(mu, w)
    raise ValueError(kind)
