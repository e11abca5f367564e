"""Pins of the oracle adjoint (P9): central finite differences of the exit current and of a
linear functional of phi, consistency of the two objectives, and the transpose structure
A^T = W Pi A Pi W^{-1} of the LD / S_N system that the GPU adjoint relies on."""
import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import iterations as it
from oracle import quadrature as qd
from paper_1907_13013_gb300 import inputs


def problem(seed=3, K=9, N=8, kernel="srk"):
    return inputs.random_slab(K, N, N - 1, seed=seed, kernel=kernel, thick=(1, 60), c=(0.6, 0.98))


def J_of(p, g_phi=None):
    phi, psi = it.direct_solve(p, return_psi=True)
    return adj.exit_current_right(p, psi) if g_phi is None else float(np.sum(g_phi * phi))


@pytest.mark.parametrize("use_g", [False, True])
def test_adjoint_gradients_match_central_differences(use_g):
    p = problem()
    K, L = p["h"].size, p["L"]
    g = np.random.default_rng(1).standard_normal((K, 2, L + 1)) if use_g else None
    J, d_st, d_ss, _, _ = adj.gradients(p, g)
    assert abs(J - J_of(p, g)) < 1e-14 * max(1.0, abs(J))
    rel = 1e-5
    scale_t = np.abs(d_st).max()
    for i in (0, 3, K - 1):
        q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
        d = rel * p["sigma_t"][i]
        q["sigma_t"][i] += d; jp = J_of(q, g)
        q["sigma_t"][i] -= 2 * d; jm = J_of(q, g)
        assert abs((jp - jm) / (2 * d) - d_st[i]) < 1e-6 * scale_t
    scale_s = np.abs(d_ss).max()
    for i, l in ((1, 0), (4, 1), (K - 1, 3), (2, L)):
        q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
        d = rel * max(abs(p["sigma_s"][i, l]), 1e-3)
        q["sigma_s"][i, l] += d; jp = J_of(q, g)
        q["sigma_s"][i, l] -= 2 * d; jm = J_of(q, g)
        assert abs((jp - jm) / (2 * d) - d_ss[i, l]) < 1e-6 * scale_s


def test_exit_current_equals_moment_functional():
    # with L = N-1 the exit current is the linear functional of the last cell's right-node moments
    # g_l = sum_{mu_n > 0} w_n mu_n (2l+1)/2 P_l(mu_n); both objectives give the same gradients.
    p = problem(seed=5, K=7, N=6)
    N, L, K = p["N"], p["L"], p["h"].size
    mu, w = qd.gauss_legendre(N)
    M = qd.expansion_operator(mu, L)
    g = np.zeros((K, 2, L + 1))
    pos = mu > 0
    g[-1, 1] = (w[pos] * mu[pos]) @ M[pos]
    a = adj.gradients(p)
    b = adj.gradients(p, g)
    assert abs(a[0] - b[0]) < 1e-13 * abs(a[0])
    assert np.allclose(a[1], b[1], rtol=1e-10, atol=1e-14 * np.abs(a[1]).max())
    assert np.allclose(a[2], b[2], rtol=1e-10, atol=1e-14 * np.abs(a[2]).max())


@pytest.mark.parametrize("lap_problem", ["hg", "srk"])
def test_transpose_is_mirrored_weighted_system(lap_problem):
    # A^T = W Pi A Pi W^{-1}: W = diag(w_n) per node, Pi reverses the ordinates. Transposing the
    # LD upwind streaming of mu gives the streaming of -mu, and S = M Sigma D satisfies
    # S^T = W S W^{-1}, Pi S Pi = S (P_l(-mu) = (-1)^l P_l(mu), symmetric weights).
    p = problem(seed=8, K=5, N=6, kernel=lap_problem)
    N, K = p["N"], p["h"].size
    mu, w = qd.gauss_legendre(N)
    A = it.transport_matrix(p, mu, w).toarray()
    perm = np.concatenate([(2 * i + a) * N + np.arange(N - 1, -1, -1) for i in range(K) for a in range(2)])
    Wd = np.tile(w, 2 * K)
    P = np.eye(2 * K * N)[perm]
    rhs = np.diag(Wd) @ P @ A @ P @ np.diag(1 / Wd)
    assert np.abs(A.T - rhs).max() < 1e-12 * np.abs(A).max()
    # the FP operators (MPD and WFD) have the same structure
    for lap in ("mpd", "wfd"):
        F = it.fp_matrix(p, mu, w, lap).toarray()
        assert np.abs(F.T - np.diag(Wd) @ P @ F @ P @ np.diag(1 / Wd)).max() < 1e-10 * np.abs(F).max()
