"""Pins of the oracle's LD discretization and sweep (P3, brute force, P8 per sweep)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import quadrature as qd
from oracle import transport as tr


def pade12(tau):
    return (6 - 2 * tau) / (6 + 4 * tau + tau ** 2)


def test_pure_absorber_exit_is_product_of_pade_factors():
    # P3: with no scattering and no source, each cell maps the inflow by the LD
    # transmission factor, the [1/2] Pade approximant of exp(-tau), tau = sigma h/|mu|.
    rng = np.random.default_rng(3)
    K, N = 17, 8
    mu, w = qd.gauss_legendre(N)
    h = rng.uniform(0.01, 0.2, K)
    st = rng.uniform(0.5, 20.0, K)
    inflow = rng.uniform(0.5, 2.0, N)
    psi = tr.sweep(mu, st, h, np.zeros((K, 2, N)), inflow, inflow)
    for n in range(N):
        tau = st * h / abs(mu[n])
        expect = inflow[n] * np.prod(pade12(tau))
        got = psi[-1, 1, n] if mu[n] > 0 else psi[0, 0, n]
        assert abs(got - expect) <= 1e-13 * abs(expect) + 1e-300


def test_pure_absorber_converges_third_order():
    # The Pade[1/2] transmission has a local error O(tau^4), so the exit flux of a
    # pure absorber converges to exp(-sigma Z/mu) at third order in h.
    mu, w = qd.gauss_legendre(4)
    n = 3
    errs = []
    for K in (10, 20, 40, 80):
        psi = tr.sweep(mu, np.full(K, 3.0), np.full(K, 1.0 / K), np.zeros((K, 2, 4)), np.ones(4), np.ones(4))
        errs.append(abs(psi[-1, 1, n] - np.exp(-3.0 / mu[n])))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 3.0) < 0.15), rates


def galerkin_cell_system(mu_n, sigma, h, qL, qR, inflow):
    """Build the LD equations of one cell directly from the weak form, by evaluating the
    basis functions at 3-point Gauss points on the cell (independent of the oracle's
    closed-form blocks)."""
    xg, wg = np.polynomial.legendre.leggauss(3)
    z = 0.5 * h * (xg + 1)
    wz = 0.5 * h * wg
    b = np.stack([(h - z) / h, z / h])            # b_L, b_R at the points
    db = np.array([-1.0 / h, 1.0 / h])
    A = np.zeros((2, 2)); rhs = np.zeros(2)
    q = qL * b[0] + qR * b[1]
    for j in range(2):
        for k in range(2):
            # -mu int b_j' b_k + sigma int b_j b_k
            A[j, k] = -mu_n * db[j] * np.sum(wz * b[k]) + sigma * np.sum(wz * b[j] * b[k])
        rhs[j] = np.sum(wz * b[j] * q)
    # boundary term mu [b_j psi_hat]_{0}^{h}, psi_hat upwind
    if mu_n > 0:
        A[1, 1] += mu_n            # b_R(h) = 1, psi_hat(h) = psi_R
        rhs[0] += mu_n * inflow    # -mu b_L(0) psi_in moved to the right
    else:
        A[0, 0] -= mu_n            # -mu b_L(0) psi_hat(0) with psi_hat(0) = psi_L
        rhs[1] -= mu_n * inflow    # mu b_R(h) psi_in moved to the right
    return A, rhs


def test_cell_equations_match_galerkin_weak_form():
    rng = np.random.default_rng(5)
    for mu_n in (-0.9, -0.2, 0.1, 0.7):
        h, sig = rng.uniform(0.01, 1.0), rng.uniform(0.1, 30.0)
        qL, qR, inflow = rng.uniform(0, 1, 3)
        A, rhs = galerkin_cell_system(mu_n, sig, h, qL, qR, inflow)
        mu = np.array([mu_n])
        psi = tr.sweep(mu, np.array([sig]), np.array([h]), np.array([[[qL], [qR]]]), [inflow], [inflow])
        assert np.allclose(psi[0, :, 0], np.linalg.solve(A, rhs), rtol=1e-13, atol=0)


def test_linear_manufactured_solution_is_exact():
    # LD reproduces a continuous linear solution exactly: psi = (a + b z)/sigma - mu b/sigma^2
    # solves mu psi' + sigma psi = a + b z with a constant sigma.
    mu, w = qd.gauss_legendre(6)
    K, sig, a, b = 9, 4.0, 1.0, 0.5
    edges = np.cumsum(np.r_[0.0, np.random.default_rng(7).uniform(0.05, 0.2, K)])
    h = np.diff(edges)
    q = np.zeros((K, 2, 6))
    q[:, 0, :] = (a + b * edges[:-1])[:, None]
    q[:, 1, :] = (a + b * edges[1:])[:, None]
    exact = lambda z: (a + b * z)[..., None] / sig - mu[None, :] * b / sig ** 2
    psi = tr.sweep(mu, np.full(K, sig), h, q, exact(edges[:1])[0], exact(edges[-1:])[0])
    assert np.abs(psi[:, 0, :] - exact(edges[:-1])).max() < 1e-13
    assert np.abs(psi[:, 1, :] - exact(edges[1:])).max() < 1e-13


@pytest.mark.parametrize("K,N", [(1, 2), (5, 4), (13, 8)])
def test_sweep_equals_global_matrix_solve(K, N):
    rng = np.random.default_rng(K * 100 + N)
    mu, w = qd.gauss_legendre(N)
    h = rng.uniform(0.01, 0.3, K)
    st = rng.uniform(0.1, 50, K)
    q = rng.uniform(0, 1, (K, 2, N))
    A = tr.assemble(mu, h, st[:, None, None] * np.eye(N)[None])
    ref = spla.spsolve(A.tocsc(), tr.mass_weight(h, q).ravel()).reshape(K, 2, N)
    assert np.allclose(tr.sweep(mu, st, h, q), ref, rtol=1e-12, atol=1e-14)


def test_sweep_particle_balance():
    # P8 for one sweep: leakage + absorption = emission, per ordinate summed with weights.
    rng = np.random.default_rng(11)
    K, N = 20, 16
    mu, w = qd.gauss_legendre(N)
    h = rng.uniform(0.01, 0.1, K)
    st = rng.uniform(1, 40, K)
    q = rng.uniform(0, 1, (K, 2, N))
    psi = tr.sweep(mu, st, h, q)
    emission = np.sum(w[None, :] * h[:, None] * (q[:, 0] + q[:, 1]) / 2)
    absorption = np.sum(w[None, :] * (st * h)[:, None] * (psi[:, 0] + psi[:, 1]) / 2)
    jl, jr = tr.exit_currents(mu, w, psi)
    assert abs(emission - absorption - jl - jr) < 1e-13 * emission
