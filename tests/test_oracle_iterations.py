"""Pins of the oracle's SI / FPSA iterations (P4-P8, P11) against closed forms,
the paper's stated identities, invariants and brute force."""
import numpy as np
import pytest

from oracle import iterations as it
from oracle import quadrature as qd
from oracle import transport as tr
from paper_1907_13013_gb300 import inputs


def uniform_reflective(K=3, N=8, L=7, st=10.0, c=0.9, g=0.8, S=1.0):
    p = inputs.slab(K, N, L, 1.0, st, c * st * inputs.hg_moments(g, L), S)
    p["bc"] = "reflective"
    return p


def test_si_infinite_medium_closed_form():
    # P4 / Sec. 2.1: for an infinite homogeneous medium with isotropic source S, SI from
    # phi=0 gives phi_0^m = (S/sigma_t) sum_{k<m} c^k, c = sigma_s0/sigma_t; higher moments stay 0.
    st, c, S = 10.0, 0.9, 1.0
    p = uniform_reflective(st=st, c=c, S=S)
    phi = None
    for m in range(1, 6):
        phi, _ = it.source_iteration(p, tol=0.0, max_it=1, phi0=phi)
        expect = S / st * sum(c ** k for k in range(m))
        assert np.abs(phi[..., 0] - expect).max() < 1e-13
        assert np.abs(phi[..., 1:]).max() < 1e-13


@pytest.mark.parametrize("lap", ["mpd", "wfd"])
def test_fpsa_infinite_medium_one_step(lap):
    # P4: the flat isotropic error mode is corrected exactly by the FP operator
    # (L_FP annihilates constants, so F acts as sigma_a): phi_0 = S/sigma_a after one iteration.
    st, c, S = 10.0, 0.9, 1.0
    p = uniform_reflective(st=st, c=c, S=S)
    phi, _ = it.fpsa_source_iteration(p, lap, tol=0.0, max_it=1)
    assert np.abs(phi[..., 0] - S / (st * (1 - c))).max() < 1e-12


@pytest.mark.parametrize("l", [0, 2, 4, 6])
def test_flat_mode_error_ratios(l):
    # P6: flat even-l error mode, reflective edges, zero source.
    #  SI ratio = sigma_{s,l}/sigma_t (the SI eigenvalues of Sec. 2.1);
    #  FPSA-MPD ratio = c_l - sigma_{s,l}(1 - c_l)/(sigma_a + sigma_tr l(l+1)/2),
    #  because MPD keeps P_l an eigenfunction of the discrete L_FP (Eq. fp-mpd).
    st, c, g = 10.0, 0.95, 0.9
    p = uniform_reflective(st=st, c=c, g=g, S=0.0)
    L = p["L"]
    ss = p["sigma_s"][0]
    phi0 = np.zeros((p["h"].size, 2, L + 1)); phi0[..., l] = 1.0
    phi_si, _ = it.source_iteration(p, tol=0.0, max_it=1, phi0=phi0)
    cl = ss[l] / st
    assert np.abs(phi_si[..., l] - cl).max() < 1e-12
    assert np.abs(np.delete(phi_si, l, axis=-1)).max() < 1e-12
    phi_f, _ = it.fpsa_source_iteration(p, "mpd", tol=0.0, max_it=1, phi0=phi0)
    sa, s_tr = st - ss[0], ss[0] - ss[1]
    ratio = cl - ss[l] * (1 - cl) / (sa + s_tr * l * (l + 1) / 2)
    assert np.abs(phi_f[..., l] - ratio).max() < 1e-11


@pytest.mark.parametrize("N,K,seed", [(4, 6, 0), (8, 11, 1), (16, 25, 2)])
def test_fpsa_pl_equivalent_converges_in_one_iteration(N, K, seed):
    # P5 / Eq. fsa_pl_eq: with P_L-equivalent moments and N = L+1 the MPD FP operator
    # equals L - S exactly, so one FPSA iteration returns the discrete solution.
    p = inputs.pl_equivalent_slab(K, N, seed)
    ref = it.direct_solve(p)
    phi, _ = it.fpsa_source_iteration(p, "mpd", tol=0.0, max_it=1)
    assert np.abs(phi - ref).max() < 1e-10 * np.abs(ref).max()
    # WFD does not share the identity: it needs more iterations (Sec. 3.3)
    phi_w, _ = it.fpsa_source_iteration(p, "wfd", tol=0.0, max_it=1)
    assert np.abs(phi_w - ref).max() > 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("kernel", ["hg", "srk"])
def test_iterations_reach_direct_solution(kernel):
    # P7 brute force: SI and FPSA (MPD, WFD) converge to the unique discrete solution.
    p = inputs.random_slab(12, 8, 7, seed=4, kernel=kernel, thick=(1, 30), c=(0.5, 0.9))
    ref = it.direct_solve(p)
    scale = np.abs(ref[..., 0]).max()
    for lap in ("mpd", "wfd"):
        phi, n = it.fpsa_source_iteration(p, lap, tol=1e-14, max_it=500)
        assert np.abs(phi - ref).max() < 1e-12 * scale
    phi, n = it.source_iteration(p, tol=1e-15, max_it=5000)
    assert np.abs(phi - ref).max() < 1e-11 * scale


def test_direct_solution_against_dense_brute_force():
    # P7: assemble L - S densely from the per-cell pieces written out here
    # (streaming + sigma_t mass - M diag(sigma_s) D mass) and compare with the oracle.
    p = inputs.random_slab(3, 4, 3, seed=9)
    N, L, K = p["N"], p["L"], 3
    mu, w = qd.gauss_legendre(N)
    P = qd.legendre_table(mu, L)
    D = P * w
    M = (P * ((2 * np.arange(L + 1) + 1) / 2)[:, None]).T
    n2 = 2 * N
    A = np.zeros((K * n2, K * n2)); b = np.zeros(K * n2)
    for i in range(K):
        hh = p["h"][i]
        m = hh / 6 * np.array([[2, 1], [1, 2]])
        Kc = p["sigma_t"][i] * np.eye(N) - M @ np.diag(p["sigma_s"][i]) @ D
        for a in range(2):
            for c in range(2):
                A[i * n2 + a * N:i * n2 + (a + 1) * N, i * n2 + c * N:i * n2 + (c + 1) * N] += m[a, c] * Kc
            qa = M @ p["Q"][i, 0] * m[a, 0] + M @ p["Q"][i, 1] * m[a, 1]
            b[i * n2 + a * N:i * n2 + (a + 1) * N] = qa
        for n in range(N):
            L0, R0 = i * n2 + n, i * n2 + N + n
            if mu[n] > 0:
                A[L0, L0] += mu[n] / 2; A[L0, R0] += mu[n] / 2
                A[R0, L0] += -mu[n] / 2; A[R0, R0] += mu[n] / 2
                if i > 0:
                    A[L0, (i - 1) * n2 + N + n] -= mu[n]
            else:
                A[L0, L0] += -mu[n] / 2; A[L0, R0] += mu[n] / 2
                A[R0, L0] += -mu[n] / 2; A[R0, R0] += -mu[n] / 2
                if i < K - 1:
                    A[R0, (i + 1) * n2 + n] += mu[n]
    psi = np.linalg.solve(A, b).reshape(K, 2, N)
    ref = np.einsum("ln,kan->kal", D, psi)
    assert np.abs(it.direct_solve(p) - ref).max() < 1e-12 * np.abs(ref).max()


def test_converged_particle_balance():
    # P8: LD with consistent mass conserves particles and S conserves the l=0 moment:
    # emission = absorption + leakage at the converged solution.
    p = inputs.random_slab(30, 16, 15, seed=6, kernel="srk", thick=(5, 200), c=(0.9, 0.999))
    N = p["N"]
    phi, n, psi = it.fpsa_source_iteration(p, "mpd", tol=1e-14, max_it=500, return_psi=True)
    mu, w = qd.gauss_legendre(N)
    h = p["h"]
    sa = p["sigma_t"] - p["sigma_s"][:, 0]
    emission = np.sum(h * (p["Q"][:, 0, 0] + p["Q"][:, 1, 0]) / 2)
    absorption = np.sum(sa * h * (phi[:, 0, 0] + phi[:, 1, 0]) / 2)
    jl, jr = tr.exit_currents(mu, w, psi)
    assert abs(emission - absorption - jl - jr) < 1e-11 * emission


def test_si_spectral_radius_bound_and_thick_limit():
    # P11 / Sec. 2.1: SI eigenvalues are sigma_{s,l}/sigma_t; measured error ratios on a
    # finite slab are bounded by max_l of them and approach sigma_s0/sigma_t for a thick slab.
    c = 0.95
    for st, lo in ((5.0, 0.5), (400.0, 0.93)):
        p = inputs.slab(40, 8, 7, 1.0, st, c * st * inputs.hg_moments(0.7, 7), 1.0)
        _, n, hist = it.source_iteration(p, tol=1e-9, max_it=3000, history=True)
        # geometric mean over the last 20 changes (well above rounding)
        ratio = (hist[-1] / hist[-21]) ** (1 / 20)
        assert ratio <= c + 1e-4
        assert ratio > lo


def test_fpsa_faster_than_si_forward_peaked():
    # Sec. 4: FPSA cuts the iteration count by orders of magnitude for forward-peaked kernels.
    p = inputs.plain_hg_slab(K=50)
    _, n_si = it.source_iteration(p, tol=1e-8, max_it=20000)
    _, n_f = it.fpsa_source_iteration(p, "mpd", tol=1e-8)
    assert n_f * 20 < n_si
