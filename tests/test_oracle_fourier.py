"""Pins of the angularly-discrete Fourier analysis tool (oracle.fourier, Sec. 3.3)
against closed forms, the one-iteration property of P_L-equivalent moments, the
paper's printed spectral radii (Table 1) and the oracle's own discrete iteration."""
import os

import numpy as np
import pytest

from oracle import fourier as fo
from oracle import iterations as it
from oracle import quadrature as qd
from paper_1907_13013_gb300 import inputs


def hg(c, g, L):
    return c * g ** np.arange(L + 1)


@pytest.mark.parametrize("N,c", [(8, hg(0.95, 0.7, 7)), (16, hg(0.99, 0.9, 15)), (16, hg(0.999, 0.9, 5))])
def test_si_sweep_matrix_closed_form(N, c):
    # Step 1: at lambda = 0 the sweep map is M diag(c) D, whose eigenvalues are the c_l
    # (zero beyond L); the SI spectral radius is c_0 = sigma_s0 / sigma_t, reached at lambda = 0
    cl = np.zeros(N)
    cl[:c.size] = c
    ev = np.linalg.eigvals(fo.sweep_matrix(0.0, c, N))
    assert np.abs(np.sort(ev.real) - np.sort(cl)).max() < 1e-13
    assert np.abs(ev.imag).max() < 1e-13
    r, lam = fo.sup_rho(c, N, "si")
    assert abs(r - c[0]) < 1e-12 and lam < 1e-6
    # away from lambda = 0 streaming only damps the mode
    assert all(fo.rho(x, c, N, "si") < c[0] for x in (0.1, 1.0, 10.0))


def test_sweep_matrix_is_paper_form():
    # A = Y^{-1} Z with Y[l,n] = w_n P_l(mu_n)(1 + i lambda mu_n), Z[l,n] = c_l w_n P_l(mu_n)
    # equals the per-ordinate form (I + i lambda H)^{-1} M diag(c) D
    N, lam = 8, 0.7
    c = hg(0.9, 0.6, 7)
    mu, w = qd.gauss_legendre(N)
    D = qd.moment_operator(mu, w, N - 1)
    M = qd.expansion_operator(mu, N - 1)
    ref = np.diag(1.0 / (1.0 + 1j * lam * mu)) @ M @ np.diag(c) @ D
    assert np.abs(fo.sweep_matrix(lam, c, N) - ref).max() < 1e-13


@pytest.mark.parametrize("N,c", [(8, hg(0.95, 0.7, 7)), (16, hg(0.9999, 0.9, 15)), (16, hg(0.99, 0.9, 7))])
def test_fpsa_mpd_flat_mode_closed_form(N, c):
    # lambda = 0 with MPD: D F = Lambda D decouples the Legendre moments, and the FPSA
    # error ratio of moment l is c_l - c_l (1 - c_l) / (sigma_a + sigma_tr l(l+1)/2)
    cl = np.zeros(N)
    cl[:c.size] = c
    l = np.arange(N)
    sa, st = 1.0 - cl[0], cl[0] - cl[1]
    pred = cl - cl * (1.0 - cl) / (sa + st * l * (l + 1) / 2.0)
    ev = np.linalg.eigvals(fo.fpsa_matrix(0.0, c, N, "mpd"))
    tol = 1e-14 / sa  # the l = 0 correction divides by sigma_a
    assert np.abs(np.sort(ev.real) - np.sort(pred)).max() < tol
    assert np.abs(ev.imag).max() < tol


@pytest.mark.parametrize("N", [4, 8, 16])
def test_pl_equivalent_moments_converge_in_one_iteration(N):
    # Eq. fsa_pl_eq: sigma_{s,l} = sigma_{s,0} - sigma_tr/2 l(l+1) with N = L + 1 makes FPSA
    # with MPD exact, I_M(lambda) = 0 at every lambda; WFD keeps only moments 0 and 1
    # and does not
    st, c0 = 0.02, 0.999
    l = np.arange(N)
    c = c0 - st / 2.0 * l * (l + 1)
    for lam in (0.0, 0.05, 0.7, 3.0, 40.0):
        assert np.abs(fo.fpsa_matrix(lam, c, N, "mpd")).max() < 1e-11
    if N > 2:
        assert fo.rho(0.7, c, N, "fpsa", "wfd") > 1e-3


def read_table1():
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "fourier_table1_hgk.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_table1_hgk_spectral_radii():
    # the paper's Table 1, HGK g = 0.9, L = 15, N = 16, FA columns (c = 0.9999: see the fixture)
    ref = read_table1()
    c = hg(0.9999, 0.9, 15)
    for lap in ("mpd", "wfd"):
        r, _ = fo.sup_rho(c, 16, "fpsa", lap)
        assert round(r, 4) == ref[lap], (lap, r)
    # and FPSA's whole point: SI alone sits at c_0
    assert abs(fo.sup_rho(c, 16, "si")[0] - 0.9999) < 1e-12


@pytest.mark.parametrize("lap", ["mpd", "wfd"])
def test_discrete_iteration_rate_equals_analysis_at_lambda0(lap):
    # a uniform slab with reflective edges carries the lambda = 0 modes exactly (LD is exact
    # for flat data); the supremum of this kernel is at lambda = 0, so the spectral radius
    # of the oracle's discrete FPSA iteration is the analysis' rho
    N, L = 16, 15
    c = hg(0.9999, 0.9, L)
    p = inputs.slab(12, N, L, 12.0, 1.0, c, 0.0)
    p["bc"] = "reflective"
    G = it.fpsa_iteration_matrix(p, lap)
    rho_disc = np.abs(np.linalg.eigvals(G)).max()
    r, lam = fo.sup_rho(c, N, "fpsa", lap)
    assert lam < 1e-6
    assert abs(rho_disc - r) < 1e-10, (rho_disc, r)


@pytest.mark.parametrize("lap", ["mpd", "wfd"])
def test_discrete_iteration_rate_converges_to_analysis_at_positive_lambda(lap):
    # isotropic scattering, c = 0.99: the FPSA supremum sits at lambda ~ 1.7 (the flat mode is
    # removed exactly). On a reflective slab of width Z the modes are cos(k pi z / Z); the
    # discrete spectral radius approaches the largest rho(k pi / Z) at third order in h
    N, L, Z = 8, 1, 20.0
    c = np.array([0.99, 0.0])
    r, lam = fo.sup_rho(c, N, "fpsa", lap)
    assert 1.0 < lam < 2.5
    target = fo.slab_mode_rho(c, N, Z, "fpsa", lap)
    assert 0.0 < r - target < 1e-4
    errs = []
    for K in (40, 80):
        p = inputs.slab(K, N, L, Z, 1.0, c, 0.0)
        p["bc"] = "reflective"
        rho_disc = np.abs(np.linalg.eigvals(it.fpsa_iteration_matrix(p, lap))).max()
        errs.append(abs(rho_disc - target))
    assert errs[1] < 4e-4
    assert errs[0] / errs[1] > 5.0, errs
