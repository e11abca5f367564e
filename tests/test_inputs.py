"""Checks of the input generators' scattering-kernel moments (P10)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import quadrature as qd
from paper_1907_13013_gb300 import inputs


def test_hg_moments():
    assert np.allclose(inputs.hg_moments(0.9, 5), 0.9 ** np.arange(6), rtol=0, atol=1e-15)


@pytest.mark.parametrize("eta", [1e-3, 2.83e-5, 1e-5, 1e-6])
def test_srk_first_moment_closed_form(eta):
    # f_1 = 1 + 2 eta - 2 eta (1+eta) ln(1 + 1/eta) for sigma_s ~ (1 - mu0 + 2 eta)^-2
    f = inputs.srk_moments(eta, 3)
    assert f[0] == 1.0
    f1 = 1 + 2 * eta - 2 * eta * (1 + eta) * math.log1p(1 / eta)
    assert abs(f[1] - f1) < 1e-12


@pytest.mark.parametrize("eta,L", [(1e-3, 15), (1e-5, 63), (1e-6, 127)])
def test_srk_moments_against_quadrature(eta, L):
    # Direct numerical integration of the normalised kernel against P_l.
    f = inputs.srk_moments(eta, L)
    a = 1 + 2 * eta
    norm = 2 / (a * a - 1)
    for l in (2, 5, L // 2, L):
        val, _ = integrate.quad(lambda x: qd.legendre_table(np.array([x]), l)[l, 0] / (a - x) ** 2,
                                -1, 1, points=[1 - 10 * eta, 1 - 1000 * eta, 0.9], limit=500,
                                epsabs=0, epsrel=1e-13)
        assert abs(val / norm - f[l]) < 1e-9


def test_pl_equivalent_formula():
    p = inputs.pl_equivalent_slab(4, 8, 0)
    ss = p["sigma_s"]
    l = np.arange(8)
    s_tr = ss[:, 0] - ss[:, 1]
    assert np.allclose(ss, ss[:, :1] - 0.5 * s_tr[:, None] * l * (l + 1), rtol=1e-14)
