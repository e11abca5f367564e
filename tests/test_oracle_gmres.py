"""Pins of the oracle's FPSA-preconditioned GMRES(m) (Sec. 4): same fixed point as the direct
solve, finite termination of full GMRES, monotone residuals within a cycle, and fewer
iterations than FPSA source iteration on a forward-peaked slab."""
import numpy as np
import pytest

from oracle import iterations as it
from paper_1907_13013_gb300 import inputs


@pytest.mark.parametrize("lap", ["mpd", "wfd"])
def test_gmres_reaches_direct_solution(lap):
    p = inputs.random_slab(15, 8, 7, seed=31, kernel="srk", thick=(5, 200), c=(0.9, 0.999))
    ref = it.direct_solve(p)
    phi, n = it.fpsa_gmres(p, lap, restart=30, tol=1e-13)
    assert np.abs(phi - ref).max() < 1e-10 * np.abs(ref[..., 0]).max()


def test_full_gmres_terminates_within_dimension():
    # without restarts GMRES minimises over the whole Krylov space: it terminates in
    # at most dim = K * 2 * (L+1) iterations (here 2 * 2 * 4 = 16)
    p = inputs.random_slab(2, 4, 3, seed=32, c=(0.9, 0.99))
    dim = 2 * 2 * 4
    ref = it.direct_solve(p)
    phi, n, hist = it.fpsa_gmres(p, "wfd", restart=dim, tol=1e-14, history=True)
    assert n <= dim
    assert np.abs(phi - ref).max() < 1e-11 * np.abs(ref[..., 0]).max()


def test_gmres_residuals_monotone_within_cycles():
    p = inputs.random_slab(20, 8, 7, seed=33, kernel="hg", thick=(10, 300), c=(0.95, 0.999))
    _, n, hist = it.fpsa_gmres(p, "mpd", restart=5, tol=1e-12, history=True)
    h = np.array(hist)
    for c0 in range(0, len(h), 5):
        cyc = h[c0:c0 + 5]
        assert np.all(np.diff(cyc) <= 1e-14 * cyc[0])


def test_gmres_needs_fewer_iterations_than_fpsa_si():
    p = inputs.plain_hg_slab(K=60)
    _, n_si = it.fpsa_source_iteration(p, "mpd", tol=1e-10)
    _, n_g = it.fpsa_gmres(p, "mpd", restart=30, tol=1e-10)
    assert n_g < n_si
