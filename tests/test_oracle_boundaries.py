"""Pins of the oracle's boundary conditions: given incoming fluxes (the beam source of
Sec. 4) and reflective edges, against closed forms, mirror symmetry and invariants."""
import numpy as np
import pytest

from oracle import iterations as it
from oracle import quadrature as qd
from oracle import transport as tr
from paper_1907_13013_gb300 import inputs


@pytest.mark.parametrize("side", ["left", "right"])
@pytest.mark.parametrize("N,K,seed", [(4, 5, 0), (8, 9, 1), (16, 7, 2)])
def test_reflective_half_slab_equals_symmetric_slab(side, N, K, seed):
    # Mirror symmetry: a reflective edge is the symmetry plane of a slab twice as wide.
    half, full, part = inputs.mirrored_half_slab(K, N, N - 1, seed, side)
    ref = it.direct_solve(full)[part]
    got = it.direct_solve(half)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    # the iterations reach it too, through the LU streaming inverse of a reflective edge
    for lap in ("mpd", "wfd"):
        phi, _ = it.fpsa_source_iteration(half, lap, tol=1e-13, max_it=500)
        assert np.abs(phi - ref).max() < 1e-10 * np.abs(ref).max()
    phi, _ = it.fpsa_gmres(half, "wfd", tol=1e-13)
    assert np.abs(phi - ref).max() < 1e-10 * np.abs(ref).max()


def test_beam_through_pure_absorber():
    # P3 with a given inflow: a unit beam on the most normal ordinate of a pure absorber
    # leaves the far edge multiplied by the product of the cells' Pade[1/2] factors;
    # every other ordinate stays zero.
    N, K = 8, 13
    p = inputs.random_slab(K, N, 3, seed=5)
    p["sigma_s"][:] = 0.0
    p["Q"][:] = 0.0
    mu, w = qd.gauss_legendre(N)
    for side in ("left", "right"):
        p["psi_inc"] = tr.beam_incident(mu, w, side)
        _, psi = it.direct_solve(p, return_psi=True)
        n = N - 1 if side == "left" else 0
        tau = p["sigma_t"] * p["h"] / abs(mu[n])
        alpha = (6 - 2 * tau) / (6 + 4 * tau + tau ** 2)
        exit_val = psi[-1, 1, n] if side == "left" else psi[0, 0, n]
        assert abs(exit_val - np.prod(alpha) / (w[n] * abs(mu[n]))) < 1e-13 * abs(exit_val) + 1e-300
        others = np.delete(psi, n, axis=2)
        assert np.abs(others).max() == 0.0
        # unit incoming partial current
        assert abs(w[n] * abs(mu[n]) * p["psi_inc"][0 if side == "left" else 1, n] - 1.0) < 1e-14


@pytest.mark.parametrize("bc", ["vacuum", ("reflective", "vacuum"), ("vacuum", "reflective")])
def test_particle_balance_with_incoming_flux(bc):
    # P8 with boundary sources: source + incoming partial currents at the vacuum edges
    # = absorption + outgoing partial currents at the vacuum edges (a reflective edge
    # has zero net current).
    N, K = 8, 20
    p = inputs.random_slab(K, N, N - 1, seed=6, thick=(1, 20), c=(0.5, 0.99))
    p["bc"] = bc
    rng = np.random.default_rng(inputs.SEED_BASE + 600)
    p["psi_inc"] = rng.uniform(0, 2, (2, N))
    mu, w, D, _ = it.tables(N, N - 1)
    phi, psi = it.direct_solve(p, return_psi=True)
    left, right = tr.bc_sides(bc)
    h = p["h"]
    source = np.sum(h * 0.5 * (p["Q"][:, 0, 0] + p["Q"][:, 1, 0]))
    absorb = np.sum((p["sigma_t"] - p["sigma_s"][:, 0]) * h * 0.5 * (phi[:, 0, 0] + phi[:, 1, 0]))
    pos, neg = mu > 0, mu < 0
    j_in = j_out = 0.0
    if left == "vacuum":
        j_in += np.sum(w[pos] * mu[pos] * p["psi_inc"][0, pos])
        j_out += np.sum(w[neg] * -mu[neg] * psi[0, 0, neg])
    if right == "vacuum":
        j_in += np.sum(w[neg] * -mu[neg] * p["psi_inc"][1, neg])
        j_out += np.sum(w[pos] * mu[pos] * psi[-1, 1, pos])
    assert abs(source + j_in - absorb - j_out) < 1e-11 * (source + j_in)


def test_reflective_edges_ignore_given_inflow():
    # a reflective edge takes its inflow from the outgoing flux only
    N, K = 8, 10
    p = inputs.random_slab(K, N, N - 1, seed=7)
    p["bc"] = ("reflective", "vacuum")
    a = it.direct_solve(p)
    p["psi_inc"] = np.zeros((2, N)); p["psi_inc"][0] = 5.0
    b = it.direct_solve(p)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("method", ["si", "fpsa", "gmres"])
def test_iterations_with_beam_reach_direct_solution(method):
    # the incoming flux enters the source sweeps only; error and Krylov sweeps are homogeneous
    N, K = 8, 15
    p = inputs.random_slab(K, N, N - 1, seed=8, thick=(1, 30), c=(0.5, 0.9))
    p["Q"][:] = 0.0
    mu, w = qd.gauss_legendre(N)
    p["psi_inc"] = tr.beam_incident(mu, w, "left")
    ref = it.direct_solve(p)
    if method == "si":
        phi, _ = it.source_iteration(p, tol=1e-14, max_it=5000)
    elif method == "fpsa":
        phi, _ = it.fpsa_source_iteration(p, "mpd", tol=1e-14, max_it=500)
    else:
        phi, _ = it.fpsa_gmres(p, "mpd", tol=1e-13)
    assert np.abs(phi - ref).max() < 1e-10 * np.abs(ref).max()


def test_bc_validation():
    with pytest.raises(ValueError):
        tr.bc_sides(("vacuum", "periodic"))
