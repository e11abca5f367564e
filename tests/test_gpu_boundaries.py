"""GPU parity of the edge conditions (through the C ABI): given incoming fluxes (the
beam source of Sec. 4) and reflective edges, against the FP64 oracle, which is
itself pinned by mirror symmetry, the pure-absorber beam and particle balance."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import iterations as oit
from oracle import quadrature as oqd
from oracle import transport as otr
from paper_1907_13013_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def binding():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_1907_13013_gb300 import binding as b
    return b


def relerr(phi, ref):
    return np.abs(phi - ref).max() / np.abs(ref[..., 0]).max()


def edge_slab(K, N, seed, bc, beam=None, kernel="srk"):
    p = inputs.random_slab(K, N, N - 1, seed=seed, kernel=kernel, thick=(2, 200), c=(0.7, 0.995))
    p["bc"] = bc
    if beam:
        mu, w = oqd.gauss_legendre(N)
        p["psi_inc"] = otr.beam_incident(mu, w, beam)
    return p


CASES = [(("reflective", "vacuum"), None), (("vacuum", "reflective"), "left"), ("reflective", None),
         ("vacuum", "left"), ("vacuum", "right")]


@pytest.mark.parametrize("bc,beam", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("method", ["fpsa", "gmres"])
def test_edges_against_oracle(binding, bc, beam, precision, method):
    p = edge_slab(40, 16, 200, bc, beam)
    ref = oit.direct_solve(p)
    for lap in ("mpd", "wfd"):
        ctx = binding.context_for(p, laplacian=lap, precision=precision)
        phi, st = ctx.solve(method, tol=1e-13 if method == "fpsa" else 1e-12, max_iterations=500)
        assert relerr(phi[0], ref) < TOL, (lap, relerr(phi[0], ref), st)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_si_with_edges(binding, precision):
    p = edge_slab(25, 8, 201, ("reflective", "vacuum"), "right", kernel="hg")
    p["sigma_s"] *= 0.5  # a fast-converging SI problem
    ref = oit.direct_solve(p)
    ctx = binding.context_for(p, precision=precision)
    phi, _ = ctx.solve("si", tol=1e-14, max_iterations=3000)
    assert relerr(phi[0], ref) < TOL


def test_mirror_half_slab_on_gpu(binding):
    # the half slab with a reflective edge equals the symmetric full slab on the GPU too
    half, full, part = inputs.mirrored_half_slab(60, 32, 31, 3, "left")
    a = binding.context_for(half).solve("fpsa", tol=1e-13)[0][0]
    b = binding.context_for(full).solve("fpsa", tol=1e-13)[0][0][part]
    assert relerr(a, b) < TOL


@pytest.mark.parametrize("lap", ["mpd", "wfd"])
def test_infinite_medium_one_fpsa_iteration(binding, lap):
    # P4 on the GPU: reflective at both edges, uniform medium, isotropic source: phi_0 = S/sigma_a,
    # higher moments 0, reached by one FPSA iteration (the second only confirms the change is 0)
    st, c, S, K, N = 10.0, 0.9, 1.0, 17, 16
    p = inputs.slab(K, N, N - 1, 1.0, st, c * st * inputs.hg_moments(0.8, N - 1), S)
    p["bc"] = "reflective"
    ctx = binding.context_for(p)
    phi, stats = ctx.solve("fpsa", tol=1e-12, max_iterations=10)
    assert stats["iterations"] <= 2
    assert np.abs(phi[0, ..., 0] - S / (st * (1 - c))).max() < 1e-11 * S / (st * (1 - c))
    assert np.abs(phi[0, ..., 1:]).max() < 1e-11


def test_beam_through_pure_absorber(binding):
    # P3 with a beam: the exit value is the product of the cells' Pade[1/2] factors
    N, K = 16, 300
    p = inputs.random_slab(K, N, N - 1, seed=202)
    p["sigma_s"][:] = 0.0
    p["sigma_t"] *= 0.01
    p["Q"][:] = 0.0
    mu, w = oqd.gauss_legendre(N)
    p["psi_inc"] = otr.beam_incident(mu, w, "left")
    ctx = binding.context_for(p)
    phi, _ = ctx.solve("si", tol=1e-14, max_iterations=5)
    n = N - 1
    tau = p["sigma_t"] * p["h"] / mu[n]
    exit_val = np.prod((6 - 2 * tau) / (6 + 4 * tau + tau ** 2)) / (w[n] * mu[n])
    # psi at the right node of the last cell from its moments: psi_n = sum_l (2l+1)/2 P_l(mu_n) phi_l
    _, _, _, M = oit.tables(N, N - 1)
    psi_exit = M @ phi[0, -1, 1]
    assert abs(psi_exit[n] - exit_val) < 1e-12 * exit_val


def test_mixed_batch_of_edge_conditions(binding):
    # one context, instances with different edges and beams, ragged K (including K = 1)
    specs = [(37, "vacuum", None), (1, "reflective", None), (20, ("reflective", "vacuum"), "right"),
             (9, ("vacuum", "reflective"), "left"), (64, "reflective", None), (5, "vacuum", "left")]
    probs = [edge_slab(K, 16, 210 + i, bc, beam, kernel="hg") for i, (K, bc, beam) in enumerate(specs)]
    for precision in ("fp64", "mixed"):
        ctx = binding.context_for(probs, precision=precision, laplacian="wfd")
        phi, _ = ctx.solve("fpsa", tol=1e-13, max_iterations=500)
        off = 0
        for p in probs:
            K = p["h"].size
            assert relerr(phi[0, off:off + K], oit.direct_solve(p)) < TOL, (precision, K, p["bc"])
            off += K


@pytest.mark.parametrize("bc,beam", [(("reflective", "vacuum"), "right"), (("vacuum", "reflective"), "left"),
                                     ("vacuum", "left")])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_with_edges(binding, bc, beam, precision):
    # A^T = W Pi A Pi W^{-1} holds with reflective edges (the weights are mirror-symmetric);
    # the incoming flux is forward source only
    p = edge_slab(30, 16, 220, bc, beam)
    J, d_st, d_ss, _, _ = oadj.gradients(p)
    ctx = binding.context_for(p, precision=precision)
    ctx.solve("fpsa", tol=1e-13, max_iterations=500)
    gt, gs, Jg, _ = ctx.adjoint(tol=1e-13)
    assert abs(Jg[0, 0] - J) < 1e-10 * abs(J)
    assert np.abs(gt - d_st).max() < 1e-8 * np.abs(d_st).max()
    assert np.abs(gs - d_ss).max() < 1e-8 * np.abs(d_ss).max()


def test_incident_rules(binding):
    p = edge_slab(10, 8, 230, "vacuum", "left")
    ctx = binding.context_for(p)
    ctx.solve("fpsa", tol=1e-12)
    with pytest.raises(ValueError):
        ctx.set_incident(np.zeros((1, 1, 2, 4)))
    bad = np.zeros((1, 1, 2, 8)); bad[0, 0, 0, 5] = np.nan
    with pytest.raises(binding.FpsaError) as e:
        ctx.set_incident(bad)
    assert e.value.code == binding.ENONFINITE
    # a new incoming flux invalidates the forward state of the adjoint
    ctx.set_incident(None)
    with pytest.raises(binding.FpsaError) as e:
        ctx.adjoint()
    assert e.value.code == binding.ESTATE
