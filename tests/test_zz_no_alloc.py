"""The allocation-free sweep entry point, checked against the context entry point.

fpsa_sweep_noalloc serves callers that cannot call cudaMalloc (an outside memory
pool, allocation-free graph recording, memory reserved up front): it keeps its
coefficient scratch in a fixed device array. Its sweep, followed by the moment
sum phi = D psi, must reproduce one source iteration of fpsa_solve
(method SI, one iteration from phi0), i.e. phi^1 = D L^{-1} M (Sigma phi0 + Q).
Two calls in a row with different slabs check that the shared array's leftover
contents from the first call do not leak into the second.
This file sorts last so a run that stops at the first failure has run the rest.
"""
import numpy as np
import pytest

from oracle import quadrature as qd
from paper_1907_13013_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def one_si_step_with_context(binding, p, phi0):
    ctx = binding.context_for(p)
    out, st = ctx.solve("si", tol=0.0, max_iterations=1, phi0=phi0[None], raise_on_notconv=False)
    ctx.close()
    return out[0]


def one_si_step_with_noalloc(binding, p, phi0):
    import torch
    N, L = p["N"], p["L"]
    mu, w = qd.gauss_legendre(N)
    D = qd.moment_operator(mu, w, L)
    M = qd.expansion_operator(mu, L)
    q = np.einsum("nl,kal->kan", M, p["sigma_s"][:, None, :] * phi0 + p["Q"])
    dev = torch.device("cuda:0")
    K = p["h"].size
    psi = torch.full((K, 2, N), np.nan, dtype=torch.float64, device=dev)
    binding.sweep_noalloc(N, torch.tensor(p["h"], device=dev), torch.tensor(p["sigma_t"], device=dev),
                          torch.tensor(q, device=dev), psi)
    torch.cuda.synchronize()
    return np.einsum("ln,kan->kal", D, psi.cpu().numpy())


def test_noalloc_sweep_matches_context_solve_twice_in_a_row():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_1907_13013_gb300 import binding
    torch.cuda.set_device(0)
    cases = [inputs.random_slab(500, 16, 15, seed=31, kernel="srk", thick=(5, 300), c=(0.9, 0.999)),
             inputs.random_slab(1999, 64, 63, seed=32, kernel="hg", thick=(1, 100), c=(0.5, 0.99))]
    rng = np.random.default_rng(5)
    for p in cases:
        phi0 = rng.uniform(0.0, 1.0, (p["h"].size, 2, p["L"] + 1))
        ref = one_si_step_with_context(binding, p, phi0)
        got = one_si_step_with_noalloc(binding, p, phi0)
        err = np.abs(got - ref).max() / np.abs(ref[..., 0]).max()
        assert err < TOL, err
    # requests beyond the fixed scratch capacity are refused before any work is enqueued
    dev = torch.device("cuda:0")
    K = binding.NOALLOC_MAX_CELL_ANGLES // 16 + 1
    z = torch.zeros(K, dtype=torch.float64, device=dev)
    big = torch.zeros((K, 2, 16), dtype=torch.float64, device=dev)
    with pytest.raises(binding.FpsaError) as e:
        binding.sweep_noalloc(16, z, z, big, big)
    assert e.value.code == binding.ENOTSUP
