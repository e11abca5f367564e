"""The allocation-free sweep entry point, checked against the oracle's sweep and the context entry point.

fpsa_sweep_noalloc serves callers that cannot call cudaMalloc (code inside another
framework's memory pool or allocator lock, a process whose device memory is
reserved up front): it keeps its coefficient scratch in a fixed device array.
Each call's angular flux is compared element by element with the oracle's LD
sweep (oracle.transport.sweep) on the same nodal source, and its moments D psi
with one source iteration of fpsa_solve (method SI, one iteration from phi0),
phi^1 = D L^{-1} M (Sigma phi0 + Q). The calls run large slab first, then a
smaller slab with other cross sections twice, so that coefficients a larger
call left in the shared array would show up in the smaller one; free device
memory is the same before and after the calls.
This file sorts last so a run that stops at the first failure has run the rest.
"""
import numpy as np
import pytest

from oracle import quadrature as qd
from oracle import transport as ot
from paper_1907_13013_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def one_si_step_with_context(binding, p, phi0):
    ctx = binding.context_for(p)
    out, st = ctx.solve("si", tol=0.0, max_iterations=1, phi0=phi0[None], raise_on_notconv=False)
    ctx.close()
    return out[0]


def nodal_source(p, phi0):
    N, L = p["N"], p["L"]
    mu, w = qd.gauss_legendre(N)
    M = qd.expansion_operator(mu, L)
    return np.einsum("nl,kal->kan", M, p["sigma_s"][:, None, :] * phi0 + p["Q"])


def test_noalloc_sweep_matches_oracle_and_context_repeatedly():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_1907_13013_gb300 import binding
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    large = inputs.random_slab(1999, 64, 63, seed=32, kernel="hg", thick=(1, 100), c=(0.5, 0.99))
    small = inputs.random_slab(500, 16, 15, seed=31, kernel="srk", thick=(5, 300), c=(0.9, 0.999))
    rng = np.random.default_rng(5)
    cases = []
    for p in (large, small):
        phi0 = rng.uniform(0.0, 1.0, (p["h"].size, 2, p["L"] + 1))
        q = nodal_source(p, phi0)
        mu, w = qd.gauss_legendre(p["N"])
        cases.append(dict(p=p, q=q, psi_ref=ot.sweep(mu, p["sigma_t"], p["h"], q),
                          phi_ref=one_si_step_with_context(binding, p, phi0),
                          D=qd.moment_operator(mu, w, p["L"])))
    torch.cuda.synchronize()
    # every device buffer of the calls exists before free memory is recorded
    for c in cases:
        p = c["p"]
        c["dev"] = (torch.tensor(p["h"], device=dev), torch.tensor(p["sigma_t"], device=dev),
                    torch.tensor(c["q"], device=dev),
                    torch.full(c["q"].shape, np.nan, dtype=torch.float64, device=dev))
    big_n = binding.NOALLOC_MAX_CELL_ANGLES // 16 + 1
    z = torch.zeros(big_n, dtype=torch.float64, device=dev)
    big = torch.zeros((big_n, 2, 16), dtype=torch.float64, device=dev)

    def run(c):
        h, st, q, psi = c["dev"]
        psi.fill_(np.nan)
        binding.sweep_noalloc(c["p"]["N"], h, st, q, psi)
        torch.cuda.synchronize()
        got = psi.cpu().numpy()
        err_psi = np.abs(got - c["psi_ref"]).max() / np.abs(c["psi_ref"]).max()
        assert err_psi < TOL, err_psi
        phi = np.einsum("ln,kan->kal", c["D"], got)
        err_phi = np.abs(phi - c["phi_ref"]).max() / np.abs(c["phi_ref"][..., 0]).max()
        assert err_phi < TOL, err_phi

    run(cases[1])  # first call on the device: its one-time set-up
    free0 = torch.cuda.mem_get_info()[0]
    for c in (cases[0], cases[1], cases[1]):
        run(c)
    # requests beyond the fixed scratch capacity are refused before any work is enqueued
    with pytest.raises(binding.FpsaError) as e:
        binding.sweep_noalloc(16, z, z, big, big)
    assert e.value.code == binding.ENOTSUP
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
