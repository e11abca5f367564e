"""The GPU FPSA iteration (through the C ABI) contracts errors at the rate the
angularly-discrete Fourier analysis predicts (Sec. 3.3): on a uniform slab with
reflective edges, a spatially flat error equal to the analysis' dominant lambda = 0
eigenvector is multiplied by rho = sup_lambda rho(I_M(lambda)) in every iteration
(the paper's Table 1 problem, HGK g = 0.9, N = 16, L = 15, c = 0.9999)."""
import numpy as np
import pytest

from oracle import fourier as fo
from oracle import quadrature as oqd
from paper_1907_13013_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_1907_13013_gb300 import binding as b
    return b


@pytest.mark.parametrize("lap", ["mpd", "wfd"])
def test_gpu_error_contraction_equals_fourier_rho(binding, lap):
    N, L, K = 16, 15, 24
    c = 0.9999 * 0.9 ** np.arange(L + 1)
    rho, lam = fo.sup_rho(c, N, "fpsa", lap)
    assert lam < 1e-6
    ev, vec = np.linalg.eig(fo.fpsa_matrix(0.0, c, N, lap))
    k = int(np.argmax(np.abs(ev)))
    assert abs(abs(ev[k]) - rho) < 1e-12
    v = vec[:, k]
    v = (v / v[np.argmax(np.abs(v))]).real  # real at lambda = 0
    mu, w = oqd.gauss_legendre(N)
    assert np.abs(v - v[::-1]).max() < 1e-10  # even in mu: consistent with reflective edges
    mom = oqd.moment_operator(mu, w, L) @ v
    p = inputs.slab(K, N, L, 30.0, 2.0, 2.0 * c, 0.0)
    p["bc"] = "reflective"
    ctx = binding.context_for(p, laplacian=lap, precision="fp64")
    phi0 = np.broadcast_to(mom, (1, K, 2, L + 1)).copy()
    prev = phi0
    for m in (1, 2, 3):
        phi, _ = ctx.solve("fpsa", tol=1e-300, max_iterations=m, phi0=phi0, raise_on_notconv=False)
        # each iteration multiplies the whole flat mode by rho (all cells, nodes, moments)
        assert np.abs(phi - rho * prev).max() < 1e-10 * np.abs(prev).max(), (m, lap)
        prev = phi
    ctx.close()
