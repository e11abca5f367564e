"""GMRES-IR with its FP32 inner GMRES solves on tensor-core contractions (the FP
right-hand side from moments, the correction update and the moments of the sweep,
split BF16 on tcgen05; operators in shared memory for N <= 128, streamed for N = 256)
against the same solve on SIMT contractions and the FP64 oracle, through the C ABI:
both reach the oracle's converged flux (1e-9) in a similar number of Krylov steps."""
import numpy as np
import pytest

from oracle import iterations as oit
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


def relerr(a, b):
    return np.abs(a - b).max() / np.abs(b[..., 0]).max()


@pytest.mark.parametrize("N,K,R", [(16, 150, 2), (64, 97, 1), (128, 40, 2), (256, 33, 2)])
def test_gmres_ir_tensor_contractions(binding, N, K, R):
    p = inputs.random_slab(K, N, N - 1, seed=970 + N, kernel="srk", thick=(5, 300), c=(0.9, 0.999))
    rng = np.random.default_rng(N)
    p["Q"] = np.concatenate([p["Q"][None]] + [rng.uniform(0, 1, (1,) + p["Q"].shape) for _ in range(R - 1)])
    ctx = binding.context_for(p, laplacian="mpd", precision="mixed")
    phi_t, st_t = ctx.solve("gmres", tol=1e-12, max_iterations=100, restart=20, contraction="tensor")
    phi_s, st_s = ctx.solve("gmres", tol=1e-12, max_iterations=100, restart=20, contraction="simt")
    ctx.close()
    assert st_t["status"] == 0 and st_s["status"] == 0
    assert st_t["outer_iterations"] <= st_s["outer_iterations"] + 1, (st_t, st_s)
    for r in range(R):
        ref = oit.direct_solve(dict(p, Q=p["Q"][r]))
        assert relerr(phi_t[r], ref) < 1e-9, (r, relerr(phi_t[r], ref))
        assert relerr(phi_s[r], ref) < 1e-9
