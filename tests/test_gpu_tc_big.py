"""Tensor-core contractions with streamed operators (N a multiple of 32 in (128, 256]:
the operators are requested in K-chunks of 32 during each GEMM) against the SIMT
contractions and the FP64 oracle, through the C ABI: the mixed-precision FPSA solve
with either engine reaches the oracle's converged flux (1e-9) with iteration counts
within one of each other, over several 128-column tiles with a ragged last tile and
several right-hand sides."""
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


@pytest.mark.parametrize("N,K,R,lap", [(256, 71, 3, "mpd"), (256, 40, 1, "wfd"), (160, 93, 2, "wfd")])
def test_streamed_tensor_contractions_match_simt_and_oracle(binding, N, K, R, lap):
    p = inputs.random_slab(K, N, N - 1, seed=900 + N + K, kernel="hg", thick=(1, 100), c=(0.5, 0.99))
    rng = np.random.default_rng(N + K)
    p["Q"] = np.concatenate([p["Q"][None]] + [rng.uniform(0, 1, (1,) + p["Q"].shape) for _ in range(R - 1)])
    ctx = binding.context_for(p, laplacian=lap, precision="mixed")
    phi_t, st_t = ctx.solve("fpsa", tol=1e-13, max_iterations=300, contraction="tensor", inner_iterations=4)
    phi_s, st_s = ctx.solve("fpsa", tol=1e-13, max_iterations=300, contraction="simt", inner_iterations=4)
    ctx.close()
    assert abs(st_t["outer_iterations"] - st_s["outer_iterations"]) <= 1, (st_t, st_s)
    for r in range(R):
        ref = oit.direct_solve(dict(p, Q=p["Q"][r]))
        assert relerr(phi_t[r], ref) < 1e-9, (r, relerr(phi_t[r], ref))
        assert relerr(phi_s[r], ref) < 1e-9


def test_tensor_request_outside_the_supported_orders(binding):
    p = inputs.random_slab(20, 8, 7, seed=950)  # N = 8: below the tensor-core tile widths
    ctx = binding.context_for(p, precision="mixed")
    with pytest.raises(binding.FpsaError) as e:
        ctx.solve("fpsa", contraction="tensor")
    assert e.value.code == binding.ENOTSUP
    ctx.close()
