"""The coarse step of the BCR solve (a single slab with one right-hand side replaces
the reduction's top levels and root by the dense inverse of the coarse system) gives
the solution of the full reduction: the same slab solved alone (coarse step on) and
as one instance of a two-slab batch (coarse step off: more than one instance) agree
to rounding, and both agree with the FP64 oracle. Through the C ABI."""
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


@pytest.mark.parametrize("K,N,bc", [(300, 16, "vacuum"), (257, 32, ("reflective", "vacuum")), (1000, 64, "reflective")])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_coarse_step_matches_full_reduction(binding, K, N, bc, precision):
    p = inputs.random_slab(K, N, N - 1, seed=400 + K, kernel="srk", thick=(2, 200), c=(0.7, 0.995))
    p["bc"] = bc
    other = inputs.random_slab(17, N, N - 1, seed=401, kernel="hg")
    other["bc"] = "vacuum"
    alone = binding.context_for(p, laplacian="wfd", precision=precision)
    phi_a, st_a = alone.solve("fpsa", tol=1e-13, max_iterations=500)
    batch = binding.context_for([p, other], laplacian="wfd", precision=precision)
    phi_b, st_b = batch.solve("fpsa", tol=1e-13, max_iterations=500)
    ref = oit.direct_solve(p)
    scale = np.abs(ref[..., 0]).max()
    diff = np.abs(phi_a[0] - phi_b[0, :K]).max() / scale
    assert diff < (1e-11 if precision == "fp64" else 1e-9), diff
    assert np.abs(phi_a[0] - ref).max() / scale < 1e-9
    alone.close()
    batch.close()
