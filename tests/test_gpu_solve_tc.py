"""The tensor-core BCR solve (each unit one split-BF16 tcgen05 GEMM of a cell's A^{-1} by a
tile of up to 64 right-hand sides) against the dataflow solve on the FP32 cores and the FP64
oracle, through the C ABI: the mixed-precision FPSA-SI and FPSA-GMRES solves with either
solve engine reach the oracle's converged flux (1e-9, sampled right-hand sides of every
instance) and each other's (every right-hand side), with iteration counts within one of each
other. Cases: 2N = 128, 256 and 512; a tile padded with zero right-hand sides (R = 20, tiles
of 32); two tiles, the second ragged (R = 70: 64 + 6); several instances, one of a single cell
(a root without neighbours)."""
import numpy as np
import pytest

from oracle import iterations as oit
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


def relerr(a, b):
    return np.abs(a - b).max() / np.abs(b[..., 0]).max()


CASES = [
    (64, [37], 16, "fpsa", "wfd"),
    (128, [45], 20, "fpsa", "mpd"),
    (256, [23], 64, "fpsa", "wfd"),
    (64, [15, 1, 30], 70, "fpsa", "wfd"),
    (128, [29], 16, "gmres", "wfd"),
]


@pytest.mark.parametrize("N,Ks,R,method,lap", CASES)
def test_tensor_core_solve_matches_dataflow_solve_and_oracle(binding, N, Ks, R, method, lap):
    probs = [inputs.random_slab(K, N, N - 1, seed=1200 + N + K + R + b, kernel="hg", thick=(1, 100),
                                c=(0.5, 0.99), nrhs=R) for b, K in enumerate(Ks)]
    kw = {"restart": 30} if method == "gmres" else {"inner_iterations": 4}  # fixed: step-for-step comparison
    ctx = binding.context_for(probs, laplacian=lap, precision="mixed")
    assert ctx.get_tuning()["solve_engine"] == 2
    phi_t, st_t = ctx.solve(method, tol=1e-13, max_iterations=300, **kw)
    ctx.set_tuning({"solve_engine": 1})
    assert ctx.get_tuning()["solve_engine"] == 1
    phi_s, st_s = ctx.solve(method, tol=1e-13, max_iterations=300, **kw)
    ctx.close()
    assert abs(st_t["outer_iterations"] - st_s["outer_iterations"]) <= 1, (st_t, st_s)
    off = np.concatenate([[0], np.cumsum(Ks)])
    for b, p in enumerate(probs):
        sl = slice(off[b], off[b + 1])
        for r in range(R):
            assert relerr(phi_t[r, sl], phi_s[r, sl]) < TOL, (b, r, relerr(phi_t[r, sl], phi_s[r, sl]))
        for r in sorted({0, R // 2, R - 1}):
            ref = oit.direct_solve(dict(p, Q=p["Q"][r]))
            assert relerr(phi_t[r, sl], ref) < TOL, (b, r, relerr(phi_t[r, sl], ref))


def test_tensor_core_solve_outside_its_shapes(binding):
    # FP64 factors, too few right-hand sides, 2N not a multiple of 128: the dataflow solve only
    for N, R, prec in ((64, 16, "fp64"), (64, 8, "mixed"), (32, 16, "mixed")):
        p = inputs.random_slab(12, N, N - 1, seed=1300 + N + R, nrhs=R)
        ctx = binding.context_for(p, precision=prec)
        assert ctx.get_tuning()["solve_engine"] == 1
        with pytest.raises(binding.FpsaError) as e:
            ctx.set_tuning({"solve_engine": 2})
        assert e.value.code == binding.ENOTSUP
        ctx.close()
    p = inputs.random_slab(12, 64, 63, seed=1310, nrhs=16)
    ctx = binding.context_for(p, precision="mixed")
    with pytest.raises(binding.FpsaError) as e:
        ctx.set_tuning({"solve_engine": 3})
    assert e.value.code == binding.EINVAL
    ctx.close()
