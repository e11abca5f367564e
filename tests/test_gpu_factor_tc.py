"""The BCR factorization with tensor-core inversions (FP32 factors; 2N = 128: blocked
Gauss-Jordan with tcgen05 trailing updates in split BF16; 2N = 256 and 512: the
recursive block inversion's GEMMs as tcgen05 split-BF16 products) against the SIMT
factorization and the FP64 oracle, through the C ABI.

The factors are the FP correction's preconditioner inside the mixed-precision
refinement, so both engines must give the oracle's converged flux (1e-9) with
iteration counts within one of each other, on single slabs (the coarse step of
the solve on), ragged batches, reflective edges and the precision SRK slab at
full size; the pivot growth both report agrees to the rounding of the updates.
"""
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


def solve_with(binding, probs, engine, laplacian):
    ctx = binding.Context([p["h"].size for p in probs], np.concatenate([p["h"] for p in probs]), probs[0]["N"],
                          probs[0]["L"], laplacian=laplacian, precision="mixed",
                          bc=[p.get("bc", "vacuum") for p in probs])
    ctx.set_tuning({"factor_engine": engine})
    assert ctx.get_tuning()["factor_engine"] == engine
    ctx.set_xs(np.concatenate([p["sigma_t"] for p in probs]), np.concatenate([p["sigma_s"] for p in probs]),
               np.concatenate([p["Q"] for p in probs])[None])
    # a fixed inner count: the engines are compared step for step
    phi, st = ctx.solve("fpsa", tol=1e-13, max_iterations=500, inner_iterations=4)
    ctx.close()
    return phi[0], st


CASES = {
    "single_srk": lambda: [inputs.random_slab(1000, 64, 63, seed=610, kernel="srk", thick=(2, 200),
                                              c=(0.7, 0.995))],
    "single_odd_K": lambda: [inputs.random_slab(333, 64, 40, seed=611, kernel="hg", thick=(1, 100),
                                                c=(0.5, 0.99))],
    "tiny": lambda: [inputs.random_slab(3, 64, 63, seed=612, kernel="hg")],
    "batch_ragged": lambda: [inputs.random_slab(K, 64, 63, seed=620 + K, kernel="srk" if K % 2 else "hg")
                             for K in (1, 2, 7, 64, 129, 500)],
    "reflective": lambda: [dict(inputs.random_slab(257, 64, 63, seed=630, kernel="srk", thick=(2, 200),
                                                   c=(0.7, 0.995)), bc=("reflective", "vacuum"))],
}


@pytest.mark.parametrize("laplacian", ["wfd", "mpd"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_tensor_core_factorization_matches_simt_and_oracle(binding, case, laplacian):
    probs = CASES[case]()
    phi_tc, st_tc = solve_with(binding, probs, 2, laplacian)
    phi_si, st_si = solve_with(binding, probs, 1, laplacian)
    assert st_tc["status"] == 0 and st_si["status"] == 0
    assert abs(st_tc["outer_iterations"] - st_si["outer_iterations"]) <= 1, (st_tc, st_si)
    g_tc, g_si = st_tc["pivot_growth"], st_si["pivot_growth"]
    assert g_tc > 0 and abs(g_tc - g_si) <= 1e-3 * g_si, (g_tc, g_si)
    off = 0
    for p in probs:
        K = p["h"].size
        ref = oit.direct_solve(p)
        assert relerr(phi_tc[off:off + K], ref) < TOL, (case, relerr(phi_tc[off:off + K], ref))
        assert relerr(phi_si[off:off + K], ref) < TOL
        off += K


# 2N = 256 and 512: the recursive block inversion (128 x 128 leaves by Gauss-Jordan)
# with its block GEMMs on the tensor cores (engine 2) or the FP32 cores (engine 1)
LARGE_CASES = {
    "n128_single": lambda: [inputs.random_slab(301, 128, 127, seed=650, kernel="srk", thick=(5, 500),
                                               c=(0.8, 0.999))],
    "n128_batch": lambda: [inputs.random_slab(K, 128, 100, seed=651 + K, kernel="hg", thick=(2, 200),
                                              c=(0.6, 0.995)) for K in (1, 5, 130)],
    "n256_single": lambda: [inputs.random_slab(61, 256, 255, seed=660, kernel="hg", thick=(5, 500),
                                               c=(0.8, 0.999))],
    "n256_reflective": lambda: [dict(inputs.random_slab(33, 256, 200, seed=661, kernel="srk", thick=(2, 200),
                                                        c=(0.7, 0.995)), bc=("vacuum", "reflective"))],
}


@pytest.mark.parametrize("case", sorted(LARGE_CASES))
def test_tensor_core_block_gemms_match_simt_and_oracle(binding, case):
    probs = LARGE_CASES[case]()
    phi_tc, st_tc = solve_with(binding, probs, 2, "mpd")
    phi_si, st_si = solve_with(binding, probs, 1, "mpd")
    assert st_tc["status"] == 0 and st_si["status"] == 0
    assert abs(st_tc["outer_iterations"] - st_si["outer_iterations"]) <= 1, (st_tc, st_si)
    # the growth max|A| max|A^{-1}| of both engines: each split-BF16 product carries about
    # 2^-15 of relative error, amplified through the Schur complements of two levels of
    # recursion (2N = 512) to a few 1e-3 of the largest inverse entry
    g_tc, g_si = st_tc["pivot_growth"], st_si["pivot_growth"]
    assert g_tc > 0 and abs(g_tc - g_si) <= 1e-2 * g_si, (g_tc, g_si)
    off = 0
    for p in probs:
        K = p["h"].size
        ref = oit.direct_solve(p)
        assert relerr(phi_tc[off:off + K], ref) < TOL, (case, relerr(phi_tc[off:off + K], ref))
        assert relerr(phi_si[off:off + K], ref) < TOL
        off += K


def test_engine_request_is_validated(binding):
    p = inputs.random_slab(40, 32, 31, seed=640)
    ctx = binding.context_for(p, precision="mixed")  # 2N = 64: the tensor-core engine does not apply
    with pytest.raises(binding.FpsaError) as e:
        ctx.set_tuning({"factor_engine": 2})
    assert e.value.code == binding.ENOTSUP
    assert ctx.get_tuning()["factor_engine"] == 1
    ctx.close()
    p = inputs.random_slab(40, 64, 63, seed=641)
    ctx = binding.context_for(p, precision="fp64")  # FP64 factors stay on the SIMT engine
    with pytest.raises(binding.FpsaError) as e:
        ctx.set_tuning({"factor_engine": 2})
    assert e.value.code == binding.ENOTSUP
    for bad in (-1, 3):
        with pytest.raises(binding.FpsaError) as e:
            ctx.set_tuning({"factor_engine": bad})
        assert e.value.code == binding.EINVAL
    ctx.close()


def test_precision_slab_full_size_both_engines(binding):
    p = inputs.precision_srk_slab()
    ref = np.loadtxt(__file__.replace("test_gpu_factor_tc.py", "golden/precision_srk_slab_fpsa_wfd_phi0.txt"))
    phi_tc, st_tc = solve_with(binding, [p], 2, "wfd")
    phi_si, st_si = solve_with(binding, [p], 1, "wfd")
    for phi in (phi_tc, phi_si):
        got = phi[..., 0].reshape(-1)
        assert np.abs(got - ref.reshape(-1)).max() / np.abs(ref).max() < TOL
    assert abs(st_tc["iterations"] - st_si["iterations"]) <= 1, (st_tc, st_si)
