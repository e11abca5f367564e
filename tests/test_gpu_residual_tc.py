"""The FP64 refinement residual with its contractions on the tensor cores (exact digit-slice
products, FP64 recombination) against the FP64-core residual and the FP64 oracle, through
the C ABI. The converged flux of a mixed-precision solve is limited by the accuracy of this
residual amplified by about 1 / (1 - c) (the fixed point of (L - S) psi = q): on the
precision SRK slab (c = 0.99999) a residual accurate to 1e-12 instead of FP64's 1e-16
would leave errors near 1e-7, so agreement with the oracle to 1e-9 there checks that the
tensor-core residual is FP64-grade. Both engines take the same refinement steps.
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


def solve(binding, probs, engine, method="fpsa", **kw):
    ctx = binding.context_for(probs, laplacian=kw.pop("laplacian", "wfd"), precision="mixed")
    ctx.set_tuning({"residual_engine": engine})
    assert ctx.get_tuning()["residual_engine"] == engine
    extra = {"restart": 30} if method == "gmres" else {"inner_iterations": 4}
    phi, st = ctx.solve(method, tol=1e-13, max_iterations=200, **extra, **kw)
    ctx.close()
    return phi, st


CASES = {
    "n32_batch": lambda: [inputs.random_slab(K, 32, 31, seed=800 + K, kernel="srk", thick=(2, 300), c=(0.9, 0.999))
                          for K in (1, 17, 90)],
    "n64_srk": lambda: [inputs.random_slab(150, 64, 63, seed=810, kernel="srk", thick=(5, 500), c=(0.99, 0.99999))],
    "n64_L_below": lambda: [inputs.random_slab(70, 64, 20, seed=811, kernel="hg", thick=(5, 200), c=(0.9, 0.999))],
    "n128_rhs": lambda: [inputs.random_slab(60, 128, 127, seed=820, kernel="hg", thick=(5, 500), c=(0.9, 0.9999),
                                            nrhs=3)],
    "n160_reflective": lambda: [dict(inputs.random_slab(33, 160, 159, seed=830, kernel="srk", thick=(2, 200),
                                                        c=(0.8, 0.999)), bc=("reflective", "vacuum"))],
    "n256": lambda: [inputs.random_slab(21, 256, 255, seed=840, kernel="hg", thick=(5, 500), c=(0.9, 0.9999))],
}


def refs(p):
    if p["Q"].ndim == 4:
        return [oit.direct_solve(dict(p, Q=p["Q"][r])) for r in range(p["Q"].shape[0])]
    return [oit.direct_solve(p)]


@pytest.mark.parametrize("case", sorted(CASES))
def test_tensor_core_residual_matches_fp64_residual_and_oracle(binding, case):
    probs = CASES[case]()
    phi_t, st_t = solve(binding, probs, 2)
    phi_f, st_f = solve(binding, probs, 1)
    assert st_t["status"] == 0 and st_f["status"] == 0
    assert st_t["outer_iterations"] == st_f["outer_iterations"], (st_t, st_f)
    assert np.abs(phi_t - phi_f).max() <= 1e-11 * np.abs(phi_f[..., 0]).max()
    off = 0
    for p in probs:
        K = p["h"].size
        for r, ref in enumerate(refs(p)):
            assert relerr(phi_t[r, off:off + K], ref) < TOL, (case, r, relerr(phi_t[r, off:off + K], ref))
        off += K


def test_tensor_core_residual_gmres_ir(binding):
    p = inputs.random_slab(80, 64, 63, seed=850, kernel="srk", thick=(5, 300), c=(0.9, 0.999))
    phi_t, st_t = solve(binding, [p], 2, method="gmres")
    phi_f, st_f = solve(binding, [p], 1, method="gmres")
    assert relerr(phi_t[0], oit.direct_solve(p)) < TOL
    assert np.abs(phi_t - phi_f).max() <= 1e-11 * np.abs(phi_f[..., 0]).max()


@pytest.mark.parametrize("lap", ["wfd", "mpd"])
def test_precision_slab_full_size_both_residual_engines(binding, lap):
    p = inputs.precision_srk_slab()
    ref = np.loadtxt(__file__.replace("test_gpu_residual_tc.py", "golden/precision_srk_slab_fpsa_%s_phi0.txt" % lap))
    for engine in (2, 1):
        phi, st = solve(binding, [p], engine, laplacian=lap)
        got = phi[0, :, :, 0].reshape(-1)
        err = np.abs(got - ref.reshape(-1)).max() / np.abs(ref).max()
        assert err < 1e-10, (engine, err)


def test_residual_engine_request_is_validated(binding):
    p = inputs.random_slab(20, 16, 15, seed=860)
    ctx = binding.context_for(p, precision="mixed")  # N = 16: not a multiple of 32
    assert ctx.get_tuning()["residual_engine"] == 1
    with pytest.raises(binding.FpsaError) as e:
        ctx.set_tuning({"residual_engine": 2})
    assert e.value.code == binding.ENOTSUP
    ctx.close()
    p = inputs.random_slab(20, 64, 63, seed=861)
    ctx = binding.context_for(p, precision="fp64")
    with pytest.raises(binding.FpsaError) as e:
        ctx.set_tuning({"residual_engine": 2})
    assert e.value.code == binding.ENOTSUP
    with pytest.raises(binding.FpsaError) as e:
        ctx.set_tuning({"residual_engine": 3})
    assert e.value.code == binding.EINVAL
    ctx.close()
