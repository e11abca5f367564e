"""Error paths of the C ABI on the GPU, made to fire on ordinary inputs by shortened limits
(fpsa_set_limits), through the C ABI.

A BCR dataflow wait that gives up after one poll makes fpsa_set_xs (the dataflow
factorization: items of the narrow reduction levels run at the same time as the
items they wait for) and fpsa_solve (the dataflow solve: the narrow levels and the
coarse step wait on each other's pushes) return FPSA_ETIMEOUT; a pivot-growth
limit below every block's growth makes fpsa_set_xs return FPSA_EPIVOT. A wait
that gives up records the failure and its kernel runs on to completion, so
nothing hangs or faults; afterwards the same context, with the default limits
restored, solves to the oracle's answer.
"""
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


@pytest.fixture(scope="module")
def slab():
    p = inputs.random_slab(2000, 16, 15, seed=777, kernel="srk", thick=(2, 200), c=(0.7, 0.995))
    return p, oit.direct_solve(p)


def fresh_context(binding, p, precision):
    return binding.Context([p["h"].size], p["h"], p["N"], p["L"], laplacian="wfd", precision=precision)


def set_xs(ctx, p):
    ctx.set_xs(p["sigma_t"], p["sigma_s"], p["Q"][None])


def check_solution(ctx, ref):
    phi, st = ctx.solve("fpsa", tol=1e-13, max_iterations=500)
    err = np.abs(phi[0] - ref).max() / np.abs(ref[..., 0]).max()
    assert err < 1e-9, err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_factorization_wait_runs_out_then_context_recovers(binding, slab, precision):
    p, ref = slab
    ctx = fresh_context(binding, p, precision)
    ctx.set_limits(wait_polls=1)
    with pytest.raises(binding.FpsaError) as e:
        set_xs(ctx, p)
    assert e.value.code == binding.ETIMEOUT
    with pytest.raises(binding.FpsaError) as e:  # no solve on factors that did not complete
        ctx.solve("fpsa")
    assert e.value.code == binding.ESTATE
    ctx.set_limits()
    set_xs(ctx, p)
    check_solution(ctx, ref)
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_wait_runs_out_then_context_recovers(binding, slab, precision):
    p, ref = slab
    ctx = fresh_context(binding, p, precision)
    set_xs(ctx, p)
    ctx.set_limits(wait_polls=1)
    with pytest.raises(binding.FpsaError) as e:
        ctx.solve("fpsa", tol=1e-13, max_iterations=500)
    assert e.value.code == binding.ETIMEOUT
    ctx.set_limits()
    check_solution(ctx, ref)  # the factors were untouched; the solve's counters start afresh
    ctx.close()


def test_growth_limit_reports_epivot_then_context_recovers(binding, slab):
    p, ref = slab
    ctx = fresh_context(binding, p, "mixed")
    ctx.set_limits(growth_limit=1e-9)  # below max|A| max|A^-1| >= 1/(2N) of any block
    with pytest.raises(binding.FpsaError) as e:
        set_xs(ctx, p)
    assert e.value.code == binding.EPIVOT
    ctx.set_limits()
    set_xs(ctx, p)
    check_solution(ctx, ref)
    ctx.close()


def test_limits_reject_negative_values(binding, slab):
    p, _ = slab
    ctx = fresh_context(binding, p, "fp64")
    for args in ((-1, 0.0), (0, -1.0)):
        with pytest.raises(binding.FpsaError) as e:
            ctx.set_limits(*args)
        assert e.value.code == binding.EINVAL
    ctx.close()


def test_tensor_core_solve_wait_runs_out_then_context_recovers(binding):
    # 16 right-hand sides, 2N = 128: the tensor-core BCR solve, whose units take their
    # work from a queue and give up their waits at once when another has recorded one
    p = inputs.random_slab(300, 64, 63, seed=778, kernel="srk", thick=(2, 200), c=(0.7, 0.995), nrhs=16)
    ctx = binding.context_for(p, laplacian="wfd", precision="mixed")
    assert ctx.get_tuning()["solve_engine"] == 2
    ctx.set_limits(wait_polls=1)
    with pytest.raises(binding.FpsaError) as e:
        ctx.solve("fpsa", tol=1e-13, max_iterations=500)
    assert e.value.code == binding.ETIMEOUT
    ctx.set_limits()
    phi, st = ctx.solve("fpsa", tol=1e-13, max_iterations=500)
    ctx.close()
    for r in (0, 15):
        ref = oit.direct_solve(dict(p, Q=p["Q"][r]))
        err = np.abs(phi[r] - ref).max() / np.abs(ref[..., 0]).max()
        assert err < 1e-9, (r, err)
