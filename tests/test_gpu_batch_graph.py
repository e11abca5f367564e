"""Batched solves of slabs of different orders as one CUDA graph launch
(fpsa_solve_batch): every context's FP64 refinement loop is a device-side while node
of one graph, the contexts concurrent branches. Checked against the FP64 oracle's
discrete solution, against the same contexts solved one by one with fpsa_solve, and
for its argument checks and stopping rule.
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


def groups():
    """Four contexts of different orders: ragged instances, a reflective edge, two rhs."""
    g16 = [inputs.random_slab(K, 16, 15, seed=700 + K, kernel="hg", thick=(2, 300)) for K in (1, 37, 150)]
    g32 = [dict(inputs.random_slab(90, 32, 31, seed=710, kernel="srk", thick=(5, 200)), bc=("reflective", "vacuum"))]
    g64 = [inputs.random_slab(K, 64, 63, seed=720 + K, kernel="srk", thick=(2, 200), c=(0.8, 0.995)) for K in (3, 61)]
    g128 = [inputs.random_slab(40, 128, 127, seed=730, kernel="hg", thick=(5, 500), c=(0.8, 0.999), nrhs=2)]
    return [g16, g32, g64, g128]


def make(binding, probs, laplacian="wfd"):
    return binding.context_for(probs, laplacian=laplacian, precision="mixed")


def split(phi, probs, r=0):
    out, off = [], 0
    for p in probs:
        K = p["h"].size
        out.append(phi[r, off:off + K])
        off += K
    return out


def oracle_ref(p, r=0):
    if p["Q"].ndim == 4:
        p = dict(p, Q=p["Q"][r])
    return oit.direct_solve(p)


@pytest.mark.parametrize("inner", [0, 3])
@pytest.mark.parametrize("laplacian", ["wfd", "mpd"])
def test_graph_batch_matches_oracle_and_single_solves(binding, laplacian, inner):
    gs = groups()
    ctxs = [make(binding, g, laplacian) for g in gs]
    phis, sts = binding.solve_batch(ctxs, tol=1e-13, max_iterations=200, inner_iterations=inner)
    for g, phi, st in zip(gs, phis, sts):
        assert st["status"] == 0
        for r in range(phi.shape[0]):
            for p, got in zip(g, split(phi, g, r)):
                assert relerr(got, oracle_ref(p, r)) < TOL, (g[0]["N"], r, relerr(got, oracle_ref(p, r)))
    # the same contexts one by one: the same converged flux, at most one refinement step more
    for c, phi, st in zip(ctxs, phis, sts):
        one, st1 = c.solve("fpsa", tol=1e-13, max_iterations=200, inner_iterations=inner or 4)
        assert np.abs(one - phi).max() <= 1e-10 * np.abs(one[..., 0]).max()
        assert st1["outer_iterations"] <= st["outer_iterations"] <= st1["outer_iterations"] + 1, (st1, st)
    # the contexts stay usable: a second graph solve gives the same answer
    phis2, _ = binding.solve_batch(ctxs, tol=1e-13, max_iterations=200, inner_iterations=inner)
    for a, b in zip(phis, phis2):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a[..., 0]).max()
    for c in ctxs:
        c.close()


def test_graph_batch_si_and_adjoint_after(binding):
    p16 = inputs.random_slab(30, 16, 15, seed=740, kernel="hg", thick=(1, 20), c=(0.5, 0.9))
    p64 = inputs.random_slab(25, 64, 63, seed=741, kernel="srk", thick=(1, 20), c=(0.5, 0.9))
    ctxs = [make(binding, [p16]), make(binding, [p64])]
    phis, sts = binding.solve_batch(ctxs, method="si", tol=1e-13, max_iterations=400)
    for p, phi in zip((p16, p64), phis):
        assert relerr(phi[0], oit.direct_solve(p)) < TOL
    # a converged batch solve leaves each context ready for its adjoint
    for c in ctxs:
        c.adjoint(tol=1e-12)
        c.close()


def test_graph_batch_stopping_rule_and_checks(binding):
    p = inputs.random_slab(50, 32, 31, seed=750, kernel="srk", thick=(5, 300), c=(0.9, 0.999))
    c1, c2 = make(binding, [p]), make(binding, [p])
    # max_iterations refinement steps, then ENOTCONV with the last iterate
    phis, sts = binding.solve_batch([c1, c2], tol=1e-15, max_iterations=2, raise_on_notconv=False)
    assert all(s["status"] == binding.ENOTCONV and s["outer_iterations"] == 3 for s in sts), sts
    with pytest.raises(binding.FpsaError) as e:
        binding.solve_batch([c1, c1])
    assert e.value.code == binding.EINVAL
    with pytest.raises(binding.FpsaError) as e:
        binding.solve_batch([c1], method="gmres")
    assert e.value.code == binding.ENOTSUP
    c64 = binding.context_for(p, precision="fp64")
    with pytest.raises(binding.FpsaError) as e:
        binding.solve_batch([c1, c64])
    assert e.value.code == binding.ENOTSUP
    fresh = binding.Context([p["h"].size], p["h"], 32, 31, precision="mixed")
    with pytest.raises(binding.FpsaError) as e:
        binding.solve_batch([fresh])
    assert e.value.code == binding.ESTATE
    for c in (c1, c2, c64, fresh):
        c.close()


def test_batch_driver_graph_rounds(binding):
    from paper_1907_13013_gb300 import batch
    probs = inputs.batch_slabs(40, seed=2, K_range=(20, 140))
    solver = batch.BatchSolver(probs, precision="mixed", laplacian="wfd", budget_bytes=48 << 20, graph=True)
    rounds = solver.rounds()
    assert len(rounds) > 1 and len({w[0] for w in rounds[0]}) == 4  # every N in the first graph, several rounds
    phis, stats = solver.solve(tol=1e-12, max_iterations=200)
    assert sum(s["instances"] for s in stats) == len(probs) and all(s["status"] == 0 for s in stats)
    rng = np.random.default_rng(3)
    for i in rng.choice(len(probs), 8, replace=False):
        assert relerr(phis[i], oit.direct_solve(probs[i])) < TOL, (i, probs[i]["N"])


def test_graph_batch_with_tensor_core_residual(binding):
    """The refinement residual on the tensor cores (exact digit-slice products) inside the
    graph's while loops: the same fluxes as the FP64-core residual and the oracle's."""
    gs = [[inputs.random_slab(K, 32, 31, seed=760 + K, kernel="srk", thick=(2, 300), c=(0.9, 0.999))
           for K in (5, 77)],
          [inputs.random_slab(120, 64, 63, seed=770, kernel="srk", thick=(5, 500), c=(0.99, 0.9999))],
          [dict(inputs.random_slab(33, 128, 127, seed=780, kernel="hg", thick=(2, 200), c=(0.8, 0.999)),
                bc=("reflective", "vacuum"))]]
    out = {}
    for engine in (2, 1):
        ctxs = [make(binding, g) for g in gs]
        for c in ctxs:
            c.set_tuning({"residual_engine": engine})
            assert c.get_tuning()["residual_engine"] == engine
        out[engine] = binding.solve_batch(ctxs, tol=1e-13, max_iterations=200, inner_iterations=4)
        for c in ctxs:
            c.close()
    (phis_t, sts_t), (phis_f, sts_f) = out[2], out[1]
    for g, pt, pf, st, sf in zip(gs, phis_t, phis_f, sts_t, sts_f):
        assert st["status"] == 0 and sf["status"] == 0
        assert st["outer_iterations"] == sf["outer_iterations"], (st, sf)
        assert np.abs(pt - pf).max() <= 1e-11 * np.abs(pf[..., 0]).max()
        for p, got in zip(g, split(pt, g)):
            assert relerr(got, oracle_ref(p)) < TOL, (g[0]["N"], relerr(got, oracle_ref(p)))
