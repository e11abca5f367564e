"""Launch shapes and the autotuner, through the C ABI. A shape (cells per lane of the
transport sweep, resident blocks per SM and row slices of the cooperative BCR solve)
changes how the iteration is laid out, never what it computes: every shape must give
the FP64 oracle's solution, and the same iterates as the library's own shape up to
rounding order. The autotuner must keep one of its candidates and leave a context
that solves to the oracle's flux; the batch driver reuses its choices from a JSON
cache."""
import json
import os

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


def relerr(phi, ref):
    return np.abs(phi - ref).max() / np.abs(ref[..., 0]).max()


def split(phi, probs, r=0):
    out, off = [], 0
    for p in probs:
        K = p["h"].size
        out.append(phi[r, off:off + K])
        off += K
    return out


def golden_phi0(name):
    """Stored oracle flux phi_0 (one value per line after '#' comments)."""
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        return np.array([float(x) for x in f if not x.startswith("#")])


CASES = {
    # one slab, one right-hand side: the BCR solve takes its coarse step
    "single_coarse": lambda: [dict(inputs.random_slab(700, 64, 63, seed=500, kernel="srk", thick=(2, 300),
                                                      c=(0.8, 0.999)), bc="vacuum")],
    # three slabs, three right-hand sides (two rhs chunks), one reflective edge
    "batch_rhs": lambda: [dict(inputs.random_slab(K, 32, 31, seed=510 + i, kernel="hg", c=(0.7, 0.99), nrhs=3),
                               bc=bc)
                          for i, (K, bc) in enumerate([(150, "vacuum"), (61, ("reflective", "vacuum")),
                                                       (233, "vacuum")])],
    # many sweep segments (2000 cells, the smallest cells per lane)
    "long_slab": lambda: [dict(inputs.random_slab(2000, 16, 15, seed=520, kernel="hg", thick=(1, 100),
                                                  c=(0.6, 0.99)), bc="vacuum")],
}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_every_shape_gives_the_oracle_solution(binding, case, precision):
    probs = CASES[case]()
    R = probs[0]["Q"].shape[0] if probs[0]["Q"].ndim == 4 else 1
    refs = [[oit.direct_solve(dict(p, Q=p["Q"][r] if p["Q"].ndim == 4 else p["Q"])) for r in range(R)]
            for p in probs]
    ctx = binding.context_for(probs, laplacian="wfd", precision=precision)
    lib_shape = ctx.get_tuning()
    cmin = lib_shape["sweep_cells_per_thread"]
    assert cmin >= 4 and 1 <= lib_shape["solve_blocks_per_sm"] <= 4 and lib_shape["solve_max_slices"] == 4
    base, _ = ctx.solve("fpsa", tol=1e-13, max_iterations=500)
    kmax = max(p["h"].size for p in probs)
    cpts = sorted({cmin, 2 * cmin, 8 * cmin, -(-kmax // 8)})  # the last: one segment per slab
    seen = set()
    for b in (1, 2, 3, 4):
        for s in (1, 2, 4):
            for c in cpts:
                ctx.set_tuning({"sweep_cells_per_thread": c, "solve_blocks_per_sm": b, "solve_max_slices": s})
                t = ctx.get_tuning()
                assert t["sweep_cells_per_thread"] == max(c, cmin) and t["solve_max_slices"] == s
                assert 1 <= t["solve_blocks_per_sm"] <= b
                key = tuple(sorted(t.items()))
                if key in seen:
                    continue
                seen.add(key)
                phi, st = ctx.solve("fpsa", tol=1e-13, max_iterations=500)
                assert st["status"] == 0
                if precision == "fp64":
                    assert np.abs(phi - base).max() / np.abs(base[..., 0]).max() < 1e-11, (t, st)
                for r in range(R):
                    for got, ref in zip(split(phi, probs, r), [x[r] for x in refs]):
                        assert relerr(got, ref) < TOL, (t, r, relerr(got, ref))
    ctx.set_tuning(None)
    assert ctx.get_tuning() == lib_shape
    ctx.close()


def test_set_tuning_validates(binding):
    p = inputs.random_slab(40, 16, 15, seed=530)
    ctx = binding.context_for(p)
    before = ctx.get_tuning()
    for bad in ({"solve_max_slices": 3}, {"solve_blocks_per_sm": 5}, {"solve_blocks_per_sm": -1},
                {"sweep_cells_per_thread": -2}, {"sweep_cells_per_thread": (1 << 20) + 1}):
        with pytest.raises(binding.FpsaError) as e:
            ctx.set_tuning(bad)
        assert e.value.code == binding.EINVAL
        assert ctx.get_tuning() == before
    ctx.set_tuning({"sweep_cells_per_thread": 1})  # below the smallest: raised to it
    assert ctx.get_tuning() == before
    ctx.close()


def test_autotune_needs_cross_sections(binding):
    ctx = binding.Context([30], np.full(30, 1 / 30), 16, 15)
    with pytest.raises(binding.FpsaError) as e:
        ctx.autotune()
    assert e.value.code == binding.ESTATE
    ctx.close()


@pytest.mark.parametrize("lap", ["mpd", "wfd"])
def test_autotune_on_the_precision_workload(binding, lap):
    # the benchmark workload (2000 cells, S64, screened Rutherford to L = 63), mixed
    # precision: the chosen shape is one of the candidates, is kept, and solves to the
    # stored oracle flux; the adjoint still runs from the kept moments
    p = inputs.precision_srk_slab()
    ref = golden_phi0("precision_srk_slab_fpsa_%s_phi0.txt" % lap)
    ctx = binding.context_for(p, laplacian=lap, precision="mixed")
    lib_shape = ctx.get_tuning()
    shapes, ms = ctx.autotune(tol=1e-10, max_iterations=50, repeats=2)
    assert ms > 0 and np.isfinite(ms)
    assert ctx.get_tuning() == shapes
    c = lib_shape["sweep_cells_per_thread"]
    assert shapes["sweep_cells_per_thread"] in (c, 2 * c, 4 * c, 8 * c)
    assert 1 <= shapes["solve_blocks_per_sm"] <= lib_shape["solve_blocks_per_sm"]
    assert shapes["solve_max_slices"] in (1, 2, 4)
    gt, gs, J, _ = ctx.adjoint()
    assert np.all(np.isfinite(gt)) and np.all(np.isfinite(gs))
    phi, st = ctx.solve("fpsa", tol=1e-10, max_iterations=50)
    err = np.abs(phi[0, :, :, 0].ravel() - ref).max() / np.abs(ref).max()
    assert err < TOL, (err, shapes, st)
    ctx.close()


def test_batch_driver_tuning_cache(binding, tmp_path):
    from paper_1907_13013_gb300 import batch
    probs = inputs.batch_slabs(12, seed=3, K_range=(20, 120))
    path = str(tmp_path / "shapes.json")
    cache = batch.TuningCache(path)
    phis, stats = batch.BatchSolver(probs, tuning=cache).solve(tol=1e-12, max_iterations=200)
    assert "search" in {s["tuning_source"] for s in stats}
    with open(path) as f:
        saved = json.load(f)
    assert 1 <= len(saved) <= len(stats)
    assert all(e["ms"] > 0 and set(e["shapes"]) == {"sweep_cells_per_thread", "solve_blocks_per_sm",
                                                     "solve_max_slices", "factor_engine", "solve_engine",
                                                     "residual_engine"}
               for e in saved.values())
    phis2, stats2 = batch.BatchSolver(probs, tuning=batch.TuningCache(path)).solve(tol=1e-12, max_iterations=200)
    assert {s["tuning_source"] for s in stats2} == {"cache"}
    for s in stats2:
        assert s["tuning"]["solve_max_slices"] in (1, 2, 4)
    for i in np.random.default_rng(3).choice(len(probs), 5, replace=False):
        p = probs[i]
        ref = oit.direct_solve(p)
        assert relerr(phis[i], ref) < TOL and relerr(phis2[i], ref) < TOL, (i, p["N"], p["h"].size)
