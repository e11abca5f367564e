"""CPU-side checks of the C-ABI library: it builds, loads, exports every symbol the
header declares, and rejects bad descriptors without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1907_13013_gb300 import binding
    return binding.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fpsa.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*(fpsa_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("fpsa_create", "fpsa_set_xs", "fpsa_solve", "fpsa_destroy", "fpsa_strerror", "fpsa_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_strerror_texts(lib):
    from paper_1907_13013_gb300 import binding
    for code in (binding.OK, binding.EINVAL, binding.ENOTCONV, binding.EPIVOT, binding.ENOTSUP):
        assert lib.fpsa_strerror(code)
    assert isinstance(lib.fpsa_last_error(None), bytes)


def test_create_rejects_bad_descriptors_before_any_cuda_call(lib):
    from paper_1907_13013_gb300 import binding
    K = np.array([4], dtype=np.int32)
    h = np.full(4, 0.25)

    def create(**kw):
        args = dict(n_instances=1, n_ordinates=8, n_moments=8, n_rhs=1, laplacian=0, precision=0, bc=None)
        args.update(kw)
        bc = None if args["bc"] is None else np.asarray(args["bc"], dtype=np.int32)
        d = binding.FpsaDesc(args["n_instances"], args["n_ordinates"], args["n_moments"], args["n_rhs"],
                             K.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             h.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             args["laplacian"], args["precision"], 0, None,
                             None if bc is None else bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        out = ctypes.c_void_p()
        return lib.fpsa_create(ctypes.byref(out), ctypes.byref(d)), out

    for bad in (dict(n_ordinates=7), dict(n_ordinates=0), dict(n_moments=9), dict(n_moments=0),
                dict(n_rhs=0), dict(n_instances=0), dict(laplacian=5), dict(precision=7),
                dict(bc=[0, 2]), dict(bc=[-1, 0])):
        rc, out = create(**bad)
        assert rc == binding.EINVAL and not out.value, bad
    rc, out = create(n_ordinates=2 * binding.MAX_ORDINATES, n_moments=2)
    assert rc == binding.ENOTSUP and not out.value


def test_batch_wave_planning():
    # host logic of the batch driver: grouping by (N, L) and memory-bounded waves
    from paper_1907_13013_gb300 import batch, inputs
    probs = inputs.batch_slabs(40, seed=2, K_range=(100, 5000))
    budget = 2 << 30
    waves = batch.plan_waves(probs, budget, "mixed")
    seen = sorted(i for _, _, idx in waves for i in idx)
    assert seen == list(range(len(probs)))
    for N, L, idx in waves:
        assert all(probs[i]["N"] == N and probs[i]["L"] == L for i in idx)
        total = sum(batch.factor_bytes(probs[i]["h"].size, N, "mixed") for i in idx)
        assert total <= budget or len(idx) == 1


def test_boundary_condition_marshalling():
    from paper_1907_13013_gb300 import binding
    assert binding._bc_array(None, 3) is None
    assert binding._bc_array("vacuum", 2) is None
    a = binding._bc_array(["vacuum", ("reflective", "vacuum"), "reflective"], 3)
    assert a.tolist() == [[0, 0], [1, 0], [1, 1]]
    with pytest.raises(ValueError):
        binding._bc_array(["vacuum"], 2)
    with pytest.raises(KeyError):
        binding._bc_array("periodic", 1)


def test_batch_graph_rounds():
    # graph mode of the batch driver: every wave is solved exactly once, rounds hold at
    # most max_streams waves, the first round one wave of every (N, L) group, a group's
    # waves in their planned order, and only the last round is less than full
    from paper_1907_13013_gb300 import batch, inputs
    probs = inputs.batch_slabs(60, seed=4, K_range=(100, 5000))
    solver = batch.BatchSolver(probs, precision="mixed", laplacian="wfd", budget_bytes=1 << 30, graph=True)
    rounds = solver.rounds()
    flat = [w for rnd in rounds for w in rnd]
    assert sorted(map(id, flat)) == sorted(map(id, solver.waves))
    assert all(len(rnd) <= solver.max_streams for rnd in rounds)
    assert all(len(rnd) == solver.max_streams for rnd in rounds[:-1])
    groups = {(p["N"], p["L"]) for p in probs}
    assert {(N, L) for N, L, _ in rounds[0]} == groups
    for key in groups:
        mine = [w for w in flat if (w[0], w[1]) == key]
        planned = [w for w in solver.waves if (w[0], w[1]) == key]
        assert [id(w) for w in mine] == [id(w) for w in planned]
    assert solver._round_bytes(rounds[0]) == sum(
        batch.factor_bytes(sum(probs[i]["h"].size for i in w[2]), w[0], "mixed") for w in rounds[0])
    with pytest.raises(ValueError):
        batch.BatchSolver(probs, precision="fp64", graph=True)


def test_batch_solve_rejects_empty_and_null_arguments(lib):
    # argument checks that precede any CUDA call (no GPU needed)
    import ctypes as ct
    from paper_1907_13013_gb300 import binding
    binding.load()
    assert lib.fpsa_solve_batch(None, 1, None, None, 0, None) == binding.EINVAL
    handles = (ct.c_void_p * 1)(None)
    assert lib.fpsa_solve_batch(handles, 0, None, None, 0, None) == binding.EINVAL
    assert lib.fpsa_solve_batch(handles, 1, None, None, 0, None) == binding.EINVAL


def test_limits_entry_point_rejects_a_null_context(lib):
    from paper_1907_13013_gb300 import binding
    assert lib.fpsa_set_limits(None, 0, 0.0) == binding.EINVAL
    assert lib.fpsa_set_limits(None, 4, 1.0) == binding.EINVAL


def test_tuning_entry_points_reject_a_null_context(lib):
    # argument checks come before any CUDA call
    from paper_1907_13013_gb300 import binding
    t = binding.FpsaTuning()
    assert ctypes.sizeof(t) == 24  # six int32 fields, as in include/fpsa.h
    ms = ctypes.c_double()
    assert lib.fpsa_get_tuning(None, ctypes.byref(t)) == binding.EINVAL
    assert lib.fpsa_set_tuning(None, None) == binding.EINVAL
    assert lib.fpsa_autotune(None, None, 1, ctypes.byref(t), ctypes.byref(ms)) == binding.EINVAL


def test_tuning_cache_keys_and_file(tmp_path):
    from paper_1907_13013_gb300 import batch
    k = batch.TuningCache.key(64, 63, 1, 3, 1000, "mixed", "wfd", "fpsa")
    assert k == "mixed/wfd/fpsa/N64/L63/R1/B4/K1024"
    # the instance count and the largest cell count share a key within a power of two
    assert batch.TuningCache.key(64, 63, 1, 4, 513, "mixed", "wfd", "fpsa") == k
    assert batch.TuningCache.key(64, 63, 1, 5, 1000, "mixed", "wfd", "fpsa") != k
    assert batch.TuningCache.key(16, 15, 1, 1, 1, "fp64", "mpd", "si").endswith("/B1/K1")
    path = str(tmp_path / "shapes.json")
    c = batch.TuningCache(path)
    assert c.get(k) is None
    shapes = {"sweep_cells_per_thread": 8, "solve_blocks_per_sm": 2, "solve_max_slices": 4}
    c.put(k, shapes, 3.5)
    c.save()
    c2 = batch.TuningCache(path)
    assert c2.get(k) == shapes and c2.entries[k]["ms"] == 3.5
    assert batch.TuningCache(None).get(k) is None


@pytest.mark.parametrize("N,L", [(2, 1), (16, 15), (16, 7), (64, 63), (256, 255)])
@pytest.mark.parametrize("lap", ["mpd", "wfd"])
def test_library_tables_match_the_oracle(lib, N, L, lap):
    # host logic of the library (fpsa_tables: no GPU): its Gauss-Legendre rule, D, M
    # and angular Laplacian against the oracle's, which is pinned to 50-digit roots
    from oracle import quadrature as qd
    from paper_1907_13013_gb300 import binding
    t = binding.tables(N, L, lap)
    mu, w = qd.gauss_legendre(N)
    assert np.all(np.abs(t["mu"] - mu) <= 2.3e-16)
    # weights: first-order change at a node one ulp apart, plus the recurrences' rounding
    bound = 2 * np.abs(mu) * 2.3e-16 / ((1 - mu) * (1 + mu)) + 8 * N * 2.2e-16
    assert np.all(np.abs(t["w"] / w - 1) <= bound), np.max(np.abs(t["w"] / w - 1) / bound)
    D = qd.moment_operator(mu, w, L)
    M = qd.expansion_operator(mu, L)
    assert np.abs(t["D"] - D).max() <= 1e-13 * np.abs(D).max()
    assert np.abs(t["M"] - M).max() <= 1e-13 * np.abs(M).max()
    A = qd.angular_laplacian(mu, w, lap)
    assert np.abs(t["A"] - A).max() <= 1e-11 * np.abs(A).max()


def test_library_tables_reject_bad_sizes(lib):
    from paper_1907_13013_gb300 import binding
    for N, L1, lap in ((3, 1, 0), (0, 1, 0), (258, 1, 0), (16, 0, 0), (16, 17, 0), (16, 4, 2)):
        assert lib.fpsa_tables(N, L1, lap, None, None, None, None, None) == binding.EINVAL
    assert lib.fpsa_tables(16, 16, 1, None, None, None, None, None) == binding.OK


def test_batch_driver_searches_each_missing_key_once_then_uses_the_cache(tmp_path, monkeypatch):
    # host logic of BatchSolver with a stand-in for the library context and for
    # torch's CUDA stream objects (no GPU): one serial fpsa_autotune per key the cache
    # lacks, before any wave solves; every wave then runs with its key's shapes
    import contextlib
    import threading
    import torch
    from paper_1907_13013_gb300 import batch, binding, inputs

    log, lock = [], threading.Lock()
    solving = {"n": 0}

    class FakeCtx:
        def __init__(self, probs):
            self.probs, self.R = probs, 1
            self.shape = {"sweep_cells_per_thread": 4, "solve_blocks_per_sm": 2, "solve_max_slices": 4}

        def autotune(self, **kw):
            with lock:
                assert solving["n"] == 0  # no wave is solving while a search times solves
                log.append(("autotune", self.probs[0]["N"], len(self.probs)))
            return {"sweep_cells_per_thread": 8, "solve_blocks_per_sm": 1, "solve_max_slices": 2}, 1.5

        def set_tuning(self, t):
            self.shape = dict(t)

        def get_tuning(self):
            return dict(self.shape)

        def solve(self, **kw):
            with lock:
                solving["n"] += 1
                log.append(("solve", self.probs[0]["N"], tuple(sorted(self.shape.items()))))
            K = sum(p["h"].size for p in self.probs)
            with lock:
                solving["n"] -= 1
            return np.zeros((1, K, 2, self.probs[0]["L"] + 1)), {"status": 0, "cell_angles": 0.0}

        def close(self):
            pass

    monkeypatch.setattr(binding, "context_for", lambda probs, **kw: FakeCtx(probs))
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "Stream", lambda device=None: type("S", (), {"cuda_stream": 0})())
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())

    probs = inputs.batch_slabs(30, seed=5, K_range=(20, 200))
    budget = batch.factor_bytes(200, 128, "mixed")  # one large S128 slab: several waves per group
    cache = batch.TuningCache(str(tmp_path / "shapes.json"))
    solver = batch.BatchSolver(probs, budget_bytes=budget, tuning=cache)
    keys = {solver._key(w, "fpsa") for w in solver.waves}
    assert len(keys) < len(solver.waves)  # some waves share a key
    phis, stats = solver.solve(tol=1e-10)
    searches = [e for e in log if e[0] == "autotune"]
    assert len(searches) == len(keys)
    first_solve = next(i for i, e in enumerate(log) if e[0] == "solve")
    assert all(i < first_solve for i, e in enumerate(log) if e[0] == "autotune")
    assert all(dict(e[2])["solve_max_slices"] == 2 for e in log if e[0] == "solve")
    assert {s["tuning_source"] for s in stats} == {"search"}
    assert len(phis) == len(probs) and all(phi.shape == (p["h"].size, 2, p["L"] + 1) for phi, p in zip(phis, probs))
    # a second driver over the same cache file searches nothing
    log.clear()
    _, stats2 = batch.BatchSolver(probs, budget_bytes=budget, tuning=batch.TuningCache(cache.path)).solve(tol=1e-10)
    assert not [e for e in log if e[0] == "autotune"]
    assert {s["tuning_source"] for s in stats2} == {"cache"}
