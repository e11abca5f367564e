"""The batch driver on the CPU, with stand-in contexts (and, for the graph rounds, a
stand-in fpsa_solve_batch): every wave's flux lands at its problems and every context is
closed once, also when a solve raises (in graph mode while the next round is being
prepared; in thread mode while other waves run)."""
import threading

import numpy as np
import pytest


class FakeCtx:
    created = []
    lock = threading.Lock()

    def __init__(self, wave):
        self.wave, self.closed = wave, 0
        with FakeCtx.lock:
            FakeCtx.created.append(self)

    def close(self):
        self.closed += 1

    def get_tuning(self):
        return {"source": "fake"}


def setup(monkeypatch, fail_round=None, free_bytes=1 << 40):
    import torch

    from paper_1907_13013_gb300 import batch, binding, inputs
    FakeCtx.created = []
    probs = inputs.batch_slabs(40, seed=5, K_range=(20, 300))
    solver = batch.BatchSolver(probs, precision="mixed", laplacian="wfd", budget_bytes=2 << 20, graph=True)
    rounds = solver.rounds()
    assert len(rounds) >= 3
    calls = []

    def prepare(self, wave, method, searched):
        return FakeCtx(wave), None, "library"

    def solve_batch(ctxs, **kw):
        r = len(calls)
        calls.append([c.wave for c in ctxs])
        if r == fail_round:
            raise binding.FpsaError(binding.ENOTCONV, "stand-in failure")
        phis = []
        for c in ctxs:
            # phi [1][cells][2][L + 1] with the problem index in every entry of its cells
            parts = [np.full((probs[i]["h"].size, 2, probs[i]["L"] + 1), float(i)) for i in c.wave[2]]
            phis.append(np.concatenate(parts)[None])
        return phis, [{"status": 0, "outer_iterations": 3} for _ in ctxs]

    monkeypatch.setattr(batch.BatchSolver, "_prepare_wave", prepare)
    monkeypatch.setattr(binding, "solve_batch", solve_batch)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda device=None: (free_bytes, free_bytes))
    return solver, probs, rounds, calls


@pytest.mark.parametrize("free_bytes", [1 << 40, 1 << 20])  # next round prepared during the solve, or after it
def test_graph_rounds_deliver_every_flux_and_close_every_context(monkeypatch, free_bytes):
    solver, probs, rounds, calls = setup(monkeypatch, free_bytes=free_bytes)
    phis, stats = solver.solve(tol=1e-10, max_iterations=50)
    assert [len(c) for c in calls] == [len(r) for r in rounds]
    for i, phi in enumerate(phis):
        assert phi.shape == (probs[i]["h"].size, 2, probs[i]["L"] + 1) and np.all(phi == i)
    assert sum(s["instances"] for s in stats) == len(probs)
    assert sorted({s["graph_round"] for s in stats}) == list(range(len(rounds)))
    assert len(FakeCtx.created) == sum(len(r) for r in rounds)
    assert all(c.closed == 1 for c in FakeCtx.created)


@pytest.mark.parametrize("fail_round", [0, 1])
def test_a_failing_round_closes_its_contexts_and_the_next_rounds(monkeypatch, fail_round):
    from paper_1907_13013_gb300 import binding
    solver, probs, rounds, calls = setup(monkeypatch, fail_round=fail_round)
    with pytest.raises(binding.FpsaError):
        solver.solve(tol=1e-10, max_iterations=50)
    assert len(calls) == fail_round + 1
    # the failing round's contexts and the next round's, prepared meanwhile, are all closed
    assert len(FakeCtx.created) == sum(len(r) for r in rounds[:fail_round + 2])
    assert all(c.closed == 1 for c in FakeCtx.created)


class FakeSolveCtx(FakeCtx):
    def __init__(self, probs, wave, fail):
        super().__init__(wave)
        self.probs, self.fail = probs, fail

    def set_tuning(self, t):
        pass

    def solve(self, **kw):
        if self.fail:
            from paper_1907_13013_gb300 import binding
            raise binding.FpsaError(binding.ENOTCONV, "stand-in failure")
        parts = [np.full((self.probs[i]["h"].size, 2, self.probs[i]["L"] + 1), float(i)) for i in self.wave[2]]
        return np.concatenate(parts)[None], {"status": 0}


@pytest.mark.parametrize("fail", [False, True])
def test_thread_waves_deliver_every_flux_and_close_every_context(monkeypatch, fail):
    import contextlib

    import torch

    from paper_1907_13013_gb300 import batch, binding, inputs
    FakeCtx.created = []
    probs = inputs.batch_slabs(30, seed=6, K_range=(20, 300))
    solver = batch.BatchSolver(probs, precision="mixed", laplacian="wfd", budget_bytes=2 << 20)
    first = id(solver.waves[len(solver.waves) // 2])
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "Stream", lambda device=None: None)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(batch.BatchSolver, "_context",
                        lambda self, wave, stream: FakeSolveCtx(probs, wave, fail and id(wave) == first))
    if fail:
        with pytest.raises(binding.FpsaError):
            solver.solve(tol=1e-10)
    else:
        phis, stats = solver.solve(tol=1e-10)
        for i, phi in enumerate(phis):
            assert np.all(phi == i) and phi.shape == (probs[i]["h"].size, 2, probs[i]["L"] + 1)
        assert len(stats) == len(solver.waves)
    assert FakeCtx.created and all(c.closed == 1 for c in FakeCtx.created)
