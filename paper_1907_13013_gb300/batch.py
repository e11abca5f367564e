"""Batched solves of many independent slabs of uneven cell counts and angular orders.

Slabs sharing (N, L) are solved together by one fpsa context (every kernel launch
covers all of them: ragged cell counts are handled inside the kernels through
per-instance offsets). Groups with different (N, L) run concurrently, each on its
own CUDA stream from its own host thread (the ctypes calls release the GIL). A
group whose factor storage would exceed the memory budget is split into waves,
packed greedily so that each wave's block-inverse storage stays within budget.
Launch shapes per wave can come from the library's autotuner, remembered in a
JSON cache. All arithmetic happens in the library; this module only partitions
the work.
"""

import concurrent.futures as cf
import json
import os
import threading

from . import binding

# fpsa_autotune takes the iteration settings of the solves it times
_TUNE_KEYS = ("method", "tol", "max_iterations", "inner_iterations", "inner_tol", "check_every", "contraction",
              "restart")


def _bucket(x):
    """Smallest power of two >= x (x >= 1)."""
    return 1 << max(0, int(x) - 1).bit_length()


class TuningCache:
    """Launch shapes chosen by fpsa_autotune, keyed by what decides them: (N, L), the
    right-hand sides, the precision, Laplacian and method, and power-of-two buckets of
    the instance count and of the largest cell count. Kept in a JSON file when a path
    is given (read at construction, rewritten by save()); safe to share between the
    batch driver's threads."""

    def __init__(self, path=None):
        self.path = path
        self.entries = {}
        self._lock = threading.Lock()
        if path and os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    @staticmethod
    def key(N, L, R, n_instances, max_cells, precision, laplacian, method):
        return "%s/%s/%s/N%d/L%d/R%d/B%d/K%d" % (precision, laplacian, method, N, L, R, _bucket(n_instances),
                                                 _bucket(max_cells))

    def get(self, key):
        with self._lock:
            e = self.entries.get(key)
            return dict(e["shapes"]) if e else None

    def put(self, key, shapes, ms):
        with self._lock:
            self.entries[key] = {"shapes": dict(shapes), "ms": float(ms)}

    def save(self):
        if not self.path:
            return
        with self._lock:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.entries, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def factor_bytes(K, N, precision):
    """Device bytes dominated by the FP blocks (2N x 2N per cell) and the per-level couplings."""
    es = 4 if precision == "mixed" else 8
    return es * K * (4 * N * N + 2 * 2 * (N // 2) ** 2) + 64 * es * K * N


def plan_waves(problems, budget_bytes, precision):
    """Group problem indices by (N, L), then split each group into waves within budget.
    Returns a list of (N, L, [indices]) in an order that starts the largest work first."""
    groups = {}
    for i, p in enumerate(problems):
        groups.setdefault((p["N"], p["L"]), []).append(i)
    waves = []
    for (N, L), idx in groups.items():
        idx = sorted(idx, key=lambda i: -problems[i]["h"].size)
        cur, used = [], 0
        for i in idx:
            b = factor_bytes(problems[i]["h"].size, N, precision)
            if cur and used + b > budget_bytes:
                waves.append((N, L, cur))
                cur, used = [], 0
            cur.append(i)
            used += b
        if cur:
            waves.append((N, L, cur))
    waves.sort(key=lambda w: -sum(problems[i]["h"].size for i in w[2]) * w[0] ** 2)
    return waves


class BatchSolver:
    """Solve a list of problem dicts (see inputs.py; single right-hand side each)."""

    def __init__(self, problems, precision="mixed", laplacian="wfd", budget_bytes=32 << 30, device=0,
                 max_streams=4, tuning=None, profile=False, graph=False):
        """tuning: None (the library's launch shapes), or a TuningCache: each wave takes
        the cached shapes of its key; keys missing from the cache are searched first, one
        wave at a time with nothing else on the GPU (fpsa_autotune times whole solves, so
        concurrent waves would distort each other's timings), then every wave runs.
        profile: time every launch of each wave's solve with the library's profiler (CUDA
        event pairs) and return the per-kernel-class times in the wave's stats.
        graph: solve in rounds of at most max_streams waves (different orders together,
        see rounds()), each round ONE launch of a CUDA graph (fpsa_solve_batch: every
        wave's refinement loop a device-side while node, the waves concurrent branches);
        MIXED precision, SI or FPSA. Contexts are still created and factorized on
        concurrent streams first."""
        self.problems = list(problems)
        self.precision, self.laplacian = precision, laplacian
        self.device = device
        self.waves = plan_waves(self.problems, budget_bytes, precision)
        self.max_streams = max_streams
        self.tuning = tuning
        self.profile = profile
        self.graph = graph
        if graph and precision != "mixed":
            raise ValueError("graph batches need precision='mixed'")

    def _key(self, wave, method):
        N, L, idx = wave
        return TuningCache.key(N, L, 1, len(idx), max(self.problems[i]["h"].size for i in idx), self.precision,
                               self.laplacian, method)

    def _context(self, wave, stream):
        return binding.context_for([self.problems[i] for i in wave[2]], laplacian=self.laplacian,
                                   precision=self.precision, device=self.device, stream=stream.cuda_stream)

    def _search(self, solve_kw):
        """Autotune (serially) one wave of every key the cache lacks; returns the keys searched."""
        import torch
        torch.cuda.set_device(self.device)
        searched = set()
        for wave in self.waves:
            key = self._key(wave, solve_kw.get("method", "fpsa"))
            if key in searched or self.tuning.get(key) is not None:
                continue
            stream = torch.cuda.Stream(device=self.device)
            with torch.cuda.stream(stream):
                ctx = self._context(wave, stream)
                try:
                    shapes, ms = ctx.autotune(**{k: v for k, v in solve_kw.items() if k in _TUNE_KEYS})
                finally:
                    ctx.close()
            self.tuning.put(key, shapes, ms)
            searched.add(key)
        return searched

    def _run_wave(self, wave, solve_kw, searched):
        import torch
        N, L, idx = wave
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(device=self.device)
        probs = [self.problems[i] for i in idx]
        with torch.cuda.stream(stream):
            ctx = self._context(wave, stream)
            try:
                source = "library"
                if self.tuning is not None:
                    key = self._key(wave, solve_kw.get("method", "fpsa"))
                    ctx.set_tuning(self.tuning.get(key))
                    source = "search" if key in searched else "cache"
                tuned = ctx.get_tuning()
                if self.profile:
                    ctx.profile_enable(True)
                phi, st = ctx.solve(**solve_kw)
                prof = ctx.profile_read() if self.profile else None
            finally:
                ctx.close()
        out, off = {}, 0
        for i, p in zip(idx, probs):
            K = p["h"].size
            out[i] = phi[0, off:off + K]
            off += K
        extra = {"profile": prof} if prof is not None else {}
        return out, dict(st, N=N, instances=len(idx), cells=int(sum(p["h"].size for p in probs)),
                         tuning=tuned, tuning_source=source, **extra)

    def rounds(self):
        """Graph mode: lists of at most max_streams waves, each list one graph launch. A
        round first takes the next wave of every (N, L) group that has one left, the
        groups with the most remaining work first, then further waves of the groups with
        the most work left while room remains, so orders mix in the early rounds and the
        largest group keeps max_streams waves running concurrently at the end."""
        by_group = {}
        for w in self.waves:
            by_group.setdefault((w[0], w[1]), []).append(w)
        work = lambda w: sum(self.problems[i]["h"].size for i in w[2]) * w[0] ** 2  # noqa: E731
        left = {k: list(v) for k, v in by_group.items()}
        out = []
        while any(left.values()):
            rnd = []
            order = sorted((k for k in left if left[k]), key=lambda k: -sum(work(w) for w in left[k]))
            for k in order:
                if len(rnd) < self.max_streams:
                    rnd.append(left[k].pop(0))
            while len(rnd) < self.max_streams and any(left.values()):
                k = max((k for k in left if left[k]), key=lambda k: sum(work(w) for w in left[k]))
                rnd.append(left[k].pop(0))
            out.append(rnd)
        return out

    def _prepare_wave(self, wave, method, searched):
        import torch
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(device=self.device)
        with torch.cuda.stream(stream):
            ctx = self._context(wave, stream)
            source = "library"
            if self.tuning is not None:
                key = self._key(wave, method)
                try:
                    ctx.set_tuning(self.tuning.get(key))
                except BaseException:
                    ctx.close()
                    raise
                source = "search" if key in searched else "cache"
        return ctx, stream, source

    def _round_bytes(self, rnd):
        return sum(factor_bytes(sum(self.problems[i]["h"].size for i in w[2]), w[0], self.precision) for w in rnd)

    def _solve_graph(self, solve_kw, searched):
        """Rounds of waves, each one graph launch (fpsa_solve_batch, which releases the GIL);
        the next round's contexts are created and factorized on the pool's streams while
        the current round's graph runs, when free device memory holds both rounds."""
        import torch
        results = [None] * len(self.problems)
        stats = []
        kw = {k: v for k, v in solve_kw.items() if k in ("method", "tol", "max_iterations", "inner_iterations",
                                                        "contraction")}
        method = solve_kw.get("method", "fpsa")
        rounds = self.rounds()
        with cf.ThreadPoolExecutor(max_workers=self.max_streams) as ex:
            def start(rnd):
                return [ex.submit(self._prepare_wave, w, method, searched) for w in rnd]

            def close_all(futures):
                """Close every context of a round being prepared (on the way out of an error)."""
                for f in futures or []:
                    try:
                        f.result()[0].close()
                    except Exception:
                        pass

            pending = start(rounds[0]) if rounds else None
            try:
                for r, rnd in enumerate(rounds):
                    futures, pending = pending, None
                    try:
                        prepared = [f.result() for f in futures]
                    except BaseException:
                        close_all(futures)
                        raise
                    ctxs = [c for c, _, _ in prepared]
                    try:
                        if r + 1 < len(rounds):
                            free, _ = torch.cuda.mem_get_info(self.device)
                            if free > 1.25 * self._round_bytes(rounds[r + 1]) + (4 << 30):
                                pending = start(rounds[r + 1])
                        phis, sts = binding.solve_batch(ctxs, **kw)
                        for (N, L, idx), phi, st, (ctx, _, source) in zip(rnd, phis, sts, prepared):
                            off = 0
                            for i in idx:
                                K = self.problems[i]["h"].size
                                results[i] = phi[0, off:off + K]
                                off += K
                            stats.append(dict(st, N=N, instances=len(idx), cells=int(off), tuning=ctx.get_tuning(),
                                              tuning_source=source, graph_round=r))
                    finally:
                        for c in ctxs:
                            c.close()
                    if pending is None and r + 1 < len(rounds):
                        pending = start(rounds[r + 1])
            except BaseException:
                close_all(pending)
                raise
        return results, stats

    def solve(self, method="fpsa", tol=1e-10, max_iterations=10000, **kw):
        """Returns (list of phi [K][2][L+1] per problem, list of per-wave stats)."""
        solve_kw = dict(method=method, tol=tol, max_iterations=max_iterations, **kw)
        results = [None] * len(self.problems)
        stats = []
        searched = self._search(solve_kw) if self.tuning is not None else set()
        if self.graph:
            results, stats = self._solve_graph(solve_kw, searched)
            if self.tuning is not None:
                self.tuning.save()
            return results, stats
        with cf.ThreadPoolExecutor(max_workers=self.max_streams) as ex:
            for out, st in ex.map(lambda w: self._run_wave(w, solve_kw, searched), self.waves):
                for i, phi in out.items():
                    results[i] = phi
                stats.append(st)
        if self.tuning is not None:
            self.tuning.save()
        return results, stats
