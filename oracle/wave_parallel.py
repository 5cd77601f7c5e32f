"""H-LU executed as the task graph of Alg 11, wave by wave on host threads. Oracle; test-only.

The same arithmetic as the recursive oracle (``HLUFactor``: Alg 1, Alg 2, Alg 3 and its upper
mirror), driven by the task graph of §3.1 instead of the recursion: the leaf tasks of the graph
(the tasks Alg 11 cannot refine further) are grouped by their longest-path level, and the tasks
of one level run concurrently on a thread pool. A task starts only after every task of the
previous levels has finished, so every edge of the graph is respected. Updates of one target
block inside one level have no edge between them (Def 3.2 links outputs to inputs only); they
are serialised by a lock per leaf block of the target and applied in whatever order the
threads reach them, so the result equals the recursive one up to the rounding of the
truncations (the updates commute up to rounding).

This is the CPU baseline's parallel variant: the oracle's per-task numpy work spread over the
host's cores. Its result is checked against the 10 eps bound like the recursive oracle's.
"""
from __future__ import annotations

import threading
from concurrent.futures import ThreadPoolExecutor

from .dag import LU, MUL, TRSL, TRSU, TaskGraphBuilder, levels
from .hlu import HLUFactor


class WaveParallelHLU(HLUFactor):
    def __init__(self, hm, eps=None, rank_cap=None, threads=None):
        super().__init__(hm, eps, rank_cap)
        self.threads = threads
        self._locks = {b.key: threading.Lock() for b in self.bt.leaves()}
        self._stats_lock = threading.Lock()
        self.waves = 0
        self.tasks = 0

    def _task_graph(self):
        nodes, edges = TaskGraphBuilder(self.ct, self.bt).compute_dag()
        lev = levels(nodes, edges)
        nw = 1 + max(lev.values()) if lev else 0
        waves = [[] for _ in range(nw)]
        for t in nodes:
            waves[lev[t]].append(t)
        return waves

    def _run(self, task):
        ty, a, b, c = task
        cl = self.cl
        if ty == LU:
            self.hlu(cl[a])
        elif ty == TRSL:
            self.htrsl(cl[a], cl[b])
        elif ty == TRSU:
            self.htrsu(cl[a], cl[b])
        else:
            assert ty == MUL
            C = self.bt.get(cl[a], cl[c])
            keys = sorted(lf.key for lf in ([C] if C.is_leaf else self.bt.leaves_under(C)))
            locks = [self._locks[k] for k in keys]
            for lk in locks:             # one global order: no deadlock between targets
                lk.acquire()
            try:
                self.hmul(-1.0, self.bt.get(cl[a], cl[b]), self.bt.get(cl[b], cl[c]), C)
            finally:
                for lk in reversed(locks):
                    lk.release()

    def plan(self):
        """Build the task graph and its waves (timed apart from the execution, like the DAG
        construction of the GPU path)."""
        if getattr(self, "_waves", None) is None:
            self._waves = self._task_graph()
            self.waves = len(self._waves)
            self.tasks = sum(len(w) for w in self._waves)
        return self

    def factor(self):
        self.plan()
        with ThreadPoolExecutor(max_workers=self.threads) as pool:
            for w in self._waves:
                for f in [pool.submit(self._run_counted, t) for t in w]:
                    f.result()
        return self

    def _run_counted(self, task):
        # the arithmetic of HLUFactor updates self.stats; each task counts into its own
        # counters (self.stats resolves per thread), added to the shared ones under a lock
        local = _LocalStats(self.__dict__["_stats"])
        self._tls.stats = local
        try:
            self._run(task)
        finally:
            self._tls.stats = None
            with self._stats_lock:
                base = self.__dict__["_stats"]
                base.flops += local.flops
                base.cap_hits += local.cap_hits
                base.truncations += local.truncations

    _tls = threading.local()

    @property
    def stats(self):
        s = getattr(self._tls, "stats", None)
        return s if s is not None else self.__dict__["_stats"]

    @stats.setter
    def stats(self, v):
        self.__dict__["_stats"] = v


class _LocalStats:
    """Per-task counters with the attributes HLUFactor's arithmetic updates."""

    def __init__(self, base):
        self.__dict__["_base"] = base
        self.flops = 0.0
        self.cap_hits = 0
        self.truncations = 0

    def __getattr__(self, name):
        return getattr(self.__dict__["_base"], name)
