"""Request loop for factorize-and-solve requests on one GPU.

Requests arrive over time. A request either factors a new problem and solves with it, or
solves again with a factor that an earlier request produced. The loop:

* admits a factorization when a slot is free and its device-memory estimate fits the budget
  next to the factors kept resident, evicting the least recently used idle factors when it
  does not;
* runs up to `slots` requests at once, each slot with its own CUDA stream (its own library
  context), so that the small kernel launches of concurrent factorizations overlap on the
  device; with `batch` > 1 a slot takes several waiting factorizations of the same eps and
  factors them in one call whose waves share kernel launches (hm_lu_batch);
* keeps factors resident after their request, for later solves with them (a solve runs on the
  slot that owns the factor, as soon as that slot is free);
* records arrival, start and end of every request: latency percentiles and throughput.

The device work is done by an executor: `GpuExecutor` uses the library (hm_build, hm_lu,
hm_solve); any object with the same four methods can stand in (the scheduling logic is tested
on the host with a simulated executor).
"""
from __future__ import annotations

import time
from concurrent.futures import FIRST_COMPLETED, ThreadPoolExecutor, wait

import numpy as np

__all__ = ["Server", "GpuExecutor", "latency_summary"]


class Server:
    def __init__(self, executor, slots: int = 4, budget_bytes: float = 150e9, clock=time.perf_counter,
                 batch: int = 1):
        """batch > 1: a slot that starts a factorization takes up to `batch` waiting
        factorization requests of the same eps and factors them in one call of the executor's
        factorize_batch (their waves share kernel launches: hm_lu_batch)."""
        if slots < 1 or batch < 1:
            raise ValueError("slots and batch must be >= 1")
        self.ex = executor
        self.batch = int(batch)
        self.slots = int(slots)
        self.budget = float(budget_bytes)
        self.clock = clock
        self.resident = {}      # rid -> {"handle", "bytes", "slot", "last"}
        self.used = 0.0         # bytes of resident factors and of factorizations in flight
        self.peak = 0.0
        self.evictions = 0

    # -- memory ---------------------------------------------------------------------------------
    def _make_room(self, need, busy_slots):
        """Evict least recently used factors whose slot is idle until `need` more bytes fit."""
        if self.used + need <= self.budget:
            return True
        idle = sorted((v["last"], rid) for rid, v in self.resident.items() if v["slot"] not in busy_slots)
        for _, rid in idle:
            v = self.resident.pop(rid)
            self.ex.release(v["handle"])
            self.used -= v["bytes"]
            self.evictions += 1
            if self.used + need <= self.budget:
                return True
        return self.used + need <= self.budget

    # -- the loop ---------------------------------------------------------------------------------
    def run(self, requests):
        """Serve `requests` (dicts as produced by hm_workloads.serving_requests, arrival times in
        seconds from the start); returns one record per request, in request order."""
        reqs = sorted(requests, key=lambda r: (r["arrival"], r["rid"]))
        recs = {r["rid"]: dict(rid=r["rid"], arrival=r["arrival"], kind="solve" if r["repeat_of"] is not None
                               else "factor+solve") for r in reqs}
        pending = []            # arrived, not started
        nxt = 0                 # next request to arrive
        running = {}            # future -> (slot, request, estimate)
        busy = set()
        results = {}
        t0 = self.clock()
        pool = ThreadPoolExecutor(max_workers=self.slots)

        def job(slot, group, factor):
            # returns the start time and one (request, handle, bytes, result) per request
            start = self.clock() - t0
            if factor is not None:      # a solve with a resident factor (owned by this slot)
                return start, [(group[0], None, 0.0, self.ex.solve(slot, factor, group[0]))]
            if len(group) == 1:
                made = [self.ex.factorize(slot, group[0])]
            else:
                made = self.ex.factorize_batch(slot, group)
            return start, [(r, h, nb, self.ex.solve(slot, h, r)) for r, (h, nb) in zip(group, made)]

        def new_factor(q):
            """q as a factorization request (an evicted repeat is factored again), or None."""
            if q["repeat_of"] is None:
                return q
            if q["repeat_of"] in self.resident:
                return None
            if any(x["rid"] == q["repeat_of"] for _, grp, _ in running.values() for x in grp) or \
                    any(x["rid"] == q["repeat_of"] for x in pending):
                return None
            return dict(q, repeat_of=None, refactor_of=q["repeat_of"])

        try:
            while nxt < len(reqs) or pending or running:
                now = self.clock() - t0
                while nxt < len(reqs) and reqs[nxt]["arrival"] <= now:
                    pending.append(reqs[nxt])
                    nxt += 1
                # start what can start, in arrival order
                still = []
                taken = set()
                for r in pending:
                    if r["rid"] in taken:
                        continue
                    free = [s for s in range(self.slots) if s not in busy]
                    if not free:
                        still.append(r)
                        continue
                    if r["repeat_of"] is not None:
                        src = self.resident.get(r["repeat_of"])
                        if src is None:
                            if any(q["rid"] == r["repeat_of"] for _, grp, _ in running.values() for q in grp) or \
                                    any(q["rid"] == r["repeat_of"] for q in still):
                                still.append(r)     # its factor is still being computed
                                continue
                            # evicted: factor again
                            r = dict(r, repeat_of=None, refactor_of=r["repeat_of"])
                            recs[r["rid"]]["kind"] = "refactor+solve"
                        else:
                            if src["slot"] in busy:
                                still.append(r)
                                continue
                            src["last"] = now
                            busy.add(src["slot"])
                            running[pool.submit(job, src["slot"], [r], src["handle"])] = (src["slot"], [r], [0.0])
                            continue
                    est = float(self.ex.estimate_bytes(r))
                    if not self._make_room(est, busy):
                        still.append(r)
                        continue
                    group, ests = [r], [est]
                    if self.batch > 1:
                        # later waiting factorizations of the same eps join the group while they fit
                        for q in pending:
                            if len(group) >= self.batch:
                                break
                            if q["rid"] <= r["rid"] or q["rid"] in taken:
                                continue
                            qf = new_factor(q)
                            if qf is None or qf["eps"] != r["eps"]:
                                continue
                            e = float(self.ex.estimate_bytes(qf))
                            if self.used + sum(ests) + e > self.budget:
                                continue
                            if qf.get("refactor_of") is not None:
                                recs[qf["rid"]]["kind"] = "refactor+solve"
                            group.append(qf)
                            ests.append(e)
                            taken.add(q["rid"])
                    slot = free[0]
                    busy.add(slot)
                    self.used += sum(ests)
                    self.peak = max(self.peak, self.used)
                    running[pool.submit(job, slot, group, None)] = (slot, group, ests)
                pending = still
                if running:
                    timeout = None
                    if nxt < len(reqs):
                        timeout = max(0.0, reqs[nxt]["arrival"] - (self.clock() - t0))
                    done, _ = wait(list(running), timeout=timeout, return_when=FIRST_COMPLETED)
                    for f in done:
                        slot, group, ests = running.pop(f)
                        busy.discard(slot)
                        start, outs = f.result()
                        end = self.clock() - t0
                        for (r, handle, nbytes, out), est in zip(outs, ests):
                            rec = recs[r["rid"]]
                            rec.update(start=start, end=end, latency=end - r["arrival"], slot=slot,
                                       batched=len(group))
                            results[r["rid"]] = out
                            if handle is not None:
                                self.used += nbytes - est
                                self.peak = max(self.peak, self.used)
                                key = r.get("refactor_of", r["rid"])
                                old = self.resident.pop(key, None)
                                if old is not None:
                                    self.ex.release(old["handle"])
                                    self.used -= old["bytes"]
                                self.resident[key] = dict(handle=handle, bytes=nbytes, slot=slot, last=end)
                elif nxt < len(reqs):
                    delay = reqs[nxt]["arrival"] - (self.clock() - t0)
                    if delay > 0:
                        time.sleep(delay)
                elif pending:
                    raise RuntimeError("a request can never be served (it does not fit the memory budget)")
        finally:
            pool.shutdown(wait=True)
        self.results = results
        return [recs[r["rid"]] for r in sorted(reqs, key=lambda r: r["rid"])]

    def release_all(self):
        for v in self.resident.values():
            self.ex.release(v["handle"])
        self.resident.clear()
        self.used = 0.0


def latency_summary(records):
    """p50 / p99 latency (s), throughput (requests per second of makespan) and queueing."""
    lat = np.array([r["latency"] for r in records])
    wait_s = np.array([r["start"] - r["arrival"] for r in records])
    makespan = max(r["end"] for r in records) - min(r["arrival"] for r in records)
    return {"requests": len(records), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_queue_s": float(wait_s.mean()), "throughput_per_s": len(records) / makespan,
            "makespan_s": makespan}


class GpuExecutor:
    """Factorizations and solves with the library, one context (and CUDA stream) per slot."""

    def __init__(self, slots: int = 4, device: int = 0, leaf: int = 64, eta: float = 2.0, rank_cap: int = 64,
                 refine_tol: float = 0.0, precision: int = 0):
        """refine_tol > 0: every solve is refined against the H-matrix (hm_solve with
        residual_op HM_OP_A) to that relative residual; precision: HM_PREC_* of hm_lu."""
        import torch

        from . import HMContext
        self.torch = torch
        self.ctx = [HMContext(device, stream=torch.cuda.Stream(device)) for _ in range(slots)]
        self.leaf, self.eta, self.rank_cap = leaf, eta, rank_cap
        self.refine_tol, self.precision = float(refine_tol), int(precision)

    @staticmethod
    def estimate_bytes(r):
        # factor values + matrix values + plan scratch + micro-op arrays, per point (measured at
        # n = 131072: 13.2 GB of values each, 8.2 GB scratch, 2.5 GB of micro-ops)
        return 285_000.0 * r["n"]

    def factorize(self, slot, r):
        import hm_workloads as W

        from . import hm_build, hm_lu
        ctx = self.ctx[slot]
        with self.torch.cuda.stream(ctx.stream):
            A = hm_build(ctx, W.points_for(r["geometry"], r["n"], r["seed"]), self.leaf, self.eta, r["eps"],
                         self.rank_cap)
            F = hm_lu(ctx, A, precision=self.precision)
        # resident: the matrix and factor values and the matrix's uploaded H-LU plan (~19 kB of
        # micro-ops per point); the factorization's scratch is released when hm_lu returns
        nbytes = 2.0 * F.stats()["value_bytes"] + 19_000.0 * r["n"]
        return (slot, A, F), nbytes

    def factorize_batch(self, slot, group):
        """Factor several new problems in one hm_lu_batch call (same eps): their waves share the
        kernel launches. Returns one (handle, resident bytes) per request."""
        import hm_workloads as W

        from . import hm_build, hm_lu_batch
        ctx = self.ctx[slot]
        with self.torch.cuda.stream(ctx.stream):
            mats = [hm_build(ctx, W.points_for(r["geometry"], r["n"], r["seed"]), self.leaf, self.eta, r["eps"],
                             self.rank_cap) for r in group]
            Fs = hm_lu_batch(ctx, mats, precision=self.precision)
        # resident: the matrix and factor values (the merged plan is released after the call)
        return [((slot, A, F), 2.0 * F.stats()["value_bytes"]) for A, F in zip(mats, Fs)]

    def solve(self, slot, handle, r):
        import hm_workloads as W

        from . import HM_OP_A, hm_solve
        owner, A, F = handle
        ctx = self.ctx[owner]
        with self.torch.cuda.stream(ctx.stream):
            bh = W.gaussian_rhs(r["n"], r["nrhs"], r["rhs_seed"])
            b = self.torch.from_numpy(np.ascontiguousarray(bh.T)).to(f"cuda:{ctx.device}", non_blocking=False).t()
            if self.refine_tol > 0:
                x, _ = hm_solve(ctx, F, b, A=A, refine_tol=self.refine_tol, max_iter=30, residual_op=HM_OP_A)
            else:
                x, _ = hm_solve(ctx, F, b)
            return x.cpu().numpy()

    def release(self, handle):
        _, A, F = handle
        F.free()
        A.free()


def main(argv=None):
    """Serve the serving workload's request stream on GPU 0 and print one JSON summary line."""
    import argparse
    import json

    import hm_workloads as W
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--seed", type=int, default=51)
    ap.add_argument("--batch", type=int, default=1, help="factorizations merged into one hm_lu_batch call")
    a = ap.parse_args(argv)
    rq = W.serving_requests(count=a.requests, rate=a.rate, seed=a.seed)
    srv = Server(GpuExecutor(a.slots), slots=a.slots, budget_bytes=a.budget_gb * 1e9, batch=a.batch)
    recs = srv.run(rq)
    out = latency_summary(recs)
    out.update(slots=a.slots, budget_gb=a.budget_gb, offered_rate_per_s=a.rate, evictions=srv.evictions,
               peak_gb=srv.peak / 1e9, refactors=sum(r["kind"] == "refactor+solve" for r in recs))
    srv.release_all()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
