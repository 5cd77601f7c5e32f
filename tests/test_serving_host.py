"""The serving loop's scheduling on the host, with a simulated executor (no GPU): every request
is served once with the same result as alone, no more than `slots` requests run at once, the
resident factors and factorizations in flight stay within the memory budget (evicting idle
factors, factoring again when an evicted factor is asked for), and a repeat solve uses its
factor on the slot that owns it."""
import threading
import time

import numpy as np
import pytest

import hm_workloads as W
from paper_1911_07531_gb300.serve import Server, latency_summary


class SimExecutor:
    def __init__(self, per_point=2e-8):
        self.per_point = per_point
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0
        self.factors = 0
        self.released = 0
        self.solves = []
        self.batches = []

    @staticmethod
    def estimate_bytes(r):
        return 1000.0 * r["n"]

    def _enter(self):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)

    def _leave(self):
        with self.lock:
            self.active -= 1

    def factorize(self, slot, r):
        self._enter()
        time.sleep(self.per_point * r["n"])
        with self.lock:
            self.factors += 1
        self._leave()
        return (slot, r["seed"], r["n"]), 900.0 * r["n"]

    def factorize_batch(self, slot, group):
        assert len({r["eps"] for r in group}) == 1      # one accuracy per merged call
        with self.lock:
            self.batches.append(len(group))
        return [self.factorize(slot, r) for r in group]

    def solve(self, slot, handle, r):
        owner, seed, n = handle
        assert owner == slot and n == r["n"] and seed == r["seed"]
        self._enter()
        time.sleep(1e-4)
        self._leave()
        with self.lock:
            self.solves.append(r["rid"])
        return np.random.default_rng([seed, r["rhs_seed"]]).standard_normal(r["nrhs"])

    def release(self, handle):
        with self.lock:
            self.released += 1


def _stream(count=150):
    return W.serving_requests(count=count, rate=3000.0, seed=7, n_min=2048, n_max=65536)


def test_serving_stream_recipe():
    rq = W.serving_requests(count=400, seed=3)
    assert [r["rid"] for r in rq] == list(range(400))
    assert all(b["arrival"] > a["arrival"] for a, b in zip(rq, rq[1:]))
    assert all(1 <= r["nrhs"] <= 32 and r["eps"] in (1e-4, 1e-6) for r in rq)
    firsts = {r["rid"]: r for r in rq if r["repeat_of"] is None}
    assert all(2048 <= r["n"] <= 131072 and r["geometry"] in ("sphere", "cube") for r in firsts.values())
    for r in rq:
        if r["repeat_of"] is not None:
            src = firsts[r["repeat_of"]]
            assert src["rid"] < r["rid"] and (src["n"], src["seed"], src["eps"]) == (r["n"], r["seed"], r["eps"])
    frac = sum(r["repeat_of"] is not None for r in rq) / len(rq)
    assert 0.35 < frac < 0.6


@pytest.mark.parametrize("slots,budget", [(4, 2e9), (3, 1.5e8)])
def test_every_request_served_once_with_its_result_alone(slots, budget):
    rq = _stream()
    ex = SimExecutor()
    srv = Server(ex, slots=slots, budget_bytes=budget)
    recs = srv.run(rq)
    assert [r["rid"] for r in recs] == [r["rid"] for r in rq]
    assert all(r["end"] >= r["start"] >= r["arrival"] - 1e-9 for r in recs)
    assert ex.max_active <= slots
    assert srv.peak <= budget
    # the same request served alone gives the same result
    for r in rq[:: 7]:
        alone = Server(SimExecutor(), slots=1, budget_bytes=budget)
        src = [q for q in rq if q["rid"] == r["repeat_of"]] + [r]
        alone.run(src)
        assert np.array_equal(alone.results[r["rid"]], srv.results[r["rid"]])
    s = latency_summary(recs)
    assert s["requests"] == len(rq) and 0 < s["p50_s"] <= s["p99_s"] and s["throughput_per_s"] > 0
    srv.release_all()
    assert ex.released == ex.factors


def test_tight_budget_evicts_and_factors_again():
    rq = _stream(120)
    ex = SimExecutor()
    srv = Server(ex, slots=2, budget_bytes=1.4e8)   # about two of the largest problems
    recs = srv.run(rq)
    assert srv.peak <= 1.4e8
    assert srv.evictions > 0
    kinds = {r["kind"] for r in recs}
    assert "refactor+solve" in kinds
    firsts = sum(r["repeat_of"] is None for r in rq)
    assert ex.factors == firsts + sum(r["kind"] == "refactor+solve" for r in recs)


def test_request_larger_than_the_budget_is_reported():
    rq = [dict(rid=0, arrival=0.0, geometry="cube", n=100000, eps=1e-6, nrhs=1, seed=1, rhs_seed=2, repeat_of=None)]
    with pytest.raises(RuntimeError):
        Server(SimExecutor(), slots=1, budget_bytes=1e6).run(rq)


def test_batched_factorizations_serve_every_request_with_its_result_alone():
    """With batch > 1, waiting factorizations of one eps are grouped into one executor call: every
    request is served once, groups never mix eps or exceed `batch`, the budget holds, and every
    result equals the same request served alone."""
    rq = _stream(160)
    ex = SimExecutor()
    srv = Server(ex, slots=3, budget_bytes=2e9, batch=4)
    recs = srv.run(rq)
    assert [r["rid"] for r in recs] == [r["rid"] for r in rq]
    assert ex.batches and max(ex.batches) <= 4 and max(ex.batches) > 1
    assert srv.peak <= 2e9
    by_rid = {r["rid"]: r for r in rq}
    for rec in recs:
        assert rec["batched"] >= 1
    for r in rq[:: 9]:
        alone = Server(SimExecutor(), slots=1, budget_bytes=2e9)
        src = [q for q in rq if q["rid"] == r["repeat_of"]] + [r]
        alone.run(src)
        assert np.array_equal(alone.results[r["rid"]], srv.results[r["rid"]])
    assert len(srv.results) == len(by_rid)
    srv.release_all()
    assert ex.released == ex.factors
