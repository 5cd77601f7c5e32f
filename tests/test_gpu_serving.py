"""The serving loop on the GPU: requests of different n run concurrently on several slots (one
CUDA stream each) and every result equals the same request served alone (GPU; C ABI).

Continuous batching is checked on a short stream of the serving workload's shape (Poisson
arrivals, sphere / cube, eps 1e-4 or 1e-6, repeat solves on resident factors) with small n:
the requests overlap on the device, and each solution, refined against the H-matrix to a
relative residual of 1e-10, matches the solution of the same request factored and solved alone
to 1e-8 (both solve the same H-matrix system; they differ by the rounding order of the
factorizations' atomic sums and by the refinement's stopping point)."""
import numpy as np
import pytest

import hm_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_07531_gb300 as hm
    hm.build_library()
    return hm


@pytest.mark.parametrize("batch", [1, 3])
def test_each_result_equals_alone_and_in_the_mix(hm, batch):
    """batch 3: waiting factorizations are also merged into hm_lu_batch calls across requests."""
    from paper_1911_07531_gb300.serve import GpuExecutor, Server, latency_summary
    rq = W.serving_requests(count=30, rate=400.0, seed=7, n_min=1024, n_max=6000)
    assert any(r["repeat_of"] is not None for r in rq)
    ex = GpuExecutor(slots=3, refine_tol=1e-10)
    srv = Server(ex, slots=3, budget_bytes=30e9, batch=batch)
    recs = srv.run(rq)
    mixed = srv.results
    srv.release_all()
    assert len(mixed) == len(rq)
    if batch > 1:
        assert max(r["batched"] for r in recs) > 1
    # concurrency: some request started before another one on a different slot had finished
    overlap = any(a["slot"] != b["slot"] and a["start"] < b["end"] and b["start"] < a["end"]
                  for i, a in enumerate(recs) for b in recs[i + 1:])
    assert overlap
    s = latency_summary(recs)
    assert s["p99_s"] >= s["p50_s"] > 0
    alone = GpuExecutor(slots=1, refine_tol=1e-10)
    worst = 0.0
    for r in rq:
        h, _ = alone.factorize(0, r)
        x = alone.solve(0, h, r)
        alone.release(h)
        y = mixed[r["rid"]]
        assert y.shape == x.shape
        worst = max(worst, float(np.linalg.norm(y - x) / np.linalg.norm(x)))
    assert worst <= 1e-8, worst
