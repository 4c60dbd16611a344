"""The Poisson request loop on the GPU: every request's solution matches its
closed form, results in a batched mix equal the same request solved alone,
and the HBM budget is honoured (eviction, refusal of a batch that cannot fit)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1506_07933_gb300 import afft, serve, synth

pytestmark = pytest.mark.gpu

TOL = {"f32": 2e-6, "f64": 1e-12}


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    afft.load()
    yield


@pytest.mark.parametrize("n,dtype", [(32, torch.float64), (48, torch.float64), (40, torch.float32)])
def test_device_rhs_matches_the_host_mode_sum(n, dtype):
    ks, amp, phase = synth.draw_modes((n,) * 3, 16, 77)
    got = serve._mode_sum_gpu(n, ks, amp, phase, dtype).double().cpu().numpy()
    ref = synth.mode_sum((n,) * 3, ks, amp, phase)
    assert oracle.rel_l2(got, ref) <= (1e-14 if dtype == torch.float64 else 1e-6)


@pytest.fixture(scope="module")
def pool():
    return serve.RhsPool(sizes=(16, 32, 48, 64), samples=3)


def solo(pool, req):
    with afft.Plan((req.n,) * 3, "r2c", req.precision) as p:
        u = p.poisson(pool.rhs(req))
        torch.cuda.synchronize()
        return u


def test_pool_rhs_is_minus_laplacian_of_the_closed_form(pool):
    """The pooled f against the host mode sum with |k|^2-weighted amplitudes (float64)."""
    for n in (16, 48):
        ks, amp, phase = pool.modes(n, 1)
        ref = synth.mode_sum((n,) * 3, ks, amp * (ks * ks).sum(axis=1), phase)
        got = pool.f[(n, "f64", 1)].cpu().numpy()
        assert oracle.rel_l2(got, ref) <= 1e-14
        assert pool.f[(n, "f32", 1)].dtype == torch.float32


def test_server_solves_every_request_and_batches_change_nothing(pool):
    # all at once: more requests wait than lanes are free, so groups form as lanes free up
    reqs = serve.poisson_requests(40, rate=0.0, sizes=(16, 32, 48, 64), f64_share=0.3, samples=3, seed=3)
    srv = serve.PoissonServer(pool, slots=3, max_batch_bytes=1 << 20, max_batch=8)
    try:
        srv.warm((16, 32, 48, 64))
        out, wall = srv.run(reqs, keep_results=True)
    finally:
        srv.close()
    assert sorted(r.rid for r in out) == list(range(40))
    assert max(r.batch for r in out) > 1, "the burst should have been batched"
    for r in out:
        assert r.done >= r.start >= r.arrival - 1e-9
        assert 0 < r.error <= TOL[r.precision], (r.rid, r.n, r.precision, r.error)
        alone = solo(pool, r)
        d = torch.linalg.vector_norm((srv.results[r.rid] - alone).double()) / torch.linalg.vector_norm(alone.double())
        assert float(d) <= (1e-6 if r.precision == "f32" else 1e-14), (r.rid, float(d))
    s = serve.summarize(out, wall)
    assert s["requests"] == 40 and s["p99_ms"] >= s["p50_ms"] > 0


def test_plain_loop_solves_every_request(pool):
    reqs = serve.poisson_requests(8, rate=0, sizes=(32, 64), f64_share=0.5, samples=3, seed=4)
    out, wall = serve.run_plain(pool, reqs, warm_sizes=(32, 64))
    assert len(out) == 8 and wall > 0
    for r in out:
        assert 0 < r.error <= TOL[r.precision], (r.rid, r.error)


def test_budget_evicts_idle_plans_and_refuses_what_cannot_fit(pool):
    srv = serve.PoissonServer(pool, slots=2, max_batch=1)
    srv.budget = srv._footprint(64, "f32", 1) + srv._footprint(32, "f32", 1)
    try:
        srv.warm((64, 32), ("f32",))
        assert srv.held <= srv.budget
        reqs = serve.poisson_requests(6, rate=0, sizes=(64, 48, 32), f64_share=0.0, samples=3, seed=9)
        out, _ = srv.run(reqs)
        assert srv.held <= srv.budget
        assert all(0 < r.error <= TOL["f32"] for r in out)
        with pytest.raises(MemoryError):
            srv._take(128, "f32", 1)
    finally:
        srv.close()
