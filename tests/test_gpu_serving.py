"""The request server on the GPU (mgmlmc_server_*): with fixed costs each request's
result is the same alone and in a mix of requests running at once (rounds, sample
counts and estimate), and the same as the one-context MLMC loop on the same inputs;
admission by footprint under a small HBM budget; cancellation and the refusals of
submit."""
import dataclasses
import time

import numpy as np
import pytest

import inputs
from oracle import hierarchy as ohier

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu
REL = 1e-12   # the same request, alone or in the mix: the same sample counts, the same sums


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


def _problem(name, **change):
    w = dataclasses.replace(inputs.workload(name), **change)
    return w, w.gauge(), w.start_vectors()


@pytest.fixture(scope="module")
def mix(pkg):
    """Four requests of three shapes and two precisions (2 and 3 levels, 16^2 and 32^2)."""
    reqs = []
    w, th, sv = _problem("schwinger-16x16")
    reqs.append(pkg.make_request(th, w.m0, w.agg, w.nvec, sv, 2e-2, 31, k=w.k, setup_iters=w.setup_iters,
                                 costs=[1.0, 0.1], mg_precision=16))
    reqs.append(pkg.make_request(th, -0.05, w.agg, w.nvec, sv, 2e-2, 32, k=w.k, setup_iters=w.setup_iters,
                                 costs=[1.0, 0.1], mg_precision=32))
    th3 = inputs.metropolis_u1(16, 16, 3.0, 20, 77)
    sv3 = [inputs.start_vectors(77, 1, 16 * 16 * 2, 8), inputs.start_vectors(77, 2, 4 * 4 * 16, 8)]
    reqs.append(pkg.make_request(th3, 0.0, ((4, 4), (2, 1)), (8, 8), sv3, 3e-2, 33, k=16, setup_iters=1,
                                 costs=[1.0, 0.3, 0.1], mg_precision=16))
    w32, th32, sv32 = _problem("schwinger-16x16", Lx=32, Lt=32, beta=5.0, m0=-0.03, gauge_seed=1002,
                               setup_seed=3002, sweeps=50)
    reqs.append(pkg.make_request(th32, w32.m0, w32.agg, w32.nvec, sv32, 2e-2, 34, k=w32.k,
                                 setup_iters=w32.setup_iters, costs=[1.0, 0.1], mg_precision=16))
    return reqs, (w, th, sv)


def _serve(pkg, reqs, **kw):
    with pkg.Server(**kw) as srv:
        ids = [srv.submit(r) for r in reqs]
        res = [srv.wait(i, 600.0) for i in ids]
        st = srv.stats()
    return res, st


def _same(a, b):
    ra, rb = a["result"], b["result"]
    assert a["status"] == 0 and b["status"] == 0, (a["error"], b["error"])
    assert ra["converged"] == 1 and rb["converged"] == 1
    assert ra["rounds"] == rb["rounds"]
    assert [t["nsamples"] for t in ra["terms"]] == [t["nsamples"] for t in rb["terms"]]
    assert abs(ra["trace"] - rb["trace"]) <= REL * abs(rb["trace"])


def test_results_same_alone_and_in_the_mix(pkg, mix):
    reqs, (w, th, sv) = mix
    alone = [_serve(pkg, [r], max_active=1)[0][0] for r in reqs]
    for a in alone:
        assert a["status"] == 0, a["error"]
        # a fresh server reserves the footprint model's estimate: an upper bound
        assert 0 < a["peak_bytes"] <= a["reserved_bytes"], (a["peak_bytes"], a["reserved_bytes"])
    # the same requests, twice over, all submitted at once on one server
    mixed, st = _serve(pkg, reqs + reqs, max_active=4)
    assert st["max_active_seen"] >= 2 and st["max_reserved"] <= st["budget"]
    assert st["completed"] == 2 * len(reqs) and st["active"] == 0 and st["queued"] == 0
    for i, r in enumerate(mixed):
        _same(r, alone[i % len(reqs)])
    # the served request against the one-context loop of the library on the same inputs
    ctx = pkg.Context(mg_precision=16)
    try:
        ctx.set_gauge(th)
        ctx.set_mass(w.m0)
        ctx.set_hierarchy(w.agg, w.nvec, sv, setup_iters=w.setup_iters, setup_tol=1e-12)
        ctx.compute_deflation(w.k, 1e-9, 400)
        one = ctx.estimate_trace(2e-2, 1 << 40, 31, [1.0, 0.1])
    finally:
        ctx.close()
    _same(alone[0], {"status": 0, "error": "", "result": one})
    # and the estimate against the exact trace of the 16 x 16 operator
    H = ohier.build_hierarchy(th, w.m0, w.agg, w.nvec, sv, w.setup_iters)
    exact = np.trace(np.linalg.inv(H.D[0].toarray()))
    res = alone[0]["result"]
    assert abs(res["trace"] - exact) < 5 * res["rel_err"] * abs(exact)


@pytest.mark.slow
def test_large_request_same_alone_and_in_the_mix(pkg, mix):
    """A 256^2 request shaped like the serving benchmark's (a 3-term sum over 131072 /
    65536 / 16384 unknowns with a solver-only level of 4096 below it, k = 64, BF16
    smoother and deflation) gives the same rounds, sample counts and estimate alone
    and while two small requests run beside it."""
    L = 256
    th = inputs.metropolis_u1(L, L, 5.0, 50, 5266)
    agg = ((4, 4), (2, 2), (2, 2))
    dims = [(L, L, 2), (L // 4, L // 4, 16), (L // 8, L // 8, 16)]
    sv = [inputs.start_vectors(7256, i + 1, lx * lt * d, 8) for i, (lx, lt, d) in enumerate(dims)]
    n0, n1, n2 = 2 * L * L, L * L, L * L // 4
    big = pkg.make_request(th, -0.03, agg, (8, 8, 8), sv, 1e-2, 41, k=64, setup_iters=4, defl_tol=1e-3,
                           defl_max_iters=60, costs=[(n0 + n1) / n0, (n1 + n2) / n0, n2 / n0], mg_precision=16,
                           sum_levels=3)
    alone = _serve(pkg, [big], max_active=1)[0][0]
    assert alone["status"] == 0, alone["error"]
    assert 0 < alone["peak_bytes"] <= alone["reserved_bytes"], (alone["peak_bytes"], alone["reserved_bytes"])
    assert len(alone["result"]["terms"]) == 3
    reqs, _ = mix
    mixed, st = _serve(pkg, [reqs[0], big, reqs[1]], max_active=3)
    assert st["max_active_seen"] >= 2 and st["completed"] == 3
    _same(mixed[1], alone)


def test_admission_under_a_small_budget(pkg, mix):
    reqs, _ = mix
    fp = pkg.request_footprint(reqs[0])
    # room for one request at a time: the three run one after another
    with pkg.Server(hbm_budget=int(1.5 * fp), max_active=4) as srv:
        ids = [srv.submit(reqs[0]) for _ in range(3)]
        res = [srv.wait(i, 600.0) for i in ids]
        st = srv.stats()
        assert st["max_active_seen"] == 1 and st["max_reserved"] <= st["budget"]
        for r in res:
            _same(r, res[0])
            assert r["reserved_bytes"] == fp
        # each was admitted only when the one before it had finished
        assert res[1]["queued_s"] >= res[0]["total_s"] - 0.05
        assert res[2]["queued_s"] >= res[1]["total_s"] - 0.05
        # the next request of this shape reserves 1.1 x the largest peak seen
        peak = max(r["peak_bytes"] for r in res)
        nxt = srv.wait(srv.submit(reqs[0]), 600.0)
        assert nxt["reserved_bytes"] == peak + peak // 10
        _same(nxt, res[0])


def test_cancel_and_refusals(pkg, mix):
    reqs, (w, th, sv) = mix
    fp = pkg.request_footprint(reqs[0])
    with pkg.Server(hbm_budget=int(1.5 * fp), max_active=1) as srv:
        # a queued request is cancelled at once
        a = srv.submit(reqs[0])
        b = srv.submit(reqs[0])
        srv.cancel(b)
        rb = srv.wait(b, 60.0)
        assert rb["status"] == pkg.ECANCELLED
        assert srv.wait(a, 600.0)["status"] == 0
        # a running request stops at its next round
        long = pkg.make_request(th, w.m0, w.agg, w.nvec, sv, 1e-6, 35, k=w.k, setup_iters=w.setup_iters,
                                max_samples=400000, costs=[1.0, 0.1], mg_precision=16)
        c = srv.submit(long)
        t0 = time.time()
        while srv.stats()["active"] == 0 and time.time() - t0 < 60:
            time.sleep(0.01)
        time.sleep(0.3)
        try:
            srv.cancel(c)
        except pkg.MgmlmcError as e:      # it finished first
            assert e.code == -1
        rc = srv.wait(c, 300.0)
        assert rc["status"] in (pkg.ECANCELLED, 0)
        if rc["status"] == pkg.ECANCELLED:
            assert "cancelled" in rc["error"]
        # unknown and finished ids
        with pytest.raises(pkg.MgmlmcError) as e:
            srv.poll(123456)
        assert e.value.code == -1
        with pytest.raises(pkg.MgmlmcError) as e:
            srv.cancel(a)
        assert e.value.code == -1
        # a malformed hierarchy is refused at submission
        bad = pkg.make_request(th, w.m0, [(3, 4)], w.nvec, sv, 1e-2, 1)
        with pytest.raises(pkg.MgmlmcError) as e:
            srv.submit(bad)
        assert e.value.code == -1
    # a request larger than the whole budget is refused at submission
    with pkg.Server(hbm_budget=fp // 2, max_active=1) as srv:
        with pytest.raises(pkg.MgmlmcError) as e:
            srv.submit(reqs[0])
        assert e.value.code == -2
