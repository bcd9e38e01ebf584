"""Serving loop with continuous batching: queries (select and spread) arrive
over time, from several threads, over a resident pool of graphs, and every
result equals the same query run alone (the blocking entry points, which are
checked against the oracle elsewhere, and the oracle itself for a sample),
whatever else was on the device with it; admission respects the memory
budget."""
import threading
import time

import numpy as np
import pytest

import oracle
import paper_2008_03095_gb300 as im
from paper_2008_03095_gb300 import build as im_build
from paper_2008_03095_gb300 import synth

pytestmark = pytest.mark.gpu

SEL, SPR = im.IM_REQUEST_SELECT, im.IM_REQUEST_SPREAD


@pytest.fixture(scope="module", autouse=True)
def _lib():
    im_build.build()
    im.lib()


@pytest.fixture(scope="module")
def pool():
    specs = [synth.chung_lu(800, 3200, 2.3, 71), synth.chung_lu(3000, 15000, 2.1, 72),
             synth.random_graph(500, 1500, 73), synth.chung_lu(12000, 60000, 2.4, 74),
             synth.workload_graph("powerlaw_n2000"), synth.chung_lu(6000, 40000, 2.2, 75)]
    ws = [synth.edge_weights(x, a, "uniform", i) for i, (x, a) in enumerate(specs)]
    handles = [im.im_graph_create_weighted(x, a, w) for (x, a), w in zip(specs, ws)]
    yield specs, ws, handles
    for g in handles:
        g.close()


def _stream(rng, specs, count):
    out = []
    for _ in range(count):
        gi = int(rng.integers(0, len(specs)))
        n = specs[gi][0].shape[0] - 1
        R = int(rng.choice([32, 256, 1024]))
        p = float(np.exp(rng.uniform(np.log(0.001), np.log(0.1))))
        flags = int(rng.choice([0, 0, 0, im.IM_SAMPLE_EDGE_WEIGHTS, im.IM_SAMPLE_MIXED_HASH]))
        if rng.random() < 0.7:
            out.append(dict(kind=SEL, graph=gi, K=int(min(rng.integers(5, 60), n)), R=R, p=p,
                            rng_seed=int(rng.integers(0, 1 << 31)), flags=flags))
        else:
            k = int(min(rng.integers(1, 60), n))
            out.append(dict(kind=SPR, graph=gi, R=R, p=p, rng_seed=int(rng.integers(0, 1 << 31)),
                            flags=flags, seeds=rng.choice(n, size=k, replace=False)))
    return out


def _alone(handles, q):
    g = handles[q["graph"]]
    if q["kind"] == SEL:
        return im.im_select_seeds_ex(g, q["K"], q["R"], q["p"], q["rng_seed"], q["flags"])
    return im.im_estimate_spread_ex(g, q["seeds"], q["R"], q["p"], q["rng_seed"], q["flags"])


def _submit(sv, q):
    return im.im_server_submit(sv, q["kind"], q["graph"], q.get("K", 0), q["R"], q["p"],
                               q["rng_seed"], q["flags"], q.get("seeds"))


def _same(q, got, want):
    if q["kind"] == SEL:
        return np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    return got[1] == want


def test_poisson_arrivals_every_result_equals_its_solo_run(pool):
    specs, ws, handles = pool
    rng = np.random.default_rng(5)
    qs = _stream(rng, specs, 160)
    sv = im.im_server_create(handles, slots=8, memory_budget=8 << 30)
    tickets = []
    for q in qs:  # about 2000 queries/s offered
        tickets.append(_submit(sv, q))
        time.sleep(float(rng.exponential(0.0005)))
    results = [im.im_server_wait(sv, t) for t in tickets]
    stats = im.im_server_stats(sv)
    sv.close()
    assert stats["completed"] == len(qs) and stats["in_flight_peak"] > 1, stats
    for q, r in zip(qs, results):
        assert _same(q, r, _alone(handles, q)), q
        sub, adm, done = r[2]
        assert sub <= adm <= done
    # a sample against the oracle directly
    for q, r in list(zip(qs, results))[:6]:
        x, a = specs[q["graph"]]
        kw = dict(weights=ws[q["graph"]] if q["flags"] & im.IM_SAMPLE_EDGE_WEIGHTS else None,
                  mix=bool(q["flags"] & im.IM_SAMPLE_MIXED_HASH))
        if q["kind"] == SEL:
            es, eg = oracle.select_seeds_ex(x, a, q["K"], q["R"], q["p"], q["rng_seed"], **kw)
            assert np.array_equal(r[0], es) and np.array_equal(r[1], eg)
        else:
            assert r[1] == oracle.estimate_spread_ex(x, a, q["seeds"], q["R"], q["p"],
                                                     q["rng_seed"], **kw)


def test_several_submitting_threads(pool):
    specs, ws, handles = pool
    sv = im.im_server_create(handles, slots=4, memory_budget=8 << 30)
    qs = _stream(np.random.default_rng(6), specs, 90)
    out = [None] * len(qs)
    errors = []

    def client(idx):
        try:
            for i in idx:
                t = _submit(sv, qs[i])
                out[i] = im.im_server_wait(sv, t)
        except Exception as e:  # noqa: BLE001
            errors.append(e)

    th = [threading.Thread(target=client, args=(range(k, len(qs), 3),)) for k in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    sv.close()
    assert not errors, errors
    for q, r in zip(qs, out):
        assert _same(q, r, _alone(handles, q))


def test_memory_budget_bounds_the_pool_and_evicts(pool):
    specs, ws, handles = pool
    # a workspace of the 12,000-vertex graph at R = 1024 takes about 58 MB: the
    # 80 MB budget cannot hold it beside the others, so idle ones are freed
    big = 3
    qs = [dict(kind=SEL, graph=gi, K=20, R=1024, p=0.02, rng_seed=9, flags=0)
          for gi in (big, 1, 5, big, 0, 5, 1, big)]
    sv = im.im_server_create(handles, slots=6, memory_budget=80 << 20)
    tickets = [_submit(sv, q) for q in qs]
    res = [im.im_server_wait(sv, t) for t in tickets]
    stats = im.im_server_stats(sv)
    sv.close()
    assert stats["pool_bytes_peak"] <= stats["budget"]
    assert stats["ws_evicted"] >= 1, stats
    for q, r in zip(qs, res):
        assert _same(q, r, _alone(handles, q))


def test_rejections(pool):
    specs, ws, handles = pool
    sv = im.im_server_create(handles, slots=2, memory_budget=64 << 20)
    with pytest.raises(im.IMError) as e:  # its workspace alone is larger than the budget
        _submit(sv, dict(kind=SEL, graph=3, K=5, R=4096, p=0.01, rng_seed=1, flags=0))
    assert e.value.code == im.IM_ENOMEM
    for bad in (dict(kind=SEL, graph=9, K=5, R=64, p=0.01, rng_seed=1, flags=0),
                dict(kind=SEL, graph=0, K=0, R=64, p=0.01, rng_seed=1, flags=0),
                dict(kind=SEL, graph=0, K=5, R=64, p=2.0, rng_seed=1, flags=0),
                dict(kind=SPR, graph=0, R=64, p=0.1, rng_seed=1, flags=0, seeds=[800]),
                dict(kind=SEL, graph=0, K=5, R=64, p=0.1, rng_seed=1,
                     flags=im.IM_ALGO_FUSED_SAMPLING)):
        with pytest.raises(im.IMError) as e:
            _submit(sv, bad)
        assert e.value.code == im.IM_EINVAL
    # polling: a query either is done or reports IM_EBUSY and stays waitable
    t = _submit(sv, dict(kind=SEL, graph=1, K=30, R=1024, p=0.05, rng_seed=3, flags=0))
    try:
        im.im_server_wait(sv, t, timeout_us=0)
    except im.IMError as e:
        assert e.code == im.IM_EBUSY
        im.im_server_wait(sv, t)
    sv.close()
