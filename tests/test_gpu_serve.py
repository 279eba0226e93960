"""Continuous-batching server: mixed sizes, arrivals while others run, every
result checked against the oracle and against the same request solved alone."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2411_10143_b300 import cascade as C
from paper_2411_10143_b300 import models, workloads as W

pytestmark = pytest.mark.gpu


def make_requests():
    mats = [(W.poisson2d(40), 0), (W.poisson3d(12), 0), (W.spd_powerlaw(3000, seed=3), 0),
            (W.convdiff3d(10), 1), (W.poisson3d(40), 0), (W.convdiff3d(36), 1),
            (W.poisson2d(90), 0), (W.spd_powerlaw(40000, seed=4), 0)]
    reqs = []
    rng = np.random.default_rng(0)
    for i in range(24):
        A, s = mats[int(rng.integers(0, len(mats)))]
        reqs.append((i, A, s, oracle.spmv(A, W.vector(A.nrows, 100 + i))))
    return reqs


def test_server_mixed_arrivals_match_oracle_and_alone():
    ctx = C.Context(0)
    models.load_default(ctx)
    reqs = make_requests()
    cache = {}
    loaded = {}
    for _, A, _, _ in reqs:
        if id(A) not in loaded:
            loaded[id(A)] = ctx.load(A)
    srv = C.Server(ctx, lanes=3, small_max_n=8000, max_batch=64, mem_budget=1 << 30)
    xs = {}
    rng = np.random.default_rng(1)
    for rid, A, s, b in reqs:  # arrivals spread over time, others still running
        bd = torch.as_tensor(b, device="cuda")
        xd = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
        xs[rid] = (bd, xd)
        srv.submit(rid, loaded[id(A)], s, bd, xd)
        time.sleep(float(rng.exponential(0.002)))
    srv.drain(300)
    res = {r.id: r for r in srv.poll()}
    assert sorted(res) == [r[0] for r in reqs]
    assert any(r.batched for r in res.values()) and any(not r.batched for r in res.values())
    for rid, A, s, b in reqs:
        r = res[rid]
        x = xs[rid][1].cpu().numpy()
        rel = np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)
        assert r.status == 0 and rel <= 1e-10, (rid, A.name, rel)
        assert r.t_submit_ms <= r.t_start_ms <= r.t_done_ms
        cache[rid] = x
    srv.close()
    # the same requests, each alone in an otherwise idle server
    srv = C.Server(ctx, lanes=1, small_max_n=8000, max_batch=64, mem_budget=1 << 30)
    for rid, A, s, b in reqs[:8]:
        bd = torch.as_tensor(b, device="cuda")
        xd = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
        srv.submit(rid, loaded[id(A)], s, bd, xd)
        srv.drain(300)
        x = xd.cpu().numpy()
        assert np.linalg.norm(x - cache[rid]) <= 1e-7 * np.linalg.norm(cache[rid]), rid
    srv.poll()
    srv.close()
    ctx.close()


def test_server_admission_respects_budget():
    ctx = C.Context(0)
    A = W.poisson3d(30)
    M = ctx.load(A)
    b = torch.as_tensor(oracle.spmv(A, W.vector(A.nrows, 5)), device="cuda")
    # budget below one request's workspace: requests run one at a time, all finish
    srv = C.Server(ctx, lanes=4, small_max_n=100, mem_budget=1 << 20)
    xs = [torch.zeros(A.nrows, dtype=torch.float64, device="cuda") for _ in range(4)]
    for i, x in enumerate(xs):
        srv.submit(i, M, 0, b, x)
    srv.drain(300)
    res = srv.poll()
    assert len(res) == 4 and all(r.status == 0 for r in res)
    spans = sorted((r.t_start_ms, r.t_done_ms) for r in res)
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0 - 1e-6  # never two at once
    srv.close()
    ctx.close()
