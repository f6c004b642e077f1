"""Continuous-batching server: every job's result is the same alone and in the mix.

Each job (CP or Tucker, beta in {1/2, 1, 3/2}, Poisson-noised low-rank data) runs once
alone through the regular C ABI with the server's stopping rule, and once through the
server among the others with slots shared and admissions arriving while others run.  The
kernels, launch shapes and reduction orders of a job depend only on its own shapes, so the
two runs must agree bit for bit; the check allows 1e-6 relative for safety.
"""
import time

import numpy as np
import pytest

import synth
from tests._gpu_util import dev, host, obj_tensor, rel_fro

pytestmark = pytest.mark.gpu


def _ntf():
    import paper_2602_14683_gb300 as ntf
    return ntf


def _jobs(n, seed=5):
    jobs = synth.serving_jobs(n, seed=seed, dim_lo=12, dim_hi=40, rank_lo=3, rank_hi=12)
    return [(j, synth.job_data(j)) for j in jobs]


def _alone(ntf, job, data, rtol, max_iters):
    X, G, A = data
    Xd = dev(X)
    Ad = [dev(a) for a in A]
    Gd = dev(G) if G is not None else None
    obj = obj_tensor()
    F_prev, F = None, None
    t = 0
    while True:
        ntf.jcomm_outer(Xd, job["beta"], Ad, core=Gd, objective=obj)
        t += 1
        F_prev, F = F, obj.item()
        if t > 1 and abs(F_prev - F) / F_prev <= rtol:
            break
        if t >= max_iters:
            break
    return Ad, Gd, t, F


def test_alone_equals_mixed():
    ntf = _ntf()
    import torch
    rtol, max_iters = 1e-6, 60
    jobs = _jobs(14)
    alone = [_alone(ntf, j, d, rtol, max_iters) for j, d in jobs]
    torch.cuda.synchronize()
    srv = ntf.Server(slots=4)
    mixed = {}
    for q, (j, (X, G, A)) in enumerate(jobs):
        Xd = dev(X)
        Ad = [dev(a) for a in A]
        Gd = dev(G) if G is not None else None
        jid = srv.submit(Xd, j["beta"], Ad, core=Gd, rtol=rtol, max_iters=max_iters)
        mixed[jid] = (q, Ad, Gd)
        if q % 5 == 4:
            time.sleep(0.02)  # later arrivals join while earlier jobs run
    res = srv.poll(wait_all=True)
    srv.close()
    assert len(res) == len(jobs)
    for r in res:
        assert r["status"] == 0, r
        q, Ad, Gd = mixed[r["id"]]
        A1, G1, iters, F = alone[q]
        assert r["iterations"] == iters, (q, r["iterations"], iters)
        assert abs(r["objective"] - F) <= 1e-6 * abs(F)
        for n in range(3):
            assert rel_fro(host(Ad[n]), host(A1[n])) <= 1e-6, (q, n)
        if Gd is not None:
            assert rel_fro(host(Gd), host(G1)) <= 1e-6, q
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]


def test_server_rejects_bad_jobs_and_empty_poll():
    ntf = _ntf()
    srv = ntf.Server(slots=2)
    X = dev(np.ones((4, 5, 6)))
    A = [dev(np.ones((d, 2))) for d in (4, 5, 6)]
    with pytest.raises(ntf.NtfError):
        srv.submit(X, 2.5, A)
    assert srv.poll(wait_all=True) == []
    srv.close()


def test_iteration_caps_match_alone():
    """A job capped at 1 or 2 iterations (no WHILE loop / one loop pass) stops exactly
    where the alone loop does."""
    ntf = _ntf()
    import torch
    rtol = 1e-12
    jobs = _jobs(4, seed=9)
    srv = ntf.Server(slots=2)
    for cap in (1, 2, 3):
        alone = [_alone(ntf, j, d, rtol, cap) for j, d in jobs]
        torch.cuda.synchronize()
        mixed = {}
        for q, (j, (X, G, A)) in enumerate(jobs):
            Xd = dev(X)
            Ad = [dev(a) for a in A]
            Gd = dev(G) if G is not None else None
            mixed[srv.submit(Xd, j["beta"], Ad, core=Gd, rtol=rtol, max_iters=cap)] = (q, Ad, Gd)
        res = srv.poll(wait_all=True)
        assert len(res) == len(jobs)
        for r in res:
            q, Ad, Gd = mixed[r["id"]]
            A1, G1, iters, F = alone[q]
            assert r["status"] == 0 and r["iterations"] == iters == cap, (cap, q, r, iters)
            assert abs(r["objective"] - F) <= 1e-6 * abs(F)
            for n in range(3):
                assert rel_fro(host(Ad[n]), host(A1[n])) <= 1e-6, (cap, q, n)
    srv.close()


def test_cp_jobs_larger_than_the_batch_arena_run_in_slots():
    """With a memory budget whose batch arena (half of it) holds no CP job, the CP jobs fall back
    to the slot lane (each job alone there when it exceeds the slots' half too) and still give the
    alone results; Tucker jobs share the slots."""
    ntf = _ntf()
    import torch
    rtol, max_iters = 1e-6, 15
    jobs = _jobs(6, seed=13)
    alone = [_alone(ntf, j, d, rtol, max_iters) for j, d in jobs]
    torch.cuda.synchronize()
    srv = ntf.Server(slots=2, mem_budget_bytes=64 << 10)
    mixed = {}
    for q, (j, (X, G, A)) in enumerate(jobs):
        Xd = dev(X)
        Ad = [dev(a) for a in A]
        Gd = dev(G) if G is not None else None
        mixed[srv.submit(Xd, j["beta"], Ad, core=Gd, rtol=rtol, max_iters=max_iters)] = (q, Ad, Gd)
    res = srv.poll(wait_all=True)
    srv.close()
    assert len(res) == len(jobs)
    for r in res:
        q, Ad, Gd = mixed[r["id"]]
        A1, G1, iters, F = alone[q]
        assert r["status"] == 0 and r["iterations"] == iters, (q, r, iters)
        assert abs(r["objective"] - F) <= 1e-6 * abs(F)
        for n in range(3):
            assert rel_fro(host(Ad[n]), host(A1[n])) <= 1e-6, (q, n)
        if Gd is not None:
            assert rel_fro(host(Gd), host(G1)) <= 1e-6, q
