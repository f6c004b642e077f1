"""Launches shared by many small dense CP jobs (ntf_batch_*).

A batched job runs, in every launch, exactly the work items of its own single-job FP32
launches (same plan, same row blocking, same reduction orders), so after any number of
iterations its factors, iteration count and objective must equal, bit for bit, those of the
same job driven through ntf_jcomm_outer / ntf_cp_mu_sweep on the FP32 path with the same
stopping rule -- whatever else shares the launches.  One iteration is also checked against
the FP64 oracle (1e-5 per factor, the one-sweep bar), and the batch's admission by arena
memory, its capacity, and continuous admission between launches are exercised.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._gpu_util import dev, host, obj_tensor, rel_fro

pytestmark = pytest.mark.gpu


def _ntf():
    import paper_2602_14683_gb300 as ntf
    return ntf


# (dims, rank, beta, method): ragged row tiles and column blocks, ranks in every padding
# class (8, 16, 32, 64), the four special beta values and a general one, both methods
CASES = [
    ((12, 20, 30), 3, 1.0, "jcomm"), ((33, 17, 65), 9, 1.0, "jcomm"), ((40, 130, 70), 20, 1.0, "jcomm"),
    ((21, 35, 18), 5, 0.5, "jcomm"), ((64, 48, 33), 12, 1.5, "jcomm"), ((17, 140, 66), 30, 0.0, "jcomm"),
    ((25, 30, 40), 7, 1.2, "jcomm"), ((19, 23, 29), 40, 1.5, "jcomm"),
    ((30, 22, 50), 6, 1.0, "block"), ((26, 131, 45), 17, 1.0, "block"), ((50, 20, 35), 11, 0.5, "block"),
    ((14, 36, 129), 24, 1.5, "block"), ((16, 18, 20), 4, 0.0, "block"),
]


def _data(q, dims, R):
    X, _ = synth.cp_dense(dims, R, seed=100 + q, kind="uniform_poisson")
    A = synth.init_factors(dims, R, seed=200 + q)
    return X, A


def _alone(ntf, X, A, beta, method, rtol, max_iters):
    """The job through the single-job calls, with the batch's stopping rule."""
    Xd, Ad, obj = dev(X), [dev(a) for a in A], obj_tensor()
    F_prev, F, t = None, None, 0
    while True:
        if method == "jcomm":
            ntf.jcomm_outer(Xd, beta, Ad, objective=obj, precision="fp32")
        else:
            ntf.cp_mu_sweep(Xd, beta, Ad, objective=obj, precision="fp32")
        t += 1
        F_prev, F = F, obj.item()
        if t > 1 and F_prev > 0 and abs(F_prev - F) / F_prev <= rtol:
            break
        if t >= max_iters:
            break
    return [host(a) for a in Ad], t, F


def _check_same(r, got_A, want):
    A1, iters, F = want
    assert r["status"] == 0, r
    assert r["iterations"] == iters, (r["iterations"], iters)
    assert r["objective"] == F, (r["objective"], F)
    for n in range(3):
        assert np.array_equal(host(got_A[n]), A1[n]), n


@pytest.mark.parametrize("rtol,max_iters", [(0.0, 6), (1e-4, 40)])
def test_batched_equals_single_job_calls(rtol, max_iters):
    ntf = _ntf()
    data = [_data(q, d, R) for q, (d, R, _, _) in enumerate(CASES)]
    want = [_alone(ntf, X, A, b, m, rtol, max_iters) for (X, A), (_, _, b, m) in zip(data, CASES)]
    bt = ntf.Batch(capacity=64, mem_budget_bytes=256 << 20)
    got = {}
    for q, ((X, A), (_, _, b, m)) in enumerate(zip(data, CASES)):
        Ad = [dev(a) for a in A]
        jid = bt.add(dev(X), b, Ad, method=m, rtol=rtol, max_iters=max_iters)
        assert jid is not None
        got[jid] = (q, Ad)
    res = bt.run(iters=4)
    bt.close()
    assert len(res) == len(CASES)
    for r in res:
        q, Ad = got[r["id"]]
        _check_same(r, Ad, want[q])


def test_alone_in_batch_equals_in_mix():
    """A job alone in a batch and among the others: identical bits."""
    ntf = _ntf()
    rtol, max_iters = 1e-6, 12
    data = [_data(q, d, R) for q, (d, R, _, _) in enumerate(CASES)]
    alone = {}
    for q, ((X, A), (_, _, b, m)) in enumerate(zip(data, CASES)):
        bt = ntf.Batch(capacity=4, mem_budget_bytes=64 << 20)
        Ad = [dev(a) for a in A]
        bt.add(dev(X), b, Ad, method=m, rtol=rtol, max_iters=max_iters)
        (r,) = bt.run(iters=3)
        bt.close()
        alone[q] = ([host(a) for a in Ad], r["iterations"], r["objective"])
    bt = ntf.Batch(capacity=64, mem_budget_bytes=256 << 20)
    got = {}
    for q, ((X, A), (_, _, b, m)) in enumerate(zip(data, CASES)):
        Ad = [dev(a) for a in A]
        got[bt.add(dev(X), b, Ad, method=m, rtol=rtol, max_iters=max_iters)] = (q, Ad)
    res = bt.run(iters=5)
    bt.close()
    for r in res:
        q, Ad = got[r["id"]]
        _check_same(r, Ad, alone[q])


@pytest.mark.parametrize("method", ["jcomm", "block"])
@pytest.mark.parametrize("beta", [0.5, 1.0, 1.5])
def test_one_batched_iteration_against_oracle(beta, method):
    ntf = _ntf()
    dims, R = (23, 37, 41), 6
    X, _ = synth.cp_dense(dims, R, seed=7, kind="gamma_noise")
    A = synth.init_factors(dims, R, seed=8)
    if method == "jcomm":
        want, F_want = oracle.cp_jcomm_outer(X, A, beta)
    else:
        want, F_want = oracle.cp_mu_sweep(X, A, beta)
    bt = ntf.Batch(capacity=8, mem_budget_bytes=64 << 20)
    # two other jobs share the launches
    others = [(_data(50 + q, (20 + q, 30, 25), 5 + q)) for q in range(2)]
    keep = []
    for Xo, Ao in others:
        Aod = [dev(a) for a in Ao]
        keep.append(Aod)
        bt.add(dev(Xo), 1.5, Aod, max_iters=3)
    Ad = [dev(a) for a in A]
    jid = bt.add(dev(X), beta, Ad, method=method, max_iters=1)
    res = {r["id"]: r for r in bt.run(iters=2)}
    bt.close()
    r = res[jid]
    assert r["status"] == 0 and r["iterations"] == 1
    errs = [rel_fro(host(Ad[n]), want[n]) for n in range(3)]
    assert max(errs) <= 1e-5, errs
    assert abs(r["objective"] - F_want) / F_want <= 1e-5


def test_admission_by_arena_memory_and_capacity():
    ntf = _ntf()
    dims, R = (60, 70, 80), 16
    X, A = _data(0, dims, R)
    Xd = dev(X)
    one = ntf.Batch(capacity=8, mem_budget_bytes=1 << 30)
    Ad = [dev(a) for a in A]
    assert one.add(Xd, 1.0, Ad, max_iters=2) is not None
    one.close()
    bt = ntf.Batch(capacity=2, mem_budget_bytes=64 << 20)
    ids = [bt.add(Xd, 1.0, [dev(a) for a in A], max_iters=2) for _ in range(3)]
    assert ids[0] is not None and ids[1] is not None and ids[2] is None  # capacity 2
    res = bt.run(iters=2)
    assert len(res) == 2 and all(r["status"] == 0 and r["iterations"] == 2 for r in res)
    assert bt.add(Xd, 1.0, [dev(a) for a in A], max_iters=1) is not None  # room again after retirement
    assert len(bt.run()) == 1
    bt.close()
    small = ntf.Batch(capacity=8, mem_budget_bytes=1 << 16)
    assert small.add(Xd, 1.0, [dev(a) for a in A]) is None  # larger than the whole arena
    small.close()


def test_continuous_admission_between_launches():
    """Jobs added while earlier ones run join at their class's next launch; every result is
    still the single-job result."""
    ntf = _ntf()
    rtol, max_iters = 0.0, 7
    data = [_data(q, d, R) for q, (d, R, _, _) in enumerate(CASES)]
    want = [_alone(ntf, X, A, b, m, rtol, max_iters) for (X, A), (_, _, b, m) in zip(data, CASES)]
    bt = ntf.Batch(capacity=64, mem_budget_bytes=256 << 20)
    got, res = {}, []
    for q, ((X, A), (_, _, b, m)) in enumerate(zip(data, CASES)):
        Ad = [dev(a) for a in A]
        got[bt.add(dev(X), b, Ad, method=m, rtol=rtol, max_iters=max_iters)] = (q, Ad)
        bt.tick(iters=2, wait=False)  # earlier jobs keep running while later ones arrive
        res += bt.results()
    res += bt.run(iters=2)
    bt.close()
    assert len(res) == len(CASES)
    for r in res:
        q, Ad = got[r["id"]]
        _check_same(r, Ad, want[q])


def test_batch_rejects_unsupported_jobs():
    ntf = _ntf()
    bt = ntf.Batch(capacity=4, mem_budget_bytes=16 << 20)
    X = dev(np.ones((4, 5, 6)))
    A = [dev(np.ones((d, 2))) for d in (4, 5, 6)]
    with pytest.raises(ntf.NtfError) as e:
        bt.add(X, 2.5, A)
    assert e.value.code == -2
    A65 = [dev(np.ones((d, 65))) for d in (4, 5, 6)]
    with pytest.raises(ntf.NtfError) as e:
        bt.add(X, 1.0, A65)
    assert e.value.code == -8
    assert bt.tick(iters=1) == 0 and bt.results() == []
    bt.close()
