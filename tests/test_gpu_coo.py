"""Sparse COO path (KL) against the FP64 oracle, and the per-mode stable permutation
bit-exact against the oracle's counting sort."""
import numpy as np
import pytest

import oracle
import synth
from tests._gpu_util import dev, host, obj_tensor, rel_fro

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _ntf():
    import paper_2602_14683_gb300 as ntf
    return ntf


def _coo_dev(shape, idx, vals):
    import torch
    ntf = _ntf()
    return ntf.Coo(shape, [torch.tensor(np.asarray(i, dtype=np.int32), device="cuda") for i in idx],
                   torch.tensor(np.asarray(vals, dtype=np.float32), device="cuda"))


@pytest.mark.parametrize("n,K", [(1, 1), (1000, 7), (50000, 24), (100000, 1717), (70000, 5000), (3000, 3000000)])
def test_stable_perm_bit_exact(n, K):
    import torch
    ntf = _ntf()
    g = np.random.default_rng(n + K)
    keys = g.integers(0, K, size=n).astype(np.int32)
    got = ntf.coo_stable_perm(torch.tensor(keys, device="cuda"), K).cpu().numpy()
    want = oracle.stable_perm(keys, K)
    assert np.array_equal(got.astype(np.int64), want)


def _small_coo(seed, dims=(9, 6, 31, 40), density=0.15):
    g = np.random.default_rng(seed)
    X = np.where(g.uniform(size=dims) < density, 1.0 + g.geometric(0.3, size=dims) - 1.0, 0.0)
    X[:, 2] = 0.0  # an empty slice: its rows have no stored entries (Num = 0 -> eps)
    idx, vals = synth.coo_from_dense(X)
    perm = g.permutation(len(vals))
    return dims, [i[perm] for i in idx], vals[perm]


@pytest.mark.parametrize("R", [5, 32, 40])
@pytest.mark.parametrize("L", [1, 2])
def test_coo_jcomm_parity(R, L):
    ntf = _ntf()
    dims, idx, vals = _small_coo(R + L)
    A = synth.init_factors(dims, R, seed=3)
    want, Fw = oracle.coo_kl_jcomm_outer(dims, idx, vals, A, L=L)
    Ad = [dev(a) for a in A]
    obj = obj_tensor()
    ntf.jcomm_outer(_coo_dev(dims, idx, vals), 1.0, Ad, objective=obj, inner_L=L)
    for n in range(len(dims)):
        assert rel_fro(host(Ad[n]), want[n]) <= TOL, n
    assert abs(obj.item() - Fw) / abs(Fw) <= TOL


@pytest.mark.parametrize("R", [8, 33])
def test_coo_block_mu_parity(R):
    ntf = _ntf()
    dims, idx, vals = _small_coo(10 + R)
    A = synth.init_factors(dims, R, seed=4)
    want, Fw = oracle.coo_kl_mu_sweep(dims, idx, vals, A)
    Ad = [dev(a) for a in A]
    obj = obj_tensor()
    ntf.cp_mu_sweep(_coo_dev(dims, idx, vals), 1.0, Ad, objective=obj)
    for n in range(len(dims)):
        assert rel_fro(host(Ad[n]), want[n]) <= TOL, n
    assert abs(obj.item() - Fw) / abs(Fw) <= TOL


def test_coo_objective_and_is_rejected():
    ntf = _ntf()
    dims, idx, vals = _small_coo(21)
    A = synth.init_factors(dims, 6, seed=5)
    want = oracle.coo_kl_objective(dims, idx, vals, A)
    X = _coo_dev(dims, idx, vals)
    got = ntf.beta_div(X, 1.0, [dev(a) for a in A]).item()
    assert abs(got - want) / abs(want) <= TOL
    with pytest.raises(ntf.NtfError) as e:  # beta = 0 needs x > 0 everywhere
        ntf.jcomm_outer(X, 0.0, [dev(a) for a in A])
    assert e.value.code == -8


def test_coo_full_size_jcomm():
    """183 x 24 x 1140 x 1717, 3.3M nonzeros, R = 32: one J-CoMM outer iteration, every
    factor against the oracle, and the permutation of the largest mode bit-exact."""
    import torch
    ntf = _ntf()
    dims = (183, 24, 1140, 1717)
    idx, vals = synth.coo_counts(dims, 3_300_000, seed=0)
    A = synth.init_factors(dims, 32, seed=1)
    want, Fw = oracle.coo_kl_jcomm_outer(dims, idx, vals, A, L=1)
    Ad = [dev(a) for a in A]
    obj = obj_tensor()
    X = _coo_dev(dims, idx, vals)
    ntf.jcomm_outer(X, 1.0, Ad, objective=obj)
    for n in range(4):
        assert rel_fro(host(Ad[n]), want[n]) <= TOL, n
    assert abs(obj.item() - Fw) / abs(Fw) <= TOL
    perm = ntf.coo_stable_perm(X.idx[3], dims[3]).cpu().numpy()
    assert np.array_equal(perm.astype(np.int64), oracle.stable_perm(idx[3], dims[3]))
    torch.cuda.synchronize()
