"""Sparse COO tensors at beta != 1 (Section 6.3) against the FP64 oracle on the densified
tensor.

Num^(n) runs over the stored entries only and Den^(n) over the whole index space (a dense
pass that reads no X); the oracle runs the dense updates on the same tensor with its zeros
written out, so any entry the sparse path misses or double-counts shows.  Bars: 1e-5 per
factor and on the objective (the FP32 one-sweep bar).  Shapes: orders 3 to 5 with several
cuts of the modes into three runs, an empty slice (rows with no stored entry: Num = 0, the
factor lands on eps), ranks padded to 32 and 64, and inner L = 1 and 2.
"""
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
    return _ntf().Coo(shape, [torch.tensor(np.asarray(i, dtype=np.int32), device="cuda") for i in idx],
                      torch.tensor(np.asarray(vals, dtype=np.float32), device="cuda"))


def _sparse(seed, dims, density=0.2):
    """Counts 1 + Geometric(0.3) at a random 20% of the entries, one empty slice of mode 2,
    stored in a shuffled order."""
    g = np.random.default_rng(seed)
    X = np.where(g.uniform(size=dims) < density, g.geometric(0.3, size=dims).astype(np.float64), 0.0)
    X[:, min(2, dims[1] - 1)] = 0.0
    idx, vals = synth.coo_from_dense(X)
    perm = g.permutation(len(vals))
    return X, [i[perm] for i in idx], vals[perm]


CASES = [((13, 17, 23), 5, None), ((9, 6, 31, 40), 7, None), ((9, 6, 31, 40), 7, (1, 3)), ((9, 6, 31, 40), 7, (2, 3)),
         ((4, 5, 6, 7, 8), 4, (2, 4)), ((11, 9, 21), 40, None)]


def _opts(merge):
    return {} if merge is None else {"merge": merge}


@pytest.mark.parametrize("dims,R,merge", CASES)
@pytest.mark.parametrize("beta", [0.5, 1.5, 1.2])
def test_coo_beta_block_sweep(dims, R, merge, beta):
    ntf = _ntf()
    X, idx, vals = _sparse(len(dims) + R, dims)
    A = synth.init_factors(dims, R, seed=R)
    want, Fw = oracle.cp_mu_sweep(X, A, beta)
    Ad, obj = [dev(a) for a in A], obj_tensor()
    ntf.cp_mu_sweep(_coo_dev(dims, idx, vals), beta, Ad, objective=obj, **_opts(merge))
    ntf.default_context().device_status()
    errs = [rel_fro(host(Ad[n]), want[n]) for n in range(len(dims))]
    assert max(errs) <= TOL, errs
    assert abs(obj.item() - Fw) / Fw <= TOL


@pytest.mark.parametrize("dims,R,merge", CASES)
@pytest.mark.parametrize("L", [1, 2])
@pytest.mark.parametrize("beta", [0.5, 1.5])
def test_coo_beta_jcomm(dims, R, merge, L, beta):
    ntf = _ntf()
    X, idx, vals = _sparse(3 * len(dims) + R + L, dims)
    A = synth.init_factors(dims, R, seed=R + 1)
    want, Fw = oracle.cp_jcomm_outer(X, A, beta, L=L)
    Ad, obj = [dev(a) for a in A], obj_tensor()
    ntf.jcomm_outer(_coo_dev(dims, idx, vals), beta, Ad, objective=obj, inner_L=L, **_opts(merge))
    ntf.default_context().device_status()
    errs = [rel_fro(host(Ad[n]), want[n]) for n in range(len(dims))]
    assert max(errs) <= TOL, errs
    assert abs(obj.item() - Fw) / Fw <= TOL


@pytest.mark.parametrize("beta", [0.5, 1.5, 1.2, 1.8])
def test_coo_beta_objective(beta):
    ntf = _ntf()
    dims = (9, 6, 31, 40)
    X, idx, vals = _sparse(77, dims)
    A = synth.init_factors(dims, 6, seed=5)
    want = oracle.cp_objective(X, A, beta)
    got = ntf.beta_div(_coo_dev(dims, idx, vals), beta, [dev(a) for a in A]).item()
    assert abs(got - want) / want <= TOL


def test_coo_beta_trajectory_10_iterations():
    """10 J-CoMM outer iterations at beta = 3/2: the objective trajectory within 1e-4."""
    ntf = _ntf()
    dims = (12, 10, 30, 40)
    X, idx, vals = _sparse(5, dims)
    A = synth.init_factors(dims, 5, seed=6)
    Xc, Ad, obj = _coo_dev(dims, idx, vals), [dev(a) for a in A], obj_tensor()
    worst = 0.0
    for _ in range(10):
        A, F_o = oracle.cp_jcomm_outer(X, A, 1.5)
        ntf.jcomm_outer(Xc, 1.5, Ad, objective=obj)
        worst = max(worst, abs(obj.item() - F_o) / F_o)
    assert worst <= 1e-4, worst


def test_coo_beta_rejections():
    ntf = _ntf()
    dims = (9, 6, 31)
    X, idx, vals = _sparse(8, dims)
    A = [dev(a) for a in synth.init_factors(dims, 4, seed=9)]
    Xc = _coo_dev(dims, idx, vals)
    for call in (lambda: ntf.cp_mu_sweep(Xc, 0.0, A), lambda: ntf.jcomm_outer(Xc, 0.0, A),
                 lambda: ntf.beta_div(Xc, 0.0, A)):
        with pytest.raises(ntf.NtfError) as e:
            call()
        assert e.value.code == -8
    _, idx2, vals2 = _sparse(9, (9, 6, 1))
    X2c = _coo_dev((9, 6), idx2[:2], vals2)
    A2 = [dev(a) for a in synth.init_factors((9, 6), 4, seed=9)]
    with pytest.raises(ntf.NtfError) as e:
        ntf.cp_mu_sweep(X2c, 1.5, A2)
    assert e.value.code == -8


TOL_TC, TOL_TC_OBJ = 1e-3, 2e-4


@pytest.mark.parametrize("prec", ["tf32", "3xtf32"])
@pytest.mark.parametrize("method", ["block", "jcomm"])
@pytest.mark.parametrize("beta", [0.5, 1.5, 1.2])
@pytest.mark.parametrize("dims,R", [((13, 17, 23), 5), ((9, 6, 31, 41), 7), ((11, 150, 131), 20)])
def test_coo_beta_tensor_core_dense_pass(dims, R, beta, method, prec):
    """The X-free denominator pass on the tensor cores (TF32 reconstruction, BF16 contraction of
    Q; no X is read, so the last extent need not be a multiple of 4): the tensor-core bars of the
    dense passes, 1e-3 per factor and 2e-4 on the objective."""
    ntf = _ntf()
    X, idx, vals = _sparse(5 * len(dims) + R, dims)
    A = synth.init_factors(dims, R, seed=R + 9)
    if method == "block":
        want, Fw = oracle.cp_mu_sweep(X, A, beta)
    else:
        want, Fw = oracle.cp_jcomm_outer(X, A, beta, L=2)
    Ad, obj = [dev(a) for a in A], obj_tensor()
    Xc = _coo_dev(dims, idx, vals)
    if method == "block":
        ntf.cp_mu_sweep(Xc, beta, Ad, objective=obj, precision=prec)
    else:
        ntf.jcomm_outer(Xc, beta, Ad, objective=obj, inner_L=2, precision=prec)
    ntf.default_context().device_status()
    errs = [rel_fro(host(Ad[n]), want[n]) for n in range(len(dims))]
    assert max(errs) <= TOL_TC, errs
    assert abs(obj.item() - Fw) / Fw <= TOL_TC_OBJ
