"""Sparse COO Tucker (order 3) against the FP64 oracle on the densified tensor.

P = X Xhat^(beta-2) vanishes where X does (Section 6.3), so the numerators are sums over the
stored entries; at beta = 1 (Q = 1) every denominator is a closed form of column sums, at other
beta the denominators contract Q over the whole index space in X-free passes.  The library runs
the stored entries as a 2-way COO tensor with rows (i, j) -> i I2 + j on which
Xhat = B^(3) A3^T (eq. (block_Bn)); the oracle runs the dense Tucker updates with the zeros
written out, so an entry that the sparse path misses or counts twice shows.  Bars: 1e-5 per
block and on the objective (FP32 one-sweep bar), 1e-4 on a 10-iteration trajectory.  Shapes have
empty slices (rows with no stored entry land on eps), cores with J3 padded to 32 and to 64, and a
second tensor of the same sizes to check that a new source rebuilds the cached orders.
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


def _sparse(seed, dims, density=0.15):
    g = np.random.default_rng(seed)
    X = np.where(g.uniform(size=dims) < density, g.geometric(0.3, size=dims).astype(np.float64), 0.0)
    X[:, 1] = 0.0
    X[2, :, :] = 0.0
    idx, vals = synth.coo_from_dense(X)
    perm = g.permutation(len(vals))
    return X, [i[perm] for i in idx], vals[perm]


CASES = [((17, 23, 31), (4, 5, 6)), ((40, 9, 130), (6, 3, 20)), ((12, 14, 70), (5, 4, 40))]


def _check(Gd, Ad, Gw, Aw, obj, Fw, tag):
    errs = [rel_fro(host(Gd), Gw)] + [rel_fro(host(Ad[n]), Aw[n]) for n in range(3)]
    eo = abs(obj.item() - Fw) / Fw
    assert max(errs) <= TOL, (tag, errs)
    assert eo <= TOL, (tag, eo)


@pytest.mark.parametrize("beta", [1.0, 0.5, 1.5])
@pytest.mark.parametrize("dims,J", CASES)
def test_coo_tucker_block_sweep(dims, J, beta):
    ntf = _ntf()
    X, idx, vals = _sparse(sum(dims), dims)
    G0, A0 = synth.init_tucker(dims, J, seed=3)
    Gw, Aw, Fw = oracle.tucker_mu_sweep(X, G0, A0, beta)
    Gd, Ad, obj = dev(G0), [dev(a) for a in A0], obj_tensor()
    ntf.tucker_mu_sweep(_coo_dev(dims, idx, vals), beta, Gd, Ad, objective=obj)
    ntf.default_context().device_status()
    _check(Gd, Ad, Gw, Aw, obj, Fw, "block")


@pytest.mark.parametrize("beta", [1.0, 0.5, 1.5])
@pytest.mark.parametrize("dims,J", CASES)
@pytest.mark.parametrize("L", [1, 2])
def test_coo_tucker_jcomm(dims, J, L, beta):
    ntf = _ntf()
    X, idx, vals = _sparse(2 * sum(dims) + L, dims)
    G0, A0 = synth.init_tucker(dims, J, seed=4)
    Gw, Aw, Fw = oracle.tucker_jcomm_outer(X, G0, A0, beta, L=L)
    Gd, Ad, obj = dev(G0), [dev(a) for a in A0], obj_tensor()
    ntf.jcomm_outer(_coo_dev(dims, idx, vals), beta, Ad, core=Gd, objective=obj, inner_L=L)
    ntf.default_context().device_status()
    _check(Gd, Ad, Gw, Aw, obj, Fw, "jcomm L=%d" % L)


def test_coo_tucker_objective_and_new_source():
    """The objective of different tensors of the same sizes in turn (a call must not reuse another
    tensor's cached orders), at beta = 1 and other beta, each against the oracle."""
    ntf = _ntf()
    dims, J = CASES[0]
    G0, A0 = synth.init_tucker(dims, J, seed=5)
    for seed, beta in ((11, 1.0), (12, 1.0), (11, 1.0), (13, 1.5), (14, 0.5), (13, 1.2)):
        X, idx, vals = _sparse(seed, dims)
        got = ntf.beta_div(_coo_dev(dims, idx, vals), beta, [dev(a) for a in A0], core=dev(G0)).item()
        want = oracle.tucker_objective(X, G0, A0, beta)
        assert abs(got - want) / want <= TOL, (seed, beta, got, want)


def test_coo_tucker_trajectory_10_iterations():
    ntf = _ntf()
    dims, J = CASES[1]
    X, idx, vals = _sparse(21, dims)
    G, A = synth.init_tucker(dims, J, seed=6)
    Xc = _coo_dev(dims, idx, vals)
    Gd, Ad, obj = dev(G), [dev(a) for a in A], obj_tensor()
    worst = 0.0
    for _ in range(10):
        G, A, F_o = oracle.tucker_jcomm_outer(X, G, A, 1.0)
        ntf.jcomm_outer(Xc, 1.0, Ad, core=Gd, objective=obj)
        worst = max(worst, abs(obj.item() - F_o) / F_o)
    assert worst <= 1e-4, worst


def test_coo_tucker_rejections():
    ntf = _ntf()
    dims, J = CASES[0]
    X, idx, vals = _sparse(31, dims)
    G0, A0 = synth.init_tucker(dims, J, seed=7)
    Xc = _coo_dev(dims, idx, vals)
    with pytest.raises(ntf.NtfError) as e:  # beta = 0 needs x > 0 everywhere
        ntf.tucker_mu_sweep(Xc, 0.0, dev(G0), [dev(a) for a in A0])
    assert e.value.code == -8
    d4 = dims + (3,)
    X4 = np.zeros(d4)
    X4[0, 0, 0, 0] = 1.0
    i4, v4 = synth.coo_from_dense(X4)
    G4, A4 = synth.init_tucker(d4, J + (2,), seed=8)
    with pytest.raises(ntf.NtfError) as e:
        ntf.tucker_mu_sweep(_coo_dev(d4, i4, v4), 1.0, dev(G4), [dev(a) for a in A4])
    assert e.value.code == -8
