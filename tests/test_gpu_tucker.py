"""Parity of the dense Tucker CUDA path (FP32) against the FP64 oracle.

Same bar as CP: one sweep within 1e-5 relative (Frobenius) per block, objective within
1e-5, and the objective trajectory within 1e-4.  Shapes span several 128-row tiles and
64-column blocks with ragged tails, and core sizes that pad to 8 and 16 columns.
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


CASES = [((7, 140, 36), (3, 5, 4)), ((5, 131, 70), (4, 2, 9)), ((6, 30, 20), (6, 7, 5))]


@pytest.mark.parametrize("beta", [0.0, 0.5, 1.0, 1.5])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_tucker_mu_sweep_parity(beta, case):
    ntf = _ntf()
    dims, J = CASES[case]
    X, _, _ = synth.tucker_dense(dims, J, seed=case)
    G0, A0 = synth.init_tucker(dims, J, seed=case + 10)
    Gw, Aw, Fw = oracle.tucker_mu_sweep(X, G0, A0, beta)
    Gd = dev(G0)
    Ad = [dev(a) for a in A0]
    obj = obj_tensor()
    ntf.tucker_mu_sweep(dev(X), beta, Gd, Ad, objective=obj)
    assert rel_fro(host(Gd), Gw) <= TOL
    for n in range(3):
        assert rel_fro(host(Ad[n]), Aw[n]) <= TOL, n
    assert abs(obj.item() - Fw) / Fw <= TOL


@pytest.mark.parametrize("beta", [0.0, 0.5, 1.0, 1.5])
@pytest.mark.parametrize("L", [1, 2])
def test_tucker_jcomm_parity(beta, L):
    ntf = _ntf()
    dims, J = CASES[0]
    X, _, _ = synth.tucker_dense(dims, J, seed=4)
    G0, A0 = synth.init_tucker(dims, J, seed=5)
    Gw, Aw, Fw = oracle.tucker_jcomm_outer(X, G0, A0, beta, L=L)
    Gd = dev(G0)
    Ad = [dev(a) for a in A0]
    obj = obj_tensor()
    ntf.jcomm_outer(dev(X), beta, Ad, core=Gd, objective=obj, inner_L=L)
    assert rel_fro(host(Gd), Gw) <= TOL
    for n in range(3):
        assert rel_fro(host(Ad[n]), Aw[n]) <= TOL, n
    assert abs(obj.item() - Fw) / Fw <= TOL


@pytest.mark.parametrize("beta", [0.0, 1.0, 1.5, 0.8])
def test_tucker_beta_div_parity(beta):
    ntf = _ntf()
    dims, J = CASES[1]
    X, _, _ = synth.tucker_dense(dims, J, seed=7)
    G0, A0 = synth.init_tucker(dims, J, seed=8)
    want = oracle.tucker_objective(X, G0, A0, beta)
    got = ntf.beta_div(dev(X), beta, [dev(a) for a in A0], core=dev(G0)).item()
    assert abs(got - want) / want <= TOL


def test_tucker_trajectory_beta15():
    """beta = 3/2, Poisson-noised Gamma(2,1) Tucker data: 30 sweeps within 1e-4."""
    ntf = _ntf()
    dims, J = (24, 20, 18), (4, 4, 4)
    X, _, _ = synth.tucker_dense(dims, J, seed=11)
    G, A = synth.init_tucker(dims, J, seed=12)
    Gd, Ad = dev(G), [dev(a) for a in A]
    Xd = dev(X)
    obj = obj_tensor()
    worst = 0.0
    for t in range(30):
        G, A, Fo = oracle.tucker_mu_sweep(X, G, A, 1.5)
        ntf.tucker_mu_sweep(Xd, 1.5, Gd, Ad, objective=obj)
        worst = max(worst, abs(obj.item() - Fo) / Fo)
    assert worst <= 1e-4, worst
