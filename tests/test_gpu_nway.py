"""Dense CP of order N >= 4 (leading modes merged onto the 3-way passes) against the FP64
oracle, which runs the order-N contractions directly.

Bars as for order 3: FP32 path 1e-5 per factor after one sweep / outer iteration and on the
objective, 1e-4 on a 10-sweep objective trajectory; TF32 tensor-core path 1e-3 per factor and
2e-4 on the objective.  Shapes give ragged merged-row tiles, a leading mode of size 1, and
orders 4 to 6.
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


CASES = [
    ((6, 7, 40, 50), 10, "fp32", 1e-5, 1e-5),
    ((1, 5, 33, 24), 7, "fp32", 1e-5, 1e-5),
    ((4, 3, 5, 30, 20), 6, "fp32", 1e-5, 1e-5),
    ((2, 3, 2, 3, 16, 12), 5, "fp32", 1e-5, 1e-5),
    ((8, 9, 64, 48), 32, "tf32", 1e-3, 2e-4),
]


@pytest.mark.parametrize("dims,R,prec,tol,tol_obj", CASES)
@pytest.mark.parametrize("beta", [0.5, 1.0, 1.5])
def test_nway_sweep_parity(dims, R, prec, tol, tol_obj, beta):
    ntf = _ntf()
    X, _ = synth.cp_dense(dims, R, seed=len(dims) + R, kind="gamma_noise")
    A = synth.init_factors(dims, R, seed=R + 1)
    want, F_want = oracle.cp_mu_sweep(X, A, beta)
    Ad, obj = [dev(a) for a in A], obj_tensor()
    ntf.cp_mu_sweep(dev(X), beta, Ad, objective=obj, precision=prec)
    ntf.default_context().device_status()
    errs = [rel_fro(host(Ad[n]), want[n]) for n in range(len(dims))]
    assert max(errs) <= tol, errs
    assert abs(float(obj.item()) - F_want) / F_want <= tol_obj


@pytest.mark.parametrize("dims,R,prec,tol,tol_obj", CASES)
@pytest.mark.parametrize("L", [1, 3])
def test_nway_jcomm_parity(dims, R, prec, tol, tol_obj, L):
    ntf = _ntf()
    X, _ = synth.cp_dense(dims, R, seed=len(dims) + 2 * R, kind="uniform_poisson")
    A = synth.init_factors(dims, R, seed=R + 2)
    want, F_want = oracle.cp_jcomm_outer(X, A, 1.0, L=L)
    Ad, obj = [dev(a) for a in A], obj_tensor()
    ntf.jcomm_outer(dev(X), 1.0, Ad, objective=obj, inner_L=L, precision=prec)
    ntf.default_context().device_status()
    errs = [rel_fro(host(Ad[n]), want[n]) for n in range(len(dims))]
    assert max(errs) <= tol, errs
    assert abs(float(obj.item()) - F_want) / F_want <= tol_obj


@pytest.mark.parametrize("beta", [0.0, 0.5, 1.0, 1.5, 0.3])
def test_nway_beta_div_parity(beta):
    ntf = _ntf()
    dims, R = (5, 6, 7, 41, 30), 6
    X, _ = synth.cp_dense(dims, R, seed=11, kind="uniform_poisson")
    A = synth.init_factors(dims, R, seed=12)
    want = oracle.cp_objective(X, A, beta)
    got = float(ntf.beta_div(dev(X), beta, [dev(a) for a in A]).item())
    assert abs(got - want) / want <= 1e-5


def test_nway_trajectory_10_sweeps():
    """4-way KL, 12 x 10 x 30 x 40, R = 5: objective trajectory over 10 B-CoMM sweeps and
    J-CoMM outer iterations."""
    ntf = _ntf()
    dims, R = (12, 10, 30, 40), 5
    X, _ = synth.cp_dense(dims, R, seed=21, kind="uniform_poisson")
    for step in ("sweep", "jcomm"):
        A = synth.init_factors(dims, R, seed=22)
        Xd, Ad, obj = dev(X), [dev(a) for a in A], obj_tensor()
        worst = 0.0
        for _ in range(10):
            if step == "sweep":
                A, F_o = oracle.cp_mu_sweep(X, A, 1.0)
                ntf.cp_mu_sweep(Xd, 1.0, Ad, objective=obj)
            else:
                A, F_o = oracle.cp_jcomm_outer(X, A, 1.0)
                ntf.jcomm_outer(Xd, 1.0, Ad, objective=obj)
            worst = max(worst, abs(float(obj.item()) - F_o) / F_o)
        assert worst <= 1e-4, (step, worst)


def test_nway_jcomm_beta_other_than_1_rejected():
    ntf = _ntf()
    dims = (2, 3, 8, 8)
    X = dev(np.ones(dims))
    A = [dev(np.ones((d, 3))) for d in dims]
    with pytest.raises(ntf.NtfError) as e:
        ntf.jcomm_outer(X, 0.5, A)
    assert e.value.code == -8
    with pytest.raises(ntf.NtfError) as e:
        ntf.cp_mu_sweep_extrap(X, 1.0, A, [dev(np.ones((d, 3))) for d in dims], 0.5)
    assert e.value.code == -8
