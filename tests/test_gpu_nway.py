"""Dense CP of order N >= 4 (leading modes merged onto the 3-way passes) against the FP64
oracle, which runs the order-N contractions directly.

Bars as for order 3: FP32 path 1e-5 per factor after one sweep / outer iteration (inner
L = 1 and 3, beta in {1/2, 1, 3/2}) and on the objective, 1e-4 on a 10-sweep objective trajectory; TF32 tensor-core path 1e-3 per factor and
2e-4 on the objective.  Shapes give ragged merged-row tiles, a leading mode of size 1, and
orders 4 to 8.
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
    ((2, 2, 3, 2, 2, 3, 8, 12), 4, "fp32", 1e-5, 1e-5),
    ((8, 9, 64, 48), 32, "tf32", 1e-3, 2e-4),
    ((6, 7, 40, 52), 10, "tf32", 1e-3, 2e-4),
]

# every cut of a 4-way tensor into three runs, and a 6-way cut into three runs of two
MERGES = [((6, 7, 24, 20), (1, 2)), ((6, 7, 24, 20), (1, 3)), ((6, 7, 24, 20), (2, 3)),
          ((2, 3, 4, 3, 4, 4), (2, 4)), ((5, 3, 4, 6, 8), (1, 4))]


@pytest.mark.parametrize("dims,R,prec,tol,tol_obj", CASES)
@pytest.mark.parametrize("beta", [0.0, 0.5, 1.0, 1.5, 1.2])
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
@pytest.mark.parametrize("beta", [0.5, 1.0, 1.5])
def test_nway_jcomm_parity(dims, R, prec, tol, tol_obj, L, beta):
    ntf = _ntf()
    X, _ = synth.cp_dense(dims, R, seed=len(dims) + 2 * R, kind="uniform_poisson")
    A = synth.init_factors(dims, R, seed=R + 2)
    want, F_want = oracle.cp_jcomm_outer(X, A, beta, L=L)
    Ad, obj = [dev(a) for a in A], obj_tensor()
    ntf.jcomm_outer(dev(X), beta, Ad, objective=obj, inner_L=L, precision=prec)
    ntf.default_context().device_status()
    errs = [rel_fro(host(Ad[n]), want[n]) for n in range(len(dims))]
    assert max(errs) <= tol, errs
    assert abs(float(obj.item()) - F_want) / F_want <= tol_obj


@pytest.mark.parametrize("dims,merge", MERGES)
@pytest.mark.parametrize("prec,R,tol,tol_obj", [("fp32", 10, 1e-5, 1e-5), ("tf32", 20, 3e-3, 2e-4)])
@pytest.mark.parametrize("beta", [0.5, 1.0, 1.5])
def test_nway_merge_choices(dims, merge, prec, R, tol, tol_obj, beta):
    """Explicit cuts of the modes into the three runs of the 3-way view: B-CoMM sweep and
    J-CoMM with two inner sweeps.  Tensor-core bar 3e-3: these 3-way views have 6 to 48 rows
    per mode, and the BF16 rounding of a factor operand (unit roundoff u = 2^-8, 8 significand
    bits) is shared by every term that uses that row, so it averages over a few rows only:
    about u / sqrt(rows) = 1.6e-3 per column at 6 rows, sqrt(2) times that (2.3e-3) for the two
    independently rounded operands of a contraction.  The per-factor Frobenius error averages
    these per-entry errors over the factor's rows and columns, which keeps it under the 3e-3
    bar over two inner sweeps; the other parity cases have 150+ rows per mode."""
    ntf = _ntf()
    X, _ = synth.cp_dense(dims, R, seed=sum(merge) + R, kind="gamma_noise")
    A = synth.init_factors(dims, R, seed=R + 7)
    Xd = dev(X)
    for step in ("sweep", "jcomm"):
        if step == "sweep":
            want, F_want = oracle.cp_mu_sweep(X, A, beta)
        else:
            want, F_want = oracle.cp_jcomm_outer(X, A, beta, L=2)
        Ad, obj = [dev(a) for a in A], obj_tensor()
        if step == "sweep":
            ntf.cp_mu_sweep(Xd, beta, Ad, objective=obj, precision=prec, merge=merge)
        else:
            ntf.jcomm_outer(Xd, beta, Ad, objective=obj, precision=prec, merge=merge, inner_L=2)
        ntf.default_context().device_status()
        errs = [rel_fro(host(Ad[n]), want[n]) for n in range(len(dims))]
        assert max(errs) <= tol, (step, errs)
        assert abs(float(obj.item()) - F_want) / F_want <= tol_obj, step
    got = float(ntf.beta_div(Xd, beta, [dev(a) for a in A], merge=merge).item())
    assert abs(got - oracle.cp_objective(X, A, beta)) / got <= 1e-5


def test_nway_bad_merge_rejected():
    ntf = _ntf()
    dims = (2, 3, 8, 8)
    X = dev(np.ones(dims))
    A = [dev(np.ones((d, 3))) for d in dims]
    for merge in ((0, 2), (2, 2), (3, 4), (2, 1)):
        with pytest.raises(ntf.NtfError) as e:
            ntf.cp_mu_sweep(X, 1.0, A, merge=merge)
        assert e.value.code == -1


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


def test_nway_extrap_rejected():
    """The extrapolated entries implement order 3 only."""
    ntf = _ntf()
    dims = (2, 3, 8, 8)
    X = dev(np.ones(dims))
    A = [dev(np.ones((d, 3))) for d in dims]
    with pytest.raises(ntf.NtfError) as e:
        ntf.cp_mu_sweep_extrap(X, 1.0, A, [dev(np.ones((d, 3))) for d in dims], 0.5)
    assert e.value.code == -8
