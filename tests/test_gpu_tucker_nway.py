"""Dense Tucker of order N >= 4 (modes cut into three runs on the 3-way passes, Kronecker
factors for runs of several modes) against the FP64 oracle, which runs the order-N Tucker
contractions directly.

Bars as for order 3: FP32 path 1e-5 per block (core and every factor) after one block sweep /
J-CoMM outer iteration and on the objective, 1e-4 on an 8-sweep objective trajectory; TF32
tensor-core passes 1e-3 per block and 2e-4 on the objective.  Every cut of a 4-way tensor, two
runs of two modes at order 5, three at order 6, and the cut the library picks.
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
    ((8, 7, 6, 5), (3, 2, 3, 2), None),
    ((8, 7, 6, 5), (3, 2, 3, 2), (1, 2)),
    ((8, 7, 6, 5), (3, 2, 3, 2), (1, 3)),
    ((8, 7, 6, 5), (3, 2, 3, 2), (2, 3)),
    ((4, 3, 5, 4, 6), (2, 2, 3, 2, 3), (2, 4)),
    ((2, 3, 4, 3, 4, 4), (2, 2, 2, 2, 2, 2), (2, 4)),
]


def _check(Gd, Ad, Gw, Aw, obj, Fw, tol, tol_obj):
    errs = [rel_fro(host(Gd), Gw)] + [rel_fro(host(Ad[n]), Aw[n]) for n in range(len(Aw))]
    assert max(errs) <= tol, errs
    assert abs(obj.item() - Fw) / Fw <= tol_obj


@pytest.mark.parametrize("dims,J,merge", CASES)
@pytest.mark.parametrize("beta", [0.5, 1.0, 1.5])
def test_tucker_nway_sweep_parity(dims, J, merge, beta):
    ntf = _ntf()
    X, _, _ = synth.tucker_dense(dims, J, seed=len(dims) + 1)
    G0, A0 = synth.init_tucker(dims, J, seed=len(dims) + 2)
    Gw, Aw, Fw = oracle.tucker_mu_sweep(X, G0, A0, beta)
    Gd, Ad, obj = dev(G0), [dev(a) for a in A0], obj_tensor()
    ntf.tucker_mu_sweep(dev(X), beta, Gd, Ad, objective=obj, merge=merge)
    _check(Gd, Ad, Gw, Aw, obj, Fw, 1e-5, 1e-5)


@pytest.mark.parametrize("dims,J,merge", CASES)
@pytest.mark.parametrize("beta", [0.5, 1.0, 1.5])
@pytest.mark.parametrize("L", [1, 2])
def test_tucker_nway_jcomm_parity(dims, J, merge, beta, L):
    ntf = _ntf()
    X, _, _ = synth.tucker_dense(dims, J, seed=len(dims) + 3)
    G0, A0 = synth.init_tucker(dims, J, seed=len(dims) + 4)
    Gw, Aw, Fw = oracle.tucker_jcomm_outer(X, G0, A0, beta, L=L)
    Gd, Ad, obj = dev(G0), [dev(a) for a in A0], obj_tensor()
    ntf.jcomm_outer(dev(X), beta, Ad, core=Gd, objective=obj, inner_L=L, merge=merge)
    _check(Gd, Ad, Gw, Aw, obj, Fw, 1e-5, 1e-5)


@pytest.mark.parametrize("beta", [0.5, 1.0, 1.5])
@pytest.mark.parametrize("step", ["sweep", "jcomm"])
def test_tucker_nway_tc_parity(beta, step):
    """Last run (modes 3, 4) with core extent 4 x 5 = 20 (padded to 32) and 8 x 12 = 96
    columns: the tensor-core rows and mode-3 passes."""
    ntf = _ntf()
    dims, J = (6, 5, 8, 12), (3, 2, 4, 5)
    X, _, _ = synth.tucker_dense(dims, J, seed=50)
    G0, A0 = synth.init_tucker(dims, J, seed=51)
    if step == "sweep":
        Gw, Aw, Fw = oracle.tucker_mu_sweep(X, G0, A0, beta)
    else:
        Gw, Aw, Fw = oracle.tucker_jcomm_outer(X, G0, A0, beta, L=2)
    Gd, Ad, obj = dev(G0), [dev(a) for a in A0], obj_tensor()
    if step == "sweep":
        ntf.tucker_mu_sweep(dev(X), beta, Gd, Ad, objective=obj, merge=(1, 2), precision="tf32")
    else:
        ntf.jcomm_outer(dev(X), beta, Ad, core=Gd, objective=obj, inner_L=2, merge=(1, 2), precision="tf32")
    ntf.default_context().device_status()
    _check(Gd, Ad, Gw, Aw, obj, Fw, 1e-3, 2e-4)


@pytest.mark.parametrize("beta", [0.5, 1.0, 1.5])
def test_tucker_5way_uber_like_tc_parity(beta):
    """Order 5 with the structure of the paper's Uber Tucker fit (ranks 2,2,3,3,6 here): runs
    {0,1}, {2,3}, {4}; last core extent 6 padded to 32 for the tensor-core passes; mostly-zero
    count data."""
    ntf = _ntf()
    dims, J = (6, 5, 7, 16, 24), (2, 2, 3, 3, 6)
    g = np.random.default_rng(80)
    X = np.float32(g.poisson(0.05, size=dims) * (1 + g.geometric(0.3, size=dims))).astype(np.float64)
    G0, A0 = synth.init_tucker(dims, J, seed=81)
    for step in ("sweep", "jcomm"):
        if step == "sweep":
            Gw, Aw, Fw = oracle.tucker_mu_sweep(X, G0, A0, beta)
        else:
            Gw, Aw, Fw = oracle.tucker_jcomm_outer(X, G0, A0, beta, L=2)
        Gd, Ad, obj = dev(G0), [dev(a) for a in A0], obj_tensor()
        if step == "sweep":
            ntf.tucker_mu_sweep(dev(X), beta, Gd, Ad, objective=obj, merge=(2, 4), precision="tf32")
        else:
            ntf.jcomm_outer(dev(X), beta, Ad, core=Gd, objective=obj, inner_L=2, merge=(2, 4), precision="tf32")
        ntf.default_context().device_status()
        _check(Gd, Ad, Gw, Aw, obj, Fw, 1e-3, 2e-4)


@pytest.mark.parametrize("beta", [0.0, 0.5, 1.0, 1.5, 0.3])
def test_tucker_nway_beta_div_parity(beta):
    ntf = _ntf()
    dims, J = (5, 6, 4, 7, 3), (2, 3, 2, 3, 2)
    X, _, _ = synth.tucker_dense(dims, J, seed=60)
    G0, A0 = synth.init_tucker(dims, J, seed=61)
    want = oracle.tucker_objective(X, G0, A0, beta)
    got = float(ntf.beta_div(dev(X), beta, [dev(a) for a in A0], core=dev(G0)).item())
    assert abs(got - want) / want <= 1e-5


def test_tucker_nway_trajectory_8_sweeps():
    """4-way, 10 x 9 x 8 x 7, core 3 x 3 x 2 x 2, beta = 1/2: objective trajectory over 8 block
    sweeps and 8 J-CoMM outer iterations."""
    ntf = _ntf()
    dims, J = (10, 9, 8, 7), (3, 3, 2, 2)
    X, _, _ = synth.tucker_dense(dims, J, seed=70)
    for step in ("sweep", "jcomm"):
        G, A = synth.init_tucker(dims, J, seed=71)
        Xd, Gd, Ad, obj = dev(X), dev(G), [dev(a) for a in A], obj_tensor()
        worst = 0.0
        for _ in range(8):
            if step == "sweep":
                G, A, F_o = oracle.tucker_mu_sweep(X, G, A, 0.5)
                ntf.tucker_mu_sweep(Xd, 0.5, Gd, Ad, objective=obj)
            else:
                G, A, F_o = oracle.tucker_jcomm_outer(X, G, A, 0.5)
                ntf.jcomm_outer(Xd, 0.5, Ad, core=Gd, objective=obj)
            worst = max(worst, abs(obj.item() - F_o) / F_o)
        assert worst <= 1e-4, (step, worst)


def test_tucker_nway_rejects():
    """Extrapolated Tucker entries stay order 3; a cut whose last run's core extent exceeds 64
    is refused."""
    ntf = _ntf()
    dims, J = (6, 5, 9, 9), (2, 2, 9, 9)
    X = dev(np.ones(dims))
    G = dev(np.ones(J))
    A = [dev(np.ones((d, j))) for d, j in zip(dims, J)]
    with pytest.raises(ntf.NtfError) as e:
        ntf.tucker_mu_sweep(X, 1.0, G, A, merge=(1, 2))
    assert e.value.code == -8
    with pytest.raises(ntf.NtfError) as e:
        ntf.tucker_mu_sweep_extrap(X, 1.0, G, A, dev(np.ones(J)), [dev(np.ones((d, j))) for d, j in zip(dims, J)], 0.5)
    assert e.value.code == -8
