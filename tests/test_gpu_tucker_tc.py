"""Tensor-core (tcgen05) dense Tucker passes against the FP64 oracle.

The rows pass (W = P A3n, Wd = Q A3d written per 128-column block and summed in block order)
and the mode-3 pass run on the tensor cores when the precision is "tf32" or "3xtf32", the
third core dimension is at most 32 (padded to 32) and I3 % 4 == 0 (at beta = 1 the passes carry
no denominator side: Q = 1 makes those sums column sums).  Their arithmetic is
that of the CP tensor-core pass (TF32 or split-TF32 reconstruction from the rows of the
partial tensor B^(3), BF16 contraction operands, FP32 accumulation, FP32 powers, FP64
objective sum), so the same bars apply: 1e-3 per block after one sweep and 2e-4 on the
objective (the derivation is in test_gpu_tc.py).  Shapes span several 128-row tiles and
128-column blocks with ragged tails.  When 128 divides I1 I2 the passes cut the rows i I2 + j into
slabs of exactly 128 that straddle the i boundaries (the third case: I2 = 96 < 128, I1 I2 = 9 x 128).
"""
import numpy as np
import pytest

import oracle
import synth
from tests._gpu_util import dev, host, obj_tensor, rel_fro

pytestmark = pytest.mark.gpu
TOL_TC = 1e-3
TOL_TC_OBJ = 2e-4

CASES = [((6, 140, 132), (3, 4, 20)), ((5, 131, 264), (4, 3, 32)), ((12, 96, 200), (4, 5, 28))]


def _ntf():
    import paper_2602_14683_gb300 as ntf
    return ntf


def _check(Gd, Ad, Gw, Aw, obj, Fw, tag):
    errs = [rel_fro(host(Gd), Gw)] + [rel_fro(host(Ad[n]), Aw[n]) for n in range(3)]
    eo = abs(obj.item() - Fw) / Fw
    print("%s block errs=%s obj err=%.2e" % (tag, ["%.1e" % e for e in errs], eo))
    assert max(errs) <= TOL_TC, errs
    assert eo <= TOL_TC_OBJ, eo


@pytest.mark.parametrize("prec", ["tf32", "3xtf32"])
@pytest.mark.parametrize("beta", [0.0, 0.5, 1.0, 1.5, 1.2])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_tucker_tc_sweep_parity(beta, case, prec):
    ntf = _ntf()
    dims, J = CASES[case]
    X, _, _ = synth.tucker_dense(dims, J, seed=case + 20)
    G0, A0 = synth.init_tucker(dims, J, seed=case + 30)
    Gw, Aw, Fw = oracle.tucker_mu_sweep(X, G0, A0, beta)
    Gd, Ad, obj = dev(G0), [dev(a) for a in A0], obj_tensor()
    ntf.tucker_mu_sweep(dev(X), beta, Gd, Ad, objective=obj, precision=prec)
    ntf.default_context().device_status()
    _check(Gd, Ad, Gw, Aw, obj, Fw, "tucker tc %s sweep beta=%g %s" % (prec, beta, dims))


@pytest.mark.parametrize("prec", ["tf32", "3xtf32"])
@pytest.mark.parametrize("beta", [0.5, 1.0, 1.5])
@pytest.mark.parametrize("L,case", [(1, 1), (2, 1), (2, 2)])
def test_tucker_tc_jcomm_parity(beta, L, case, prec):
    ntf = _ntf()
    dims, J = CASES[case]
    X, _, _ = synth.tucker_dense(dims, J, seed=40)
    G0, A0 = synth.init_tucker(dims, J, seed=41)
    Gw, Aw, Fw = oracle.tucker_jcomm_outer(X, G0, A0, beta, L=L)
    Gd, Ad, obj = dev(G0), [dev(a) for a in A0], obj_tensor()
    ntf.jcomm_outer(dev(X), beta, Ad, core=Gd, objective=obj, inner_L=L, precision=prec)
    ntf.default_context().device_status()
    _check(Gd, Ad, Gw, Aw, obj, Fw, "tucker tc %s jcomm beta=%g L=%d %s" % (prec, beta, L, dims))


@pytest.mark.parametrize("prec", ["tf32", "3xtf32"])
@pytest.mark.parametrize("method", ["block", "jcomm"])
def test_tucker_tc_autotuned_contractions(prec, method):
    """Contraction plans timed by the autotuner (tile width and reduction split per product):
    the first call tunes, the second reuses the table; both against the oracle at the
    tensor-core bars."""
    ntf = _ntf()
    dims, J = CASES[1]
    X, _, _ = synth.tucker_dense(dims, J, seed=44)
    G0, A0 = synth.init_tucker(dims, J, seed=45)
    if method == "block":
        Gw, Aw, Fw = oracle.tucker_mu_sweep(X, G0, A0, 1.5)
    else:
        Gw, Aw, Fw = oracle.tucker_jcomm_outer(X, G0, A0, 1.5)
    Xd = dev(X)
    for rep in range(2):
        Gd, Ad, obj = dev(G0), [dev(a) for a in A0], obj_tensor()
        if method == "block":
            ntf.tucker_mu_sweep(Xd, 1.5, Gd, Ad, objective=obj, precision=prec, autotune=True)
        else:
            ntf.jcomm_outer(Xd, 1.5, Ad, core=Gd, objective=obj, precision=prec, autotune=True)
        ntf.default_context().device_status()
        _check(Gd, Ad, Gw, Aw, obj, Fw, "tucker tc %s %s autotuned call %d" % (prec, method, rep))


def test_tucker_tc_kl_runs_on_tensor_cores():
    """beta = 1 with precision "tf32" runs the tensor-core passes without a denominator side
    (Q = 1: the Wd rows and the mode-3 denominators are column sums): tensor-core bar against
    the oracle, and a result that differs from the FP32 passes' (the BF16 contractions ran)."""
    ntf = _ntf()
    dims, J = CASES[0]
    X, _, _ = synth.tucker_dense(dims, J, seed=50)
    G0, A0 = synth.init_tucker(dims, J, seed=51)
    Gw, Aw, Fw = oracle.tucker_mu_sweep(X, G0, A0, 1.0)
    res = {}
    for prec in ("fp32", "tf32"):
        Gd, Ad, obj = dev(G0), [dev(a) for a in A0], obj_tensor()
        ntf.tucker_mu_sweep(dev(X), 1.0, Gd, Ad, objective=obj, precision=prec)
        ntf.default_context().device_status()
        res[prec] = (Gd, Ad)
        if prec == "tf32":
            _check(Gd, Ad, Gw, Aw, obj, Fw, "tucker tc tf32 sweep beta=1")
        else:
            assert rel_fro(host(Gd), Gw) <= 1e-5
    assert rel_fro(host(res["tf32"][0]), host(res["fp32"][0])) > 1e-7


def test_tucker_tc_trajectory_beta15():
    """beta = 3/2: 20 tensor-core sweeps (3xtf32) track the oracle's objective within 1e-3."""
    ntf = _ntf()
    dims, J = (8, 130, 132), (3, 3, 24)
    X, _, _ = synth.tucker_dense(dims, J, seed=60)
    G, A = synth.init_tucker(dims, J, seed=61)
    Gd, Ad, Xd, obj = dev(G), [dev(a) for a in A], dev(X), obj_tensor()
    worst = 0.0
    for t in range(20):
        G, A, Fo = oracle.tucker_mu_sweep(X, G, A, 1.5)
        ntf.tucker_mu_sweep(Xd, 1.5, Gd, Ad, objective=obj, precision="3xtf32")
        worst = max(worst, abs(obj.item() - Fo) / Fo)
    assert worst <= 1e-3, worst
