"""Tensor-core (tcgen05) dense CP passes against the FP64 oracle.

Arithmetic of this path: the reconstruction GEMM runs on TF32 operands rounded to nearest
(10-bit mantissa, unit roundoff u = 2^-11; "3xtf32" splits each operand into high and low
TF32 parts and keeps three products, about FP32 accuracy) and the two contraction GEMMs on
BF16 operands (u = 2^-8 for the stored P, Q, column factors and Khatri-Rao rows), all with
FP32 accumulation; powers and the objective stay in FP32 with an FP64 sum.  Rounding errors
of the BF16 operands are independent and unbiased, so a numerator summed over n terms
carries a relative error of about u_bf16 * sqrt(sum w^2) / sum w ~ u_bf16 / sqrt(n_eff);
with at least a few hundred effective terms per output here that is below 2e-4, and the
ratio Num/Den of one block update inherits it.  The bar below (TOL_TC = 1e-3 on each
factor after one sweep, 2e-4 on the objective, which only sees the reconstruction) leaves a
factor ~5 of margin.  With one TF32 pass Xhat carries ~u_tf32 / sqrt(R) unbiased relative
error per entry; the objective moves by sum (1 - x / y) dy, a sum of zero-mean terms, so
its relative error stays near 1e-6 (1e-8 with the split).  The objective on this path
evaluates the definition of d_beta directly with single-MUFU logarithms / roots: near x = y
its terms cancel, costing about u_fp32 * x^beta / d per entry, well inside 2e-4 on the
noisy data used here.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._gpu_util import dev, host, obj_tensor, rel_fro

pytestmark = pytest.mark.gpu
TOL_TC = 1e-3
TOL_TC_OBJ = 2e-4


def _ntf():
    import paper_2602_14683_gb300 as ntf
    return ntf


@pytest.mark.parametrize("prec", ["tf32", "3xtf32"])
@pytest.mark.parametrize("beta", [0.0, 0.5, 1.0, 1.5, 0.7])
@pytest.mark.parametrize("dims,R", [((9, 150, 200), 32), ((7, 130, 300), 20)])
def test_tc_mu_sweep_parity(beta, dims, R, prec):
    ntf = _ntf()
    X, _ = synth.cp_dense(dims, R, seed=R, kind="gamma_noise")
    A = synth.init_factors(dims, R, seed=R + 1)
    want, Fw = oracle.cp_mu_sweep(X, A, beta)
    Ad = [dev(a) for a in A]
    obj = obj_tensor()
    ctx = ntf.default_context()
    ntf.cp_mu_sweep(dev(X), beta, Ad, objective=obj, precision=prec)
    ctx.device_status()
    errs = [rel_fro(host(Ad[n]), want[n]) for n in range(3)]
    eo = abs(obj.item() - Fw) / Fw
    print("tc %s sweep beta=%g dims=%s R=%d factor errs=%s obj err=%.2e" % (prec, beta, dims, R, errs, eo))
    assert max(errs) <= TOL_TC, errs
    assert eo <= TOL_TC_OBJ


@pytest.mark.parametrize("prec", ["tf32", "3xtf32"])
@pytest.mark.parametrize("beta", [0.5, 1.0, 1.5])
@pytest.mark.parametrize("L", [1, 2])
def test_tc_jcomm_parity(beta, L, prec):
    ntf = _ntf()
    dims, R = (9, 150, 200), 32
    X, _ = synth.cp_dense(dims, R, seed=5, kind="gamma_noise")
    A = synth.init_factors(dims, R, seed=6)
    want, Fw = oracle.cp_jcomm_outer(X, A, beta, L=L)
    Ad = [dev(a) for a in A]
    obj = obj_tensor()
    ntf.jcomm_outer(dev(X), beta, Ad, objective=obj, inner_L=L, precision=prec)
    ntf.default_context().device_status()
    errs = [rel_fro(host(Ad[n]), want[n]) for n in range(3)]
    eo = abs(obj.item() - Fw) / Fw
    print("tc %s jcomm beta=%g L=%d factor errs=%s obj err=%.2e" % (prec, beta, L, errs, eo))
    assert max(errs) <= TOL_TC, errs
    assert eo <= TOL_TC_OBJ


@pytest.mark.parametrize("prec", ["tf32", "3xtf32"])
def test_tc_trajectory_c1_like(prec):
    """KL, Poisson data at mean 10: the TF32/BF16 objective trajectory stays within 1e-3
    of the FP64 oracle over 30 sweeps (errors do not compound: each sweep is a descent step
    from wherever the previous one landed)."""
    ntf = _ntf()
    dims, R = (40, 130, 136), 32
    X, _ = synth.cp_dense(dims, R, seed=0, kind="uniform_poisson")
    A = synth.init_factors(dims, R, seed=1)
    Xd = dev(X)
    Ad = [dev(a) for a in A]
    obj = obj_tensor()
    worst = 0.0
    for t in range(30):
        A, Fo = oracle.cp_mu_sweep(X, A, 1.0)
        ntf.cp_mu_sweep(Xd, 1.0, Ad, objective=obj, precision=prec)
        worst = max(worst, abs(obj.item() - Fo) / Fo)
    ntf.default_context().device_status()
    print("tc %s trajectory worst rel err %.2e" % (prec, worst))
    assert worst <= 1e-3


def test_tc_full_size_sampled_rows():
    """512^3, R = 32: one mode-1 update on tensor cores against oracle rows."""
    ntf = _ntf()
    import torch
    dims, R, beta = (512, 512, 512), 32, 1.0
    X, _ = synth.cp_dense(dims, R, seed=0, kind="gamma_noise")
    A = synth.init_factors(dims, R, seed=1)
    Ad = [dev(a) for a in A]
    ntf.cp_mu_sweep(dev(X), beta, Ad, precision="tf32")
    ntf.default_context().device_status()
    got = host(Ad[0])
    rows = [0, 1, 127, 128, 300, 511]
    num, den = oracle.cp_numden_rows(X, A, A, A, 0, rows, beta)
    want = A[0][rows] * num / den
    e = rel_fro(got[rows], want)
    print("tc full-size mode-1 rows rel err %.2e" % e)
    assert e <= TOL_TC
    torch.cuda.synchronize()
