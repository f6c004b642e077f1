"""Parity at the sizes and launch configurations that bench.py times.

* Dense CP 512^3, R = 32: one J-CoMM outer iteration (L = 1) with autotune on -- at beta = 1 the
  plan and kernel instantiation the benchmark times (all three numerators and the objective in
  one fused pass, 256-column blocks, the tuned slab split) -- in tf32 and 3xtf32, and at beta = 1/2
  (one pass per block against the reference, chi_1 / chi_2 of the current blocks).  Every row of
  all three updated factors is compared with an FP64 oracle of the same outer iteration
  (Algorithm 2; Section 5.3 "CP inner update"), built from full FP64 numerator / denominator
  contractions of ntfo_cp_numden_rows.
* Dense Tucker 400^3, core 32^3, beta = 3/2: one block-MM sweep (core, then modes 1..3) per
  precision against the FP64 mode-n-product oracle of the same sweep.

Bars: FP32 1e-5 per factor (the one-sweep bar); tensor cores 1e-3 per factor (BF16 contraction
operands, unit roundoff 2^-8, averaged over hundreds of rows: the derivation of the other
tensor-core parity tests).
"""
import numpy as np
import pytest

import oracle
import synth
from tests._gpu_util import dev, host, obj_tensor, rel_fro

pytestmark = pytest.mark.gpu
TOL_TC = 1e-3
TOL_FP32 = 1e-5


def _ntf():
    import paper_2602_14683_gb300 as ntf
    return ntf


def _gamma(beta):
    return 1.0 / (2.0 - beta) if beta < 1.0 else 1.0


def _chi1(z, zt, beta):
    return zt ** (2.0 - beta) * z ** (beta - 1.0)


def _chi2(z, zt, beta):
    return z.copy() if beta < 1.0 else z ** beta * zt ** (1.0 - beta)


def _jcomm_outer_fp64(X, At, beta, eps=1e-12):
    """One J-CoMM outer iteration with L = 1 from the reference At (Algorithm 2): for n = 1..3,
    Num_J / Den_J = CPContr^(n) of P~ / Q~ against chi_1 / chi_2 of the current blocks (modes
    m < n already updated), evaluated by the oracle's row checker over every row, then
    A^(n) = max(A~^(n) (Num_J / Den_J)^gamma, eps)."""
    A = [a.copy() for a in At]
    for n in range(3):
        B1 = [_chi1(a, at, beta) for a, at in zip(A, At)]
        B2 = [_chi2(a, at, beta) for a, at in zip(A, At)]
        rows = np.arange(X.shape[n])
        num, den = oracle.cp_numden_rows(X, At, B1, B2, n, rows, beta)
        A[n] = np.maximum(At[n] * (num / den) ** _gamma(beta), eps)
    return A


_CP = {}


def _cp_case():
    if not _CP:
        X, _ = synth.cp_dense((512, 512, 512), 32, seed=0, kind="gamma_noise")
        _CP["X"] = X
        _CP["A"] = synth.init_factors((512, 512, 512), 32, seed=1)
        _CP["want"] = {}
    return _CP


@pytest.mark.parametrize("beta,prec", [(1.0, "tf32"), (1.0, "3xtf32"), (0.5, "tf32")])
def test_cp512_jcomm_outer_all_factors(beta, prec):
    ntf = _ntf()
    c = _cp_case()
    X, A = c["X"], c["A"]
    if beta not in c["want"]:
        c["want"][beta] = _jcomm_outer_fp64(X.astype(np.float64), A, beta)
    want = c["want"][beta]
    Xd = dev(X)
    for rep in range(2):  # the first call tunes the slab split, the second reuses it
        Ad = [dev(a) for a in A]
        ntf.jcomm_outer(Xd, beta, Ad, objective=obj_tensor(), precision=prec, autotune=True)
        ntf.default_context().device_status()
        errs = [rel_fro(host(Ad[n]), want[n]) for n in range(3)]
        print("cp512 jcomm beta=%g %s call %d: per-factor rel err %s" % (beta, prec, rep, errs))
        assert max(errs) <= TOL_TC, errs


def test_tucker400_block_sweep_per_precision():
    ntf = _ntf()
    import torch
    from oracle import tucker_modeprod as tm
    n, J, beta = 400, 32, 1.5
    torch.manual_seed(3)
    G = torch.distributions.Gamma(torch.full((J, J, J), 2.0), 1.0).sample().double()
    F = [torch.distributions.Gamma(torch.full((n, J), 2.0), 1.0).sample().double() for _ in range(3)]
    M = tm.tucker_full(G, F)
    M *= 10.0 / M.mean()
    X = torch.poisson(M.float()).float()
    del M
    g = np.random.default_rng(4)
    G0 = g.uniform(0.1, 1.0, size=(J, J, J)).astype(np.float32)
    A0 = [g.uniform(0.1, 1.0, size=(n, J)).astype(np.float32) for _ in range(3)]
    Gw, Aw, Fw = tm.tucker_mu_sweep(X.double(), G0, A0, beta)
    Xd = X.cuda()
    for prec, tol in (("fp32", TOL_FP32), ("tf32", TOL_TC), ("3xtf32", TOL_TC)):
        Gd, Ad, obj = dev(G0), [dev(a) for a in A0], obj_tensor()
        ntf.tucker_mu_sweep(Xd, beta, Gd, Ad, objective=obj, precision=prec)
        ntf.default_context().device_status()
        errs = [rel_fro(host(Gd), Gw)] + [rel_fro(host(Ad[m]), Aw[m]) for m in range(3)]
        fo = abs(obj.item() - Fw) / Fw
        print("tucker400 %s: core/factor rel err %s, objective %.2e" % (prec, errs, fo))
        assert max(errs) <= tol, (prec, errs)
        assert fo <= (TOL_FP32 if prec == "fp32" else 2e-4), (prec, fo)
