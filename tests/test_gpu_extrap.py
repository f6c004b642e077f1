"""Extrapolated B-CoMM sweeps (ntf_cp_mu_sweep_extrap) against the FP64 oracle.

Same bars as the plain sweeps: FP32 path 1e-5 per factor after one sweep and on the
objective of the incoming iterate, 1e-4 on a 15-iteration objective trajectory driven by
the Nesterov-type weights; tensor-core path 1e-3 / 2e-4.  The previous-iterate buffers must
come back holding the incoming iterate exactly.
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


@pytest.mark.parametrize("prec,R,tol,tol_obj", [("fp32", 12, 1e-5, 1e-5), ("tf32", 32, 1e-3, 2e-4)])
@pytest.mark.parametrize("beta", [0.5, 1.0, 1.5])
@pytest.mark.parametrize("cap", [float("inf"), 0.3])
def test_extrap_sweep_parity(prec, R, tol, tol_obj, beta, cap):
    ntf = _ntf()
    dims = (9, 150, 200)
    X, _ = synth.cp_dense(dims, R, seed=R + 3, kind="gamma_noise")
    A = synth.init_factors(dims, R, seed=R + 4)
    g = np.random.default_rng(R)
    Ap = [a * g.uniform(0.6, 1.1, size=a.shape) for a in A]
    Ap = [np.float32(a).astype(np.float64) for a in Ap]
    alpha = 0.7
    want, want_prev, Fw = oracle.cp_mu_sweep_extrap(X, A, Ap, beta, alpha=alpha, cap=cap)
    Ad, Pd, obj = [dev(a) for a in A], [dev(a) for a in Ap], obj_tensor()
    ntf.cp_mu_sweep_extrap(dev(X), beta, Ad, Pd, alpha, cap=cap, objective=obj, precision=prec)
    ntf.default_context().device_status()
    errs = [rel_fro(host(Ad[n]), want[n]) for n in range(3)]
    assert max(errs) <= tol, errs
    for n in range(3):
        assert np.array_equal(host(Pd[n]), np.float32(A[n]).astype(np.float64)), n
    assert abs(obj.item() - Fw) / Fw <= tol_obj


def test_extrap_trajectory_nesterov():
    ntf = _ntf()
    dims, R = (12, 90, 70), 6
    X, _ = synth.cp_dense(dims, R, seed=41, kind="uniform_poisson")
    A = synth.init_factors(dims, R, seed=42)
    P = [a.copy() for a in A]
    Ad, Pd, Xd, obj = [dev(a) for a in A], [dev(a) for a in A], dev(X), obj_tensor()
    weights = ntf.nesterov_weights()
    worst = 0.0
    for t in range(15):
        w = next(weights)
        A, P, Fo = oracle.cp_mu_sweep_extrap(X, A, P, 1.0, alpha=w, cap=1.0)
        ntf.cp_mu_sweep_extrap(Xd, 1.0, Ad, Pd, w, cap=1.0, objective=obj)
        worst = max(worst, abs(obj.item() - Fo) / Fo)
    assert worst <= 1e-4, worst


@pytest.mark.parametrize("prec,R,tol,tol_obj", [("fp32", 12, 1e-5, 1e-5), ("tf32", 32, 1e-3, 2e-4)])
@pytest.mark.parametrize("beta", [0.5, 1.0, 1.5])
@pytest.mark.parametrize("L", [1, 2])
def test_jcomm_extrap_parity(prec, R, tol, tol_obj, beta, L):
    ntf = _ntf()
    dims = (9, 150, 200)
    X, _ = synth.cp_dense(dims, R, seed=R + 5, kind="gamma_noise")
    A = synth.init_factors(dims, R, seed=R + 6)
    g = np.random.default_rng(R + 1)
    Ap = [np.float32(a * g.uniform(0.6, 1.1, size=a.shape)).astype(np.float64) for a in A]
    want, want_prev, Fw = oracle.cp_jcomm_outer_extrap(X, A, Ap, beta, alpha=0.7, cap=0.5, L=L)
    Ad, Pd, obj = [dev(a) for a in A], [dev(a) for a in Ap], obj_tensor()
    ntf.cp_jcomm_outer_extrap(dev(X), beta, Ad, Pd, 0.7, cap=0.5, objective=obj, precision=prec, inner_L=L)
    ntf.default_context().device_status()
    errs = [rel_fro(host(Ad[n]), want[n]) for n in range(3)]
    assert max(errs) <= tol, errs
    for n in range(3):
        assert np.array_equal(host(Pd[n]), np.float32(A[n]).astype(np.float64)), n
    assert abs(obj.item() - Fw) / Fw <= tol_obj


TUCKER_CASES = [((7, 140, 36), (3, 5, 4), "fp32", 1e-5, 1e-5), ((6, 140, 132), (3, 4, 20), "tf32", 1e-3, 2e-4)]


@pytest.mark.parametrize("case", range(len(TUCKER_CASES)))
@pytest.mark.parametrize("beta", [0.5, 1.0, 1.5])
def test_tucker_extrap_sweep_parity(case, beta):
    ntf = _ntf()
    dims, J, prec, tol, tol_obj = TUCKER_CASES[case]
    X, _, _ = synth.tucker_dense(dims, J, seed=70 + case)
    G0, A0 = synth.init_tucker(dims, J, seed=71 + case)
    g = np.random.default_rng(case)
    Gp = np.float32(G0 * g.uniform(0.6, 1.1, size=G0.shape)).astype(np.float64)
    Ap = [np.float32(a * g.uniform(0.6, 1.1, size=a.shape)).astype(np.float64) for a in A0]
    Gw, Aw, Gpw, Apw, Fw = oracle.tucker_mu_sweep_extrap(X, G0, A0, Gp, Ap, beta, alpha=0.6, cap=0.4)
    Gd, Ad, Gpd, Apd, obj = dev(G0), [dev(a) for a in A0], dev(Gp), [dev(a) for a in Ap], obj_tensor()
    ntf.tucker_mu_sweep_extrap(dev(X), beta, Gd, Ad, Gpd, Apd, 0.6, cap=0.4, objective=obj, precision=prec)
    ntf.default_context().device_status()
    errs = [rel_fro(host(Gd), Gw)] + [rel_fro(host(Ad[n]), Aw[n]) for n in range(3)]
    assert max(errs) <= tol, errs
    assert np.array_equal(host(Gpd), np.float32(G0).astype(np.float64))
    for n in range(3):
        assert np.array_equal(host(Apd[n]), np.float32(A0[n]).astype(np.float64)), n
    assert abs(obj.item() - Fw) / Fw <= tol_obj


@pytest.mark.parametrize("case", range(len(TUCKER_CASES)))
@pytest.mark.parametrize("beta", [0.5, 1.5])
@pytest.mark.parametrize("L", [1, 2])
def test_tucker_jcomm_extrap_parity(case, beta, L):
    ntf = _ntf()
    dims, J, prec, tol, tol_obj = TUCKER_CASES[case]
    X, _, _ = synth.tucker_dense(dims, J, seed=80 + case)
    G0, A0 = synth.init_tucker(dims, J, seed=81 + case)
    g = np.random.default_rng(case + 10)
    Gp = np.float32(G0 * g.uniform(0.6, 1.1, size=G0.shape)).astype(np.float64)
    Ap = [np.float32(a * g.uniform(0.6, 1.1, size=a.shape)).astype(np.float64) for a in A0]
    Gw, Aw, _, _, Fw = oracle.tucker_jcomm_outer_extrap(X, G0, A0, Gp, Ap, beta, alpha=0.6, cap=0.4, L=L)
    Gd, Ad, Gpd, Apd, obj = dev(G0), [dev(a) for a in A0], dev(Gp), [dev(a) for a in Ap], obj_tensor()
    ntf.tucker_jcomm_outer_extrap(dev(X), beta, Gd, Ad, Gpd, Apd, 0.6, cap=0.4, objective=obj, precision=prec,
                                  inner_L=L)
    ntf.default_context().device_status()
    errs = [rel_fro(host(Gd), Gw)] + [rel_fro(host(Ad[n]), Aw[n]) for n in range(3)]
    assert max(errs) <= tol, errs
    assert np.array_equal(host(Gpd), np.float32(G0).astype(np.float64))
    assert abs(obj.item() - Fw) / Fw <= tol_obj
