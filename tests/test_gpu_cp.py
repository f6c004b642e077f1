"""Parity of the dense CP CUDA path (FP32) against the FP64 oracle.

Tolerance (FP32 path): after one sweep every factor satisfies
||A_gpu - A_oracle||_F / ||A_oracle||_F <= 1e-5, and objectives agree to 1e-5 relative;
the 50-sweep objective trajectory stays within 1e-4 relative.  Inputs are float32-exact
on both sides (synth rounds them), so the gap is FP32 arithmetic only: per-entry powers
within a few ulp and FP32 sums over <= 2.6e5 terms in blocks of at most 64.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._gpu_util import dev, host, obj_tensor, rel_fro

pytestmark = pytest.mark.gpu

TOL_SWEEP = 1e-5
TOL_TRAJ = 1e-4


def _ntf():
    import paper_2602_14683_gb300 as ntf
    return ntf


# shapes span several row tiles (128 rows; 64 at rank 64) and column blocks (64 columns)
# with ragged tails; K % 4 != 0 exercises the 4-byte copy path
SHAPES = [(60, 50, 40), (9, 150, 70), (5, 131, 130), (3, 200, 67)]


@pytest.mark.parametrize("beta", [0.0, 0.5, 1.0, 1.5, 0.7, 1.2])
@pytest.mark.parametrize("R", [5, 12, 32, 40])
def test_cp_mu_sweep_parity(beta, R):
    ntf = _ntf()
    dims = SHAPES[(R + int(beta * 10)) % len(SHAPES)]
    X, _ = synth.cp_dense(dims, R, seed=R, kind="gamma_noise")
    A = synth.init_factors(dims, R, seed=R + 100)
    want, F_want = oracle.cp_mu_sweep(X, A, beta)
    Xd = dev(X)
    Ad = [dev(a) for a in A]
    obj = obj_tensor()
    ntf.cp_mu_sweep(Xd, beta, Ad, objective=obj)
    for n in range(3):
        e = rel_fro(host(Ad[n]), want[n])
        assert e <= TOL_SWEEP, (n, e)
    assert abs(float(obj.item()) - F_want) / F_want <= TOL_SWEEP


@pytest.mark.parametrize("beta", [0.0, 0.5, 1.0, 1.5])
@pytest.mark.parametrize("L", [1, 2])
def test_cp_jcomm_parity(beta, L):
    ntf = _ntf()
    dims, R = (9, 150, 70), 8
    X, _ = synth.cp_dense(dims, R, seed=3, kind="gamma_noise")
    A = synth.init_factors(dims, R, seed=4)
    want, F_want = oracle.cp_jcomm_outer(X, A, beta, L=L)
    Ad = [dev(a) for a in A]
    obj = obj_tensor()
    ntf.jcomm_outer(dev(X), beta, Ad, objective=obj, inner_L=L)
    for n in range(3):
        e = rel_fro(host(Ad[n]), want[n])
        assert e <= TOL_SWEEP, (n, e)
    assert abs(float(obj.item()) - F_want) / F_want <= TOL_SWEEP


@pytest.mark.parametrize("beta", [0.0, 0.5, 1.0, 1.5, 0.3])
def test_beta_div_parity(beta):
    ntf = _ntf()
    dims, R = (5, 131, 130), 6
    X, _ = synth.cp_dense(dims, R, seed=9, kind="uniform_poisson")
    A = synth.init_factors(dims, R, seed=10)
    want = oracle.cp_objective(X, A, beta)
    got = float(ntf.beta_div(dev(X), beta, [dev(a) for a in A]).item())
    assert abs(got - want) / want <= TOL_SWEEP


def test_c1_trajectory_50_sweeps():
    """60x50x40, R = 5, KL, Poisson data at mean 10: objective trajectory over 50 sweeps."""
    ntf = _ntf()
    dims, R = (60, 50, 40), 5
    X, _ = synth.cp_dense(dims, R, seed=0, kind="uniform_poisson")
    A = synth.init_factors(dims, R, seed=1)
    Xd = dev(X)
    Ad = [dev(a) for a in A]
    obj = obj_tensor()
    worst = 0.0
    for t in range(50):
        A, F_o = oracle.cp_mu_sweep(X, A, 1.0)
        ntf.cp_mu_sweep(Xd, 1.0, Ad, objective=obj)
        F_g = float(obj.item())
        worst = max(worst, abs(F_g - F_o) / F_o)
    assert worst <= TOL_TRAJ, worst


def test_zero_data_and_clip():
    """All-zero slabs drive Num to 0: the update must land exactly on eps."""
    ntf = _ntf()
    dims, R = (6, 20, 12), 3
    X, _ = synth.cp_dense(dims, R, seed=2, kind="uniform_poisson")
    X[2] = 0.0
    A = synth.init_factors(dims, R, seed=5)
    want, _ = oracle.cp_mu_sweep(X, A, 1.0, eps=1e-6)
    Ad = [dev(a) for a in A]
    ntf.cp_mu_sweep(dev(X), 1.0, Ad, eps=1e-6)
    got = host(Ad[0])
    assert np.all(got[2] == np.float32(1e-6))
    for n in range(3):
        assert rel_fro(host(Ad[n]), want[n]) <= TOL_SWEEP


def test_full_size_sampled_rows_mode1():
    """512^3, R = 32, Gamma-noise data (the throughput workload): mode-1 numerators and
    denominators for sampled rows, from one launch of the same pass the sweep uses."""
    ntf = _ntf()
    import torch
    dims, R, beta = (512, 512, 512), 32, 1.5
    X, _ = synth.cp_dense(dims, R, seed=0, kind="gamma_noise")
    A = synth.init_factors(dims, R, seed=1)
    Xd = dev(X)
    Ad = [dev(a) for a in A]
    ntf.cp_mu_sweep(Xd, beta, Ad)
    torch.cuda.synchronize()
    got = host(Ad[0])
    rows = [0, 1, 127, 128, 300, 511]
    num, den = oracle.cp_numden_rows(X, A, A, A, 0, rows, beta)
    upd = np.maximum(A[0][rows] * (num / den), 1e-12)
    e = rel_fro(got[rows], upd)
    assert e <= TOL_SWEEP, e


def test_error_codes():
    ntf = _ntf()
    import torch
    X = dev(np.ones((4, 5, 6)))
    A = [dev(np.ones((d, 3))) for d in (4, 5, 6)]
    with pytest.raises(ntf.NtfError) as e:
        ntf.cp_mu_sweep(X, 2.0, A)
    assert e.value.code == -2
    with pytest.raises(ntf.NtfError) as e:
        ntf.cp_mu_sweep(X, -0.5, A)
    assert e.value.code == -2
    A65 = [dev(np.ones((d, 65))) for d in (4, 5, 6)]
    with pytest.raises(ntf.NtfError) as e:
        ntf.cp_mu_sweep(X, 1.0, A65)
    assert e.value.code == -8
    X2 = dev(np.ones((4, 5)))
    with pytest.raises(ntf.NtfError) as e:
        ntf.cp_mu_sweep(X2, 1.0, [dev(np.ones((d, 3))) for d in (4, 5)])
    assert e.value.code == -8
    with pytest.raises(ntf.NtfError) as e:
        ntf.cp_mu_sweep(X, 1.0, A, inner_L=0)
    assert e.value.code == -1
    torch.cuda.synchronize()
