"""The entry points are stream-ordered: once a call's workspaces exist it makes no allocation and
no host synchronisation, so a caller may capture calls into a CUDA graph and replay them (the C1
latency case of bench.py does).  Replaying the captured calls must give bit-identical results to
making the same calls eagerly (the kernels are deterministic and read their inputs at run time)."""
import numpy as np
import pytest

import synth
from tests._gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _ntf():
    import paper_2602_14683_gb300 as ntf
    return ntf


def _replay_vs_eager(call, blocks0, steps=3):
    """call(blocks, obj) makes one step in place; returns (eager blocks, eager obj), (graph ...)."""
    import torch
    be = [b.clone() for b in blocks0]
    oe = torch.zeros(1, dtype=torch.float64, device=blocks0[0].device)
    for _ in range(steps):
        call(be, oe)
    bw = [b.clone() for b in blocks0]  # warm-up on other tensors of the same shapes: workspaces exist
    call(bw, torch.zeros_like(oe))
    bg = [b.clone() for b in blocks0]
    og = torch.zeros_like(oe)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        call(bg, og)
    for b, b0 in zip(bg, blocks0):  # capture ran nothing, but start from the same point regardless
        b.copy_(b0)
    for _ in range(steps):
        g.replay()
    torch.cuda.synchronize()
    return (be, oe), (bg, og)


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
@pytest.mark.parametrize("method", ["sweep", "jcomm"])
def test_cp_graph_replay_bit_exact(prec, method):
    ntf = _ntf()
    dims, R = (60, 50, 40), 5
    Xn, _ = synth.cp_dense(dims, R, seed=3, kind="uniform_poisson")
    X = dev(Xn)
    A0 = [dev(a) for a in synth.init_factors(dims, R, seed=4)]

    def call(A, obj):
        if method == "sweep":
            ntf.cp_mu_sweep(X, 1.5, A, objective=obj, precision=prec)
        else:
            ntf.jcomm_outer(X, 1.5, A, objective=obj, precision=prec)
    (be, oe), (bg, og) = _replay_vs_eager(call, A0)
    for a, b in zip(be, bg):
        assert np.array_equal(host(a), host(b))
    assert oe.item() == og.item()


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_tucker_graph_replay_bit_exact(prec):
    ntf = _ntf()
    dims, J = (12, 96, 200), (4, 5, 28)
    Xn, _, _ = synth.tucker_dense(dims, J, seed=5)
    X = dev(Xn)
    G0, A0 = synth.init_tucker(dims, J, seed=6)
    blocks0 = [dev(G0)] + [dev(a) for a in A0]

    def call(B, obj):
        ntf.tucker_mu_sweep(X, 1.5, B[0], B[1:], objective=obj, precision=prec)
    (be, oe), (bg, og) = _replay_vs_eager(call, blocks0)
    for a, b in zip(be, bg):
        assert np.array_equal(host(a), host(b))
    assert oe.item() == og.item()


@pytest.mark.parametrize("beta", [1.0, 1.5])
def test_coo_graph_replay_bit_exact(beta):
    """Sparse COO J-CoMM (the orders are built by the first, eager call; the objective's factor
    set is a kernel argument, so the captured calls copy nothing from the host)."""
    import torch
    ntf = _ntf()
    g = np.random.default_rng(9)
    dims, R = (9, 6, 31, 40), 5
    X = np.where(g.uniform(size=dims) < 0.15, 1.0 + g.geometric(0.3, size=dims) - 1.0, 0.0)
    idx = np.nonzero(X)
    Xc = ntf.Coo(dims, [torch.tensor(i.astype(np.int32), device="cuda") for i in idx],
                 torch.tensor(X[idx].astype(np.float32), device="cuda"))
    A0 = [dev(a) for a in synth.init_factors(dims, R, seed=10)]

    def call(A, obj):
        ntf.jcomm_outer(Xc, beta, A, objective=obj)
    (be, oe), (bg, og) = _replay_vs_eager(call, A0)
    for a, b in zip(be, bg):
        assert np.array_equal(host(a), host(b))
    assert oe.item() == og.item()
