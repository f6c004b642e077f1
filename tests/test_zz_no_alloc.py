"""The allocation-free objective entry point (ntf_cp_beta_div_noalloc) against the regular
one (ntf_beta_div), through the C ABI.

Who needs it: callers that cannot allocate device memory at call time (a process whose
device memory belongs to another framework's allocator, or one held to a fixed budget, where
a cudaMalloc inside the library would fail or take memory already given out).
The entry point keeps its scratch in a fixed file-scope device array instead of a context
workspace.  This file is collected last on purpose, and passes alone in a fresh process as
well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

import synth
from tests._gpu_util import dev, obj_tensor

pytestmark = pytest.mark.gpu
TOL = 1e-5  # the bar of the FP32 parity tests


def _ntf():
    import paper_2602_14683_gb300 as ntf
    return ntf


def _call(ntf, X, beta, A, out):
    lib = ntf.raw_library()
    d = ntf._lib._Desc(X)
    fp = (ctypes.c_void_p * 3)(*[a.data_ptr() for a in A])
    import torch
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.ntf_cp_beta_div_noalloc(ctypes.byref(d.t), ctypes.c_float(beta), ctypes.c_int(A[0].shape[1]), fp,
                                       ctypes.c_double(1e-12), ctypes.c_double(1e-12),
                                       ctypes.c_void_p(out.data_ptr()), stream)


def test_noalloc_matches_regular_entry_point_twice():
    ntf = _ntf()
    import torch
    # ranks 5, 32 and 48 (padded to 8, 32 and 64 columns in the scratch array)
    cases = [((60, 50, 40), 5, 1.0, 0), ((9, 150, 70), 32, 0.5, 1), ((20, 70, 33), 48, 1.5, 2)]
    for dims, R, beta, seed in cases:  # two calls in a row share the scratch array
        X, _ = synth.cp_dense(dims, R, seed=seed, kind="gamma_noise")
        A = synth.init_factors(dims, R, seed=seed + 7)
        Xd = dev(X)
        Ad = [dev(a) for a in A]
        out = obj_tensor()
        rc = _call(ntf, Xd, beta, Ad, out)
        assert rc == 0
        want = ntf.beta_div(Xd, beta, Ad).item()
        got = out.item()
        assert abs(got - want) <= TOL * abs(want), (dims, got, want)
    torch.cuda.synchronize()


def test_noalloc_call_captured_in_a_cuda_graph():
    """One eager call first (which loads the kernels), then a second call captured into a CUDA
    graph and replayed: the replay writes the objective the regular entry point computes."""
    ntf = _ntf()
    import torch
    dims, R, beta = (60, 50, 40), 5, 1.5
    X, _ = synth.cp_dense(dims, R, seed=11, kind="gamma_noise")
    Xd = dev(X)
    Ad = [dev(a) for a in synth.init_factors(dims, R, seed=12)]
    out, out_g = obj_tensor(), obj_tensor()
    assert _call(ntf, Xd, beta, Ad, out) == 0
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rc = _call(ntf, Xd, beta, Ad, out_g)
    assert rc == 0
    g.replay()
    torch.cuda.synchronize()
    want = ntf.beta_div(Xd, beta, Ad).item()
    assert abs(out_g.item() - want) <= TOL * abs(want), (out_g.item(), want)
    assert out_g.item() == out.item()  # the same kernels on the same inputs


def test_noalloc_rejects_oversized_problem_before_any_work():
    ntf = _ntf()
    import torch
    # (I + J + K) * 32 ranks * 4 bytes > 4 MiB: rejected on the host; X is never read
    Xd = dev(np.ones((1, 1, 1)))
    lib = ntf.raw_library()
    dims = (ctypes.c_int64 * 3)(40000, 1, 1)
    t = ntf._lib.Tensor(3, dims, 0, Xd.data_ptr(), None, 0)
    A = [dev(np.ones((1, 32))) for _ in range(3)]
    fp = (ctypes.c_void_p * 3)(*[a.data_ptr() for a in A])
    out = obj_tensor()
    rc = lib.ntf_cp_beta_div_noalloc(ctypes.byref(t), ctypes.c_float(1.0), ctypes.c_int(32), fp, ctypes.c_double(1e-12),
                                     ctypes.c_double(1e-12), ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -8
    torch.cuda.synchronize()
