"""Failure detection of the bounded device-side waits, without a GPU fault.

The tensor-core passes wait on TMA / MMA completion barriers with a poll limit.  A context's
timeout probe makes each such pass wait on a barrier that nothing arrives on, before it has
issued any copy or MMA: the wait runs out, the pass raises its abort flag, the other warps
stop at their next wait, TMEM is freed and the kernel returns with the context's status word
set.  The host then reads NTF_ERR_TIMEOUT, and the same context computes correct results
again once the probe is off.
"""
import pytest

import oracle
import synth
from tests._gpu_util import dev, host, obj_tensor, rel_fro

pytestmark = pytest.mark.gpu


def test_wait_runs_out_and_the_context_recovers():
    import paper_2602_14683_gb300 as ntf
    ctx = ntf.Context(0)
    dims, R = (20, 300, 260), 32  # tensor-core eligible: RP 32, K % 4 == 0
    X, _ = synth.cp_dense(dims, R, seed=11, kind="gamma_noise")
    A = synth.init_factors(dims, R, seed=12)
    Xd = dev(X)
    ctx.debug_wait_limit(256, probe=True)
    Ad, obj = [dev(a) for a in A], obj_tensor()
    ntf.jcomm_outer(Xd, 1.0, Ad, objective=obj, ctx=ctx, precision="tf32")
    with pytest.raises(ntf.NtfError) as e:
        ctx.device_status()
    assert e.value.code == -6  # NTF_ERR_TIMEOUT
    ctx.device_status()  # the word was cleared by the read
    ctx.debug_wait_limit(0, probe=False)
    want, F = oracle.cp_jcomm_outer(X, A, 1.0)
    for _ in range(2):
        Ad, obj = [dev(a) for a in A], obj_tensor()
        ntf.jcomm_outer(Xd, 1.0, Ad, objective=obj, ctx=ctx, precision="tf32")
        ctx.device_status()
        errs = [rel_fro(host(Ad[n]), want[n]) for n in range(3)]
        assert max(errs) <= 1e-3, errs
        assert abs(obj.item() - F) / F <= 2e-4
    ctx.close()
