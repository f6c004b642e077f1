"""The cut of an order-N dense problem into three runs of modes (host-only planning through the C
ABI; no GPU).  Expected cuts follow from the chooser's stated rules: a last run whose extent is a
multiple of 4 (16-byte rows, hence the tensor-core passes) when the precision asks for tensor cores,
else the least padded tile work; for Tucker the last run's core extent must stay <= 64."""
import pytest


def _ntf():
    import paper_2602_14683_gb300 as ntf
    return ntf


def test_cp_4way_tensor_cores_take_the_aligned_cut():
    ntf = _ntf()
    # only the cut (80, 70, 60*50) has a last extent that is a multiple of 4
    assert ntf.plan_cut((80, 70, 60, 50), rank=10, precision="tf32") == (1, 2)


def test_cp_4way_fp32_takes_the_least_padded_work():
    ntf = _ntf()
    # padded cells: (80, 70->128, 3000->3008) = 30.8M; (80, 4200->4224, 50->64) = 21.6M;
    # (5600, 60->128, 50->64) = 45.9M
    assert ntf.plan_cut((80, 70, 60, 50), rank=10, precision="fp32") == (1, 3)


def test_cp_rank_above_32_has_no_tensor_core_cut():
    ntf = _ntf()
    assert ntf.plan_cut((80, 70, 60, 50), rank=40, precision="tf32") == (1, 3)


def test_explicit_merge_is_kept_and_checked():
    ntf = _ntf()
    assert ntf.plan_cut((2, 3, 4, 5, 6), rank=4, merge=(2, 4)) == (2, 4)
    for bad in ((0, 2), (3, 3), (2, 5)):
        with pytest.raises(ntf.NtfError) as e:
            ntf.plan_cut((2, 3, 4, 5, 6), rank=4, merge=bad)
        assert e.value.code == -1


def test_orders_outside_4_to_8_are_refused():
    ntf = _ntf()
    for dims in ((4, 5, 6), (2,) * 9):
        with pytest.raises(ntf.NtfError) as e:
            ntf.plan_cut(dims, rank=4)
        assert e.value.code == -8


def test_tucker_paper_shapes():
    ntf = _ntf()
    # 4-way synthetic Tucker: (1, 2) leaves a last core run of 8 * 7 = 56 (rank padding 64, eight
    # times the per-entry pass work of the padding 8 that the other cuts get); of those, the
    # estimate (pass work plus the small GEMMs) picks modes 1 and 2 merged
    assert ntf.plan_cut((80, 70, 60, 50), core_dims=(10, 9, 8, 7), beta=1.5) == (1, 3)
    # 5-way real-data shape: runs {0,1}, {2,3}, {4}, last core extent 10 (tensor cores at tf32)
    assert ntf.plan_cut((27, 24, 7, 100, 100), core_dims=(10, 10, 5, 10, 10), beta=1.5, precision="tf32") == (2, 4)


def test_tucker_cut_needs_a_small_last_core_run():
    ntf = _ntf()
    with pytest.raises(ntf.NtfError) as e:
        ntf.plan_cut((6, 5, 9, 9), core_dims=(2, 2, 9, 9), merge=(1, 2))
    assert e.value.code == -8
    # the library's own choice avoids that run
    a, b = ntf.plan_cut((6, 5, 9, 9), core_dims=(2, 2, 9, 9))
    assert b == 3


def test_objective_cut_is_the_fp32_cut():
    """ntf_beta_div evaluates the objective on the FP32 passes whatever the precision option says,
    so its cut is the one planned at fp32; the sweeps at tf32 take the aligned cut."""
    ntf = _ntf()
    assert ntf.plan_cut((80, 70, 60, 50), rank=10, precision="tf32") == (1, 2)
    assert ntf.plan_cut((80, 70, 60, 50), rank=10, precision="fp32") == (1, 3)


def test_planning_checks_the_options_of_the_planned_calls():
    ntf = _ntf()
    cases = [(dict(dims=(80, 70, 60, 2 ** 31)), -3),          # a dimension beyond 32 bits
             (dict(precision=7), -1),                          # unknown precision
             (dict(eps=0.0), -1), (dict(eps_x=-1.0), -1),      # floors must be positive
             (dict(inner_L=0), -1),
             (dict(beta=2.0), -2), (dict(beta=-0.5), -2)]      # beta outside [0, 2)
    for kw, code in cases:
        dims = kw.pop("dims", (80, 70, 60, 50))
        with pytest.raises(ntf.NtfError) as e:
            ntf.plan_cut(dims, rank=10, **kw)
        assert e.value.code == code, (kw, e.value.code)
