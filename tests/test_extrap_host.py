"""Host logic of the extrapolated sweeps: the Nesterov-type weight sequence."""
import math


def test_nesterov_weights_sequence():
    import paper_2602_14683_gb300 as ntf
    w = ntf.nesterov_weights()
    vals = [next(w) for _ in range(50)]
    assert vals[0] == 0.0
    # alpha_t = (a_(t-1) - 1) / a_t with a_t = (1 + sqrt(1 + 4 a_(t-1)^2)) / 2, a_0 = 1
    a_prev, a = 1.0, (1.0 + math.sqrt(5.0)) / 2.0
    assert vals[1] == (a - 1.0) / ((1.0 + math.sqrt(1.0 + 4.0 * a * a)) / 2.0)
    assert all(0.0 <= x < 1.0 for x in vals)
    assert all(y > x for x, y in zip(vals[1:], vals[2:]))
    # a_t ~ (t + 1) / 2, so alpha_t ~ 1 - 3 / t for large t
    assert abs(vals[-1] - (1.0 - 3.0 / 50)) < 0.02
