"""Host logic of the optimisation loop (no GPU): the AMSGrad step-size schedule of Sec. IV.B."""
from paper_1807_10633_gb300.optimize import alpha_schedule


def test_alpha_schedule():
    assert [alpha_schedule(k) for k in range(7)] == [0.001] * 5 + [0.01] * 2
    assert alpha_schedule(2, 0.5, 0.25, warm=3) == 0.5 and alpha_schedule(3, 0.5, 0.25, warm=3) == 0.25
