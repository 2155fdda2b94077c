"""Pins of the accuracy schedules of Eq. (11) (oracle.schedule)."""
import numpy as np

from oracle import schedule as S


def test_ramp():
    assert [S.ramp(k, 0.3, 0.6, 5) for k in range(7)] == [0.3 + 0.3 * min(1, k / 5) for k in range(7)]
    assert S.ramp(3, 0.2, 0.8, 0) == 0.8


def test_global_rule_worked_example():
    # gains 0.5, 0.05, 0.3, 0.01 with tau = 0.1: steps after iterations 2 and 4
    d_pc = [1.0, 1.0, 1.0, 1.0]
    d_pd = [0.5, 0.95, 0.7, 0.99]
    f = S.global_rule(0.2, 0.6, 4, 0.1, d_pc, d_pd)
    assert np.allclose(f, [0.2, 0.2, 0.3, 0.3, 0.4])


def test_global_rule_limits():
    rng = np.random.default_rng(0)
    d_pc = rng.uniform(1, 2, 12)
    d_pd = d_pc * rng.uniform(0.05, 0.99, 12)
    # tau = 1: every iteration steps, which is the plain ramp
    assert S.global_rule(0.3, 0.6, 5, 1.0, d_pc, d_pd) == [S.ramp(i, 0.3, 0.6, 5) for i in range(13)]
    # tau = 0: never a step
    assert S.global_rule(0.3, 0.6, 5, 0.0, d_pc, d_pd) == [0.3] * 13


def test_local_rule():
    dpc = np.array([0.1, 0.5, 1.0, 2.4])          # mean 1.0
    f = S.local_rule(2, 0.3, 0.6, 5, 1.0, dpc, dpc.sum())
    assert np.allclose(f, [0.6, 0.6, 0.6, 0.36])
    assert np.allclose(S.local_rule(1, 0.3, 0.6, 5, 1.0, dpc, None), 0.3)   # no previous iteration
    assert np.allclose(S.local_rule(3, 0.3, 0.6, 5, 0.0, dpc, dpc.sum()), 0.42)
