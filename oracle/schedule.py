"""Accuracy schedules f = f(d, d_e, i) of Eq. (11) for the approximate search
(Sec. 4.5).  TEST INFRASTRUCTURE ONLY.

ramp          f after k steps of the linear ramp from f0 to f1 in n steps:
              f0 + (f1 - f0) min(1, k / n); the plain schedule takes one step
              per iteration (k = i - 1).
global_rule   the global distance d decides: one more step after every
              iteration in which P_D gained less than the fraction tau,
              gain = 1 - d_after_PD / d_after_PC.
local_rule    the local distance d_e decides: a point whose distance after
              P_C is at most tau times the mean of the previous iteration is
              searched with f1, the others with the plain ramp value.
"""
from __future__ import annotations

import numpy as np


def ramp(k: int, f0: float, f1: float, n: int) -> float:
    if n <= 0:
        return f1
    return f0 + (f1 - f0) * min(1.0, k / n)


def global_rule(f0: float, f1: float, n: int, tau: float, d_pc, d_pd) -> list:
    """f_d of iterations 1 .. len(d_pc) + 1 given each iteration's global
    distances after P_C and after P_D."""
    steps, out = 0, [ramp(0, f0, f1, n)]
    for a, b in zip(d_pc, d_pd):
        gain = 1.0 - b / a if a > 0 else 0.0
        if gain < tau and steps < n:
            steps += 1
        out.append(ramp(steps, f0, f1, n))
    return out


def local_rule(i: int, f0: float, f1: float, n: int, tau: float, dpc: np.ndarray, d_pc_prev) -> np.ndarray:
    """Per-point f_d in iteration i: dpc are the points' weighted distances
    after P_C (summing to the global distance), d_pc_prev the previous
    iteration's global distance after P_C (None in iteration 1)."""
    far = ramp(i - 1, f0, f1, n)
    f = np.full(len(dpc), far)
    if d_pc_prev is not None:
        f[np.asarray(dpc) <= tau * d_pc_prev / len(dpc)] = f1
    return f
