"""Data-driven fixed-point iteration of Sec. 2 (FP64 oracle).

    z_{i+1} = P_D(P_C(z_i))                                   Eq. (8)

P_C (Eq. 4-6): two solves with the fixed stiffness K, then eps = B u and
sig = sig* + C B eta at every material point.  P_D (Eq. 7): exact nearest
data point of every material point under the local distance Eq. (3), found by
the brute-force scan of ``oracle.nn`` in the mapped coordinates.  The material
points start from a given (random) association (Sec. 2, last paragraph) and
the iteration stops when the association no longer changes, which under an
exact P_D is the same as the global distance Eq. (2) no longer decreasing.

The returned state is the constraint-set state y = (u, eps, sig) of the last
P_C together with the final association.  The history records, per
iteration i, the global distance Eq. (2) after P_C, D(y_{i+1}, z_i), and after
P_D, D(y_{i+1}, z_{i+1}); alternating minimisation makes the sequence
non-increasing, which tests/test_oracle_dd.py checks.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import fem as _fem
from . import metric as _metric
from . import nn as _nn


@dataclass
class DDResult:
    u: np.ndarray
    eta: np.ndarray
    eps: np.ndarray
    sig: np.ndarray
    idx: np.ndarray
    iters: int
    converged: bool
    d2_after_pc: list = field(default_factory=list)
    d2_after_pd: list = field(default_factory=list)
    changed: list = field(default_factory=list)


class DDProblem:
    """A cube problem: mesh + metric + load + material data set."""

    def __init__(self, data: np.ndarray, C: np.ndarray, n_el: int, load,
                 fixed: np.ndarray | None = None):
        self.data = np.asarray(data, dtype=np.float64)       # (eps*, sig*) rows
        self.C = np.asarray(C, dtype=np.float64)
        self.fe = _fem.HexBox(n_el, n_el, n_el, self.C)
        self.Z = _metric.to_z(self.data, self.C)
        rot = float(getattr(load, "rot_z", 0.0))
        if fixed is None:
            fixed = self.fe.clamped_bottom()
            if rot != 0.0:                       # the top face is a Dirichlet boundary
                fixed = fixed | self.fe.clamped_top()
        self.solver = _fem.DirectSolver(self.fe.K(), fixed)
        # u takes the prescribed values on the top face; eta is zero there (Eq. 5)
        self.u_d = self.fe.top_rotation(rot) if rot != 0.0 else None
        self.f = np.zeros(self.fe.n_dof) if rot != 0.0 else self.fe.top_traction_force(load.t0, load.tx, load.ty)
        self.w = self.fe.w

    def project_C(self, idx: np.ndarray):
        """P_C of the data states z_i = data[idx] (Eq. 5, Eq. 6)."""
        star = self.data[idx]
        eps_s, sig_s = star[:, :6], star[:, 6:]
        u = self.solver.solve(self.fe.assemble_BT(eps_s @ self.C.T), prescribed=self.u_d)
        eta = self.solver.solve(self.f - self.fe.assemble_BT(sig_s))
        eps = self.fe.strains(u)
        sig = sig_s + self.fe.strains(eta) @ self.C.T
        return u, eta, eps, sig

    def project_D(self, eps: np.ndarray, sig: np.ndarray):
        """P_D: exact nearest data point of every material point (Eq. 7).
        Returns (idx, |dq|^2 = d_e^2/2, second-best |dq|^2)."""
        zq = _metric.to_z(np.concatenate([eps, sig], axis=1), self.C)
        i1, d1, _, d2 = _nn.nn_top2(self.Z, zq)
        return i1.astype(np.int32), d1, d2

    def global_d2(self, eps, sig, idx) -> float:
        """Eq. (2): sum_e 1/2 w_e d_e^2(y_e, z_e)."""
        y = np.concatenate([eps, sig], axis=1)
        return float(np.sum(0.5 * self.w * _metric.local_d2(y, self.data[idx], self.C)))

    def solve(self, init_idx: np.ndarray, max_iter: int = 200) -> DDResult:
        idx = np.asarray(init_idx, dtype=np.int32).copy()
        res = None
        hist_pc, hist_pd, changed = [], [], []
        for it in range(1, max_iter + 1):
            u, eta, eps, sig = self.project_C(idx)
            hist_pc.append(self.global_d2(eps, sig, idx))
            new, d1, _ = self.project_D(eps, sig)
            hist_pd.append(float(np.sum(self.w * d1)))
            n_changed = int(np.count_nonzero(new != idx))
            changed.append(n_changed)
            res = DDResult(u, eta, eps, sig, idx.copy(), it, n_changed == 0,
                           hist_pc, hist_pd, changed)
            if n_changed == 0:
                break
            idx = new
        return res
