"""Pins of the oracle's finite-element operators (Eq. 5, Eq. 6)."""
import numpy as np

import dd_inputs as I
from oracle import fem


def box(n=3, C=None, **kw):
    return fem.HexBox(n, n + 1, n + 2, I.isotropic_C() if C is None else C, **kw)


def rigid_modes(b):
    x = b.node_coords()
    modes = []
    for c in range(3):
        u = np.zeros((b.n_nodes, 3)); u[:, c] = 1.0; modes.append(u.ravel())
    for (a, c) in ((0, 1), (1, 2), (0, 2)):      # infinitesimal rotations
        u = np.zeros((b.n_nodes, 3)); u[:, a] = -x[:, c]; u[:, c] = x[:, a]; modes.append(u.ravel())
    return modes


def test_element_stiffness_spectrum():
    b = box(2, lx=0.7, ly=1.1, lz=0.9)
    ev = np.linalg.eigvalsh(b.element_K())
    assert np.allclose(ev[:6], 0, atol=1e-12 * ev[-1])
    assert ev[6] > 1e-3 * ev[-1]


def test_rigid_body_null_space_of_K():
    b = box(2)
    K = b.K()
    assert abs(K - K.T).max() < 1e-14 * abs(K).max()
    for u in rigid_modes(b):
        assert np.abs(K @ u).max() < 1e-12 * abs(K).max() * np.abs(u).max()


def test_linear_displacement_gives_exact_strain():
    b = box(2, lx=2.0, ly=1.0, lz=0.5)
    A = np.array([[1.0, 2.0, -0.5], [0.3, -1.0, 0.7], [0.2, 0.4, 3.0]])
    u = (b.node_coords() @ A.T).ravel()                  # u_i = A_ij x_j
    eps = b.strains(u)
    want = [A[0, 0], A[1, 1], A[2, 2], A[1, 2] + A[2, 1], A[0, 2] + A[2, 0], A[0, 1] + A[1, 0]]
    assert np.allclose(eps, np.array(want)[None, :], atol=1e-13)


def test_traction_resultants():
    t = 1e-3
    b = fem.HexBox(4, 4, 4, I.isotropic_C())
    x = b.node_coords()
    for name, F, Mz_or_My in (("tension", (0, 0, t), None), ("torsion", (0, 0, 0), t / 3),
                              ("bending", (0, 0, 0), t / 6)):
        L = I.load_case(name, t)
        f = b.top_traction_force(L.t0, L.tx, L.ty).reshape(-1, 3)
        assert np.allclose(f.sum(0), F, atol=1e-15)
        if name == "torsion":   # M_z = int (x-1/2) t_y - (y-1/2) t_x dA = 2t (1/12 + 1/12)
            Mz = ((x[:, 0] - 0.5) * f[:, 1] - (x[:, 1] - 0.5) * f[:, 0]).sum()
            assert np.isclose(Mz, Mz_or_My, rtol=1e-12)
        if name == "bending":   # M = int (x-1/2) t_z dA = 2t/12
            My = ((x[:, 0] - 0.5) * f[:, 2]).sum()
            assert np.isclose(My, Mz_or_My, rtol=1e-12)


def test_patch_test_uniaxial_tension():
    """Rollers on x=0, y=0, z=0 and a uniform top traction: the exact FE
    solution is the homogeneous uniaxial field eps_zz = t/E, eps_xx = eps_yy
    = -nu t/E (trilinear hexes pass the constant-strain patch test)."""
    E, nu, t = 1.0, 0.3, 1e-3
    b = fem.HexBox(3, 2, 4, I.isotropic_C(E, nu), lx=1.0, ly=0.5, lz=2.0)
    x = b.node_coords()
    fixed = np.zeros(b.n_dof, bool)
    fixed[0::3] = x[:, 0] == 0.0
    fixed[1::3] = x[:, 1] == 0.0
    fixed[2::3] = x[:, 2] == 0.0
    s = fem.DirectSolver(b.K(), fixed)
    u = s.solve(b.top_traction_force((0, 0, t)))
    eps = b.strains(u)
    want = np.array([-nu * t / E, -nu * t / E, t / E, 0, 0, 0])
    assert np.allclose(eps, want[None, :], rtol=0, atol=1e-12 * t)


def test_clamped_mask():
    b = box(2)
    fixed = b.clamped_bottom()
    assert fixed.sum() == 3 * (b.nx + 1) * (b.ny + 1)
