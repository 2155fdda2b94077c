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


def test_top_rotation_field():
    """The prescribed field of the top face is the rigid turn of the face
    about its centre: zero at the centre, length-preserving for the face, and
    counter-clockwise seen from above for a positive angle (closed form)."""
    b = box(4)
    th = np.radians(2.0)
    u = b.top_rotation(th).reshape(-1, 3)
    xyz = b.node_coords()
    top = np.isclose(xyz[:, 2], b.lz)
    assert np.all(u[~top] == 0.0) and np.all(u[:, 2] == 0.0)
    p = xyz[top, :2] - np.array([b.lx / 2, b.ly / 2])
    q = p + u[top, :2]
    assert np.allclose(np.linalg.norm(q, axis=1), np.linalg.norm(p, axis=1), atol=1e-15)
    ang = np.arctan2(q[:, 1], q[:, 0]) - np.arctan2(p[:, 1], p[:, 0])
    ok = np.linalg.norm(p, axis=1) > 1e-12
    assert np.allclose(np.mod(ang[ok] + np.pi, 2 * np.pi) - np.pi, th, atol=1e-12)


def test_prescribed_linear_rotation_reproduced_exactly():
    """A linearised rigid rotation u = theta e_z x (x - c) prescribed on both
    the top and the bottom face is a strain-free field in the finite element
    space: the lifted solve must return it at every interior node and give
    zero strain (closed form)."""
    b = box(4)
    th = 1e-3
    xyz = b.node_coords()
    lin = np.zeros((b.n_nodes, 3))
    lin[:, 0] = -th * (xyz[:, 1] - b.ly / 2)
    lin[:, 1] = th * (xyz[:, 0] - b.lx / 2)
    fixed = b.clamped_bottom() | b.clamped_top()
    sol = fem.DirectSolver(b.K(), fixed).solve(np.zeros(b.n_dof), prescribed=lin.ravel())
    assert np.allclose(sol, lin.ravel(), atol=1e-14)
    assert np.abs(b.strains(sol)).max() < 1e-13


def test_lifted_solve_satisfies_the_equations():
    """With the top face turned and the bottom clamped, the solution takes the
    prescribed values on the fixed dofs and balances the load on the free
    ones (K u = f there), checked against the assembled K."""
    b = box(3)
    K = b.K()
    fixed = b.clamped_bottom() | b.clamped_top()
    ud = b.top_rotation(np.radians(2.0))
    f = np.random.default_rng(0).standard_normal(b.n_dof) * 1e-3
    sol = fem.DirectSolver(K, fixed).solve(f, prescribed=ud)
    assert np.array_equal(sol[fixed], ud[fixed])
    r = (K @ sol - f)[~fixed]
    assert np.abs(r).max() < 1e-10 * np.abs(K @ sol).max()
