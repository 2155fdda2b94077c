"""Finite-element substrate of the DD constraint projection (FP64 oracle).

A box [0,lx]x[0,ly]x[0,lz] meshed by nx*ny*nz trilinear hexahedra with 2x2x2
Gauss points (Sec. 3: the cube example).  Provides the operators of Eq. (5)
and Eq. (6):

  K = A_e{ w_e B_e^T C B_e }                 (left-hand side of Eq. 5a/5b)
  E = A_e{ w_e B_e^T C eps*_e }              (Eq. 5a right-hand side)
  S = f - A_e{ w_e B_e^T sig*_e }            (Eq. 5b right-hand side)
  eps_e = B_e u,  sig_e = sig*_e + C B_e eta (Eq. 6a, 6b)

K is factorised once by sparse LU (Sec. 2 remarks that K is constant for
geometric linearity and constant C; Sec. 3.1 uses Eigen's SparseLU).

Numbering (shared with the GPU path only as an interface convention):
  node (i,j,k)        -> i + (nx+1)*(j + (ny+1)*k), dof = 3*node + component
  element (i,j,k)     -> i + nx*(j + ny*k)
  local node a        =  ax + 2*ay + 4*az   (offsets ax, ay, az in {0,1})
  Gauss point g       =  gx + 2*gy + 4*gz,  xi = (2*gx - 1)/sqrt(3), ...
  material point      =  8*element + g
  Voigt order (xx, yy, zz, yz, xz, xy), engineering shear strains.

Pinned by tests/test_oracle_fem.py: rigid-body null space of K, resultant of
the traction loads, the constant-strain patch test against the analytic
uniaxial solution, and exact strains of linear displacement fields.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

GP = 1.0 / np.sqrt(3.0)


def _local_offsets():
    return np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)])


class HexBox:
    def __init__(self, nx: int, ny: int, nz: int, C: np.ndarray,
                 lx: float = 1.0, ly: float = 1.0, lz: float = 1.0):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.lx, self.ly, self.lz = lx, ly, lz
        self.h = np.array([lx / nx, ly / ny, lz / nz])
        self.C = np.asarray(C, dtype=np.float64)
        self.n_nodes = (nx + 1) * (ny + 1) * (nz + 1)
        self.n_dof = 3 * self.n_nodes
        self.n_el = nx * ny * nz
        self.m = 8 * self.n_el
        self.w = float(np.prod(self.h)) / 8.0          # Gauss weight * det J
        off = _local_offsets()
        ei, ej, ek = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
        ei, ej, ek = (a.transpose(2, 1, 0).ravel() for a in (ei, ej, ek))   # element id order
        self.conn = np.stack([self.node_id(ei + o[0], ej + o[1], ek + o[2]) for o in off], axis=1)
        self.edofs = (3 * self.conn[:, :, None] + np.arange(3)[None, None, :]).reshape(self.n_el, 24)
        self.Bg = np.stack([self._B(g) for g in range(8)])          # [8, 6, 24]

    def node_id(self, i, j, k):
        return i + (self.nx + 1) * (j + (self.ny + 1) * k)

    def node_coords(self) -> np.ndarray:
        n = np.arange(self.n_nodes)
        i = n % (self.nx + 1)
        j = (n // (self.nx + 1)) % (self.ny + 1)
        k = n // ((self.nx + 1) * (self.ny + 1))
        return np.stack([i * self.h[0], j * self.h[1], k * self.h[2]], axis=1)

    def _B(self, g: int) -> np.ndarray:
        """Strain-displacement operator of one element at Gauss point g."""
        xi = np.array([(2 * (g & 1) - 1), (2 * ((g >> 1) & 1) - 1), (2 * ((g >> 2) & 1) - 1)]) * GP
        B = np.zeros((6, 24))
        for a, o in enumerate(_local_offsets()):
            s = 2.0 * o - 1.0                                   # node sign in [-1,1]^3
            f = 1.0 + s * xi
            dN = np.array([s[0] * f[1] * f[2], f[0] * s[1] * f[2], f[0] * f[1] * s[2]]) / 8.0
            dN = dN * 2.0 / self.h                              # d/dxi -> d/dx
            c = 3 * a
            B[0, c + 0] = dN[0]
            B[1, c + 1] = dN[1]
            B[2, c + 2] = dN[2]
            B[3, c + 1] = dN[2]; B[3, c + 2] = dN[1]
            B[4, c + 0] = dN[2]; B[4, c + 2] = dN[0]
            B[5, c + 0] = dN[1]; B[5, c + 1] = dN[0]
        return B

    # -- operators --------------------------------------------------------
    def element_K(self) -> np.ndarray:
        return sum(self.w * self.Bg[g].T @ self.C @ self.Bg[g] for g in range(8))

    def K(self) -> sp.csr_matrix:
        Ke = self.element_K()
        rows = np.repeat(self.edofs, 24, axis=1).ravel()
        cols = np.tile(self.edofs, (1, 24)).ravel()
        vals = np.tile(Ke.ravel(), self.n_el)
        return sp.coo_matrix((vals, (rows, cols)), shape=(self.n_dof, self.n_dof)).tocsr()

    def assemble_BT(self, s: np.ndarray) -> np.ndarray:
        """A_e{ w B_e^T s_e } for a stress-like field s [m, 6] at the Gauss points."""
        s = np.asarray(s, dtype=np.float64).reshape(self.n_el, 8, 6)
        fe = self.w * np.einsum("gij,egi->ej", self.Bg, s)             # [n_el, 24]
        out = np.zeros(self.n_dof)
        np.add.at(out, self.edofs.ravel(), fe.ravel())
        return out

    def strains(self, u: np.ndarray) -> np.ndarray:
        """eps_e = B_e u at every material point, [m, 6] (Eq. 6a)."""
        ue = np.asarray(u)[self.edofs]                                   # [n_el, 24]
        return np.einsum("gij,ej->egi", self.Bg, ue).reshape(self.m, 6)

    def top_traction_force(self, t0, tx=(0, 0, 0), ty=(0, 0, 0)) -> np.ndarray:
        """Consistent nodal forces of the traction t(x,y) = t0 + tx (x - lx/2)
        + ty (y - ly/2) on the face z = lz (2x2 Gauss per face quad)."""
        t0, tx, ty = (np.asarray(v, dtype=np.float64) for v in (t0, tx, ty))
        f = np.zeros(self.n_dof)
        hx, hy = self.h[0], self.h[1]
        wq = hx * hy / 4.0
        for i in range(self.nx):
            for j in range(self.ny):
                for gx in (-GP, GP):
                    for gy in (-GP, GP):
                        x = (i + 0.5 * (1 + gx)) * hx
                        y = (j + 0.5 * (1 + gy)) * hy
                        t = t0 + tx * (x - self.lx / 2) + ty * (y - self.ly / 2)
                        for ax in (0, 1):
                            for ay in (0, 1):
                                N = 0.25 * (1 + (2 * ax - 1) * gx) * (1 + (2 * ay - 1) * gy)
                                n = self.node_id(i + ax, j + ay, self.nz)
                                f[3 * n:3 * n + 3] += N * t * wq
        return f

    def top_rotation(self, theta: float) -> np.ndarray:
        """Displacement of the nodes on z = lz when the top face turns rigidly by
        theta (radians) about the vertical axis through its centre:
        u = (R(theta) - I)(x - x_c, y - y_c), u_z = 0; zero elsewhere."""
        xyz = self.node_coords()
        top = np.isclose(xyz[:, 2], self.lz)
        dx, dy = xyz[:, 0] - self.lx / 2, xyz[:, 1] - self.ly / 2
        c, s = np.cos(theta), np.sin(theta)
        u = np.zeros((self.n_nodes, 3))
        u[top, 0] = ((c - 1.0) * dx - s * dy)[top]
        u[top, 1] = (s * dx + (c - 1.0) * dy)[top]
        return u.ravel()

    def clamped_top(self) -> np.ndarray:
        """Boolean mask of every dof of the nodes on z = lz."""
        fixed = np.zeros(self.n_dof, dtype=bool)
        fixed[np.repeat(np.isclose(self.node_coords()[:, 2], self.lz), 3)] = True
        return fixed

    def clamped_bottom(self) -> np.ndarray:
        """Boolean mask of the fixed dofs: every dof of the nodes on z = 0."""
        fixed = np.zeros(self.n_dof, dtype=bool)
        k0 = self.node_coords()[:, 2] == 0.0
        fixed[np.repeat(k0, 3)] = True
        return fixed


class DirectSolver:
    """K restricted to the free dofs, factorised once by sparse LU.  A solve
    takes the values of the fixed dofs (zero by default) and moves their
    coupling to the right-hand side: K_ff x_f = rhs_f - K_fd x_d."""

    def __init__(self, K: sp.csr_matrix, fixed: np.ndarray):
        self.free = ~np.asarray(fixed, dtype=bool)
        Kff = K[self.free][:, self.free].tocsc()
        self.Kfd = K[self.free][:, ~self.free].tocsr()
        self.lu = spla.splu(Kff)
        self.n = K.shape[0]

    def solve(self, rhs: np.ndarray, prescribed: np.ndarray | None = None) -> np.ndarray:
        x = np.zeros(self.n)
        b = np.asarray(rhs, dtype=np.float64)[self.free]
        if prescribed is not None:
            xd = np.asarray(prescribed, dtype=np.float64)[~self.free]
            x[~self.free] = xd
            b = b - self.Kfd @ xd
        x[self.free] = self.lu.solve(b)
        return x
