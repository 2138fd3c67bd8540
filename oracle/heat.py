"""One implicit heat step, a box objective and its adjoint gradients (eq. heat_transfer
with the laser flux of eq. laser_gauss).

Readings: backward Euler with the conductivity lagged at the previous step; the unknown
is theta = T - T_ref so that the fixed bottom temperature T_ref is a homogeneous Dirichlet
condition; the top face carries the laser flux as a Neumann load; the other faces are
adiabatic.  The objective is J = 1/2 int_box (theta_h - theta*_h)^2 over the cells whose
centre lies in the box; dJ/dp = lambda^T df/dp and dJ/dk_q = -lambda^T (dA/dk_q) theta with
A^T lambda = dJ/dtheta.  Linear systems are solved with a sparse LU (a library primitive).
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import assemble as asm
from .basis import tensor_tables

DIRICHLET_BOTTOM = 1 << 4


def box_cells(dm, half, depth):
    ztop = dm.lo[2] + dm.hspan[2]
    c = dm.cell_origin + 0.5 * dm.cell_h[:, None]
    return np.nonzero((np.abs(c[:, 0]) <= half) & (np.abs(c[:, 1]) <= half) & (c[:, 2] >= ztop - depth))[0]


class HeatStep:
    """A theta^{n+1} = (rho c_p / dt) M theta^n + f_laser(p), Dirichlet rows zero."""

    def __init__(self, dm, rhocp, dt, kq=None, beta=None, k0=None, t_boil=None, T_prev_abs=None):
        self.dm = dm
        self.A = asm.heat_matrix(dm, rhocp, dt, k0=k0, t_boil=t_boil, T_prev=T_prev_abs, kq=kq, beta=beta)
        self.M = asm.mass_matrix(dm)
        self.rhocp, self.dt = rhocp, dt
        self._lu = None
        self._luT = None

    def rhs(self, theta_prev, laser):
        b = (self.rhocp / self.dt) * (self.M @ theta_prev) + asm.laser_rhs(self.dm, **laser)
        b[self.dm.dirichlet] = 0.0
        return b

    def solve(self, b):
        if self._lu is None:
            self._lu = spla.splu(self.A.tocsc())
        return self._lu.solve(b)

    def solve_transpose(self, g):
        if self._luT is None:
            self._luT = spla.splu(self.A.T.tocsc())
        return self._luT.solve(g)


def objective(dm, theta, theta_target, cells):
    Mb = asm.mass_matrix(dm, cells)
    e = theta - theta_target
    return 0.5 * e @ (Mb @ e), Mb @ e


def gradients(step, theta_prev, theta_target, laser, cells):
    """J, dJ/d(P, r, x0, y0) and dJ/dk_q (ncell, nq) of one heat step."""
    dm = step.dm
    theta = step.solve(step.rhs(theta_prev, laser))
    J, dJ = objective(dm, theta, theta_target, cells)
    dJ[dm.dirichlet] = 0.0
    lam = step.solve_transpose(dJ)
    dF = asm.laser_rhs(dm, **laser, derivatives=True)
    g_laser = dF @ lam
    _, G, w = tensor_tables(dm.degree, dm.degree + 1)
    lam_l = asm.local_values(dm, lam)
    th_l = asm.local_values(dm, theta)
    gl = np.einsum("qid,ci->cqd", G, lam_l)
    gt = np.einsum("qid,ci->cqd", G, th_l)
    g_kq = -(w[None, :] * dm.cell_h[:, None]) * np.einsum("cqd,cqd->cq", gl, gt)
    return J, g_laser, g_kq, theta, lam
