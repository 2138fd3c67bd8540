"""Pins of the oracle's heat-step inputs (no GPU): the top-face laser load of eq. (laser_gauss)
and the temperature-dependent conductivity k(T_h^n) of the heat workloads.

Each check compares the oracle with a value the mathematics fixes independently of the oracle's
own code path: the closed-form integral of the Gaussian flux, the face weights of the Q2 basis,
the convergence order of the Gauss rule, the exact interpolation of quadratics by Q2, and values
of the law k(T) = k0 (1 + 0.5 T / T_b) at chosen temperatures.
"""
import math

import numpy as np

from oracle import assemble as asm
from oracle import mesh

LO, HI = (-3e-4, -3e-4, -3e-4), (3e-4, 3e-4, 3e-4)   # the 600 um box of Section 4.3
K0, TB = 28.63, 3133.0


def _top_dofs(dm):
    x = dm.dof_coords()
    return np.isclose(x[:, 2], HI[2], rtol=0, atol=1e-9 * (HI[2] - LO[2])), x


def _gauss_integral_1d(a, b, centre, radius):
    """int_a^b exp(-2 (s - centre)^2 / radius^2) ds by the error function."""
    c = math.sqrt(2.0) / radius
    return 0.5 * math.sqrt(math.pi) / c * (math.erf(c * (b - centre)) - math.erf(c * (a - centre)))


def _exact_face_power(power, radius, x0, y0, chi):
    """Closed-form integral of eq. (laser_gauss)'s flux 2 chi P / (pi r^2) exp(-2 rho^2 / r^2) over
    the top face [LO, HI]^2."""
    ix = _gauss_integral_1d(LO[0], HI[0], x0, radius)
    iy = _gauss_integral_1d(LO[1], HI[1], y0, radius)
    return 2.0 * chi * power / (math.pi * radius ** 2) * ix * iy


def test_laser_load_sums_to_the_absorbed_power_at_sixth_order():
    """Q2 shape functions sum to one on the face, so sum_i f_i is the composite 3x3 Gauss rule of
    the flux over the top face; it converges to the closed-form integral (-> chi P for a beam
    well inside the face) at the rule's order h^6."""
    P, r, x0, y0, chi = 200.0, 50e-6, 7e-6, -11e-6, 0.35
    exact = _exact_face_power(P, r, x0, y0, chi)
    assert abs(exact - chi * P) < 1e-12 * chi * P          # the beam sits well inside the 600 um face
    errs = []
    for n in (16, 32):
        dm = mesh.uniform_dofmap(n, LO, HI, 2, 1 << 4)
        f = asm.laser_rhs(dm, P, r, x0, y0, chi)
        errs.append(abs(f.sum() - exact) / exact)
    assert errs[1] < 2e-6
    assert errs[0] / errs[1] > 40.0                          # h^6: 64 per halving, minus a margin


def test_laser_load_lives_on_the_top_face_only():
    dm = mesh.uniform_dofmap(6, LO, HI, 2, 1 << 4)
    f = asm.laser_rhs(dm, 200.0, 150e-6, 0.0, 0.0, 0.35)
    top, _ = _top_dofs(dm)
    assert np.all(f[~top] == 0.0)
    assert np.count_nonzero(f[top]) == top.sum() and f.sum() > 0.0


def test_constant_flux_gives_the_q2_face_weights():
    """With a beam much wider than the face the flux is the constant q0 = 2 chi P / (pi r^2) to 1e-12;
    the load of top node (I, J) is then q0 h^2 w(I) w(J) with the 1D Q2 weights of Simpson's rule per
    cell: 1/6 at the two domain ends, 2/3 at a cell midpoint, 1/3 at a vertex shared by two cells.
    Their sum is q0 times the face area."""
    n = 5
    dm = mesh.uniform_dofmap(n, LO, HI, 2, 1 << 4)
    P, r, chi = 200.0, 1e3, 0.35
    q0 = 2.0 * chi * P / (math.pi * r ** 2)
    f = asm.laser_rhs(dm, P, r, 0.0, 0.0, chi)
    top, x = _top_dofs(dm)
    h = (HI[0] - LO[0]) / n
    lat = np.rint((x[top, :2] - np.array(LO[:2])) / (0.5 * h)).astype(int)   # lattice index 0..2n

    def w1(i):
        return np.where((i == 0) | (i == 2 * n), 1.0 / 6.0, np.where(i % 2 == 1, 2.0 / 3.0, 1.0 / 3.0))

    want = q0 * h * h * w1(lat[:, 0]) * w1(lat[:, 1])
    assert np.allclose(f[top], want, rtol=1e-11, atol=0)
    area = (HI[0] - LO[0]) * (HI[1] - LO[1])
    assert abs(f.sum() - q0 * area) < 1e-11 * q0 * area


def test_laser_load_derivatives_are_the_loads_of_the_closed_form_derivatives():
    """d(sum f)/dP = sum f / P exactly, and d(sum f)/dx0 vanishes for a centred beam (symmetry)."""
    dm = mesh.uniform_dofmap(8, LO, HI, 2, 1 << 4)
    f = asm.laser_rhs(dm, 200.0, 50e-6, 0.0, 0.0, 0.35)
    d = asm.laser_rhs(dm, 200.0, 50e-6, 0.0, 0.0, 0.35, derivatives=True)
    assert abs(d[0].sum() - f.sum() / 200.0) < 1e-13 * f.sum()
    assert abs(d[2].sum()) < 1e-12 * abs(d[2]).sum()
    assert abs(d[3].sum()) < 1e-12 * abs(d[3]).sum()


def test_conductivity_law_values():
    """k(T) = k0 (1 + 0.5 T / T_b): k0 at T = 0, 1.5 k0 at the boiling point, 2 k0 at twice it."""
    from oracle import coeffs
    assert coeffs.conductivity_of_temperature(0.0, K0, TB) == K0
    assert abs(coeffs.conductivity_of_temperature(TB, K0, TB) - 1.5 * K0) < 1e-15 * K0
    assert abs(coeffs.conductivity_of_temperature(2 * TB, K0, TB) - 2.0 * K0) < 1e-15 * K0


def _unit_stiffness(dm):
    nq = (dm.degree + 1) ** 3
    return asm.assemble_scalar(dm, np.zeros((dm.n_cells, nq)), diff=np.ones((dm.n_cells, nq)))


def test_heat_conductivity_from_a_constant_temperature_scales_the_unit_stiffness():
    """For T^n = T_b everywhere the stiffness part of the heat operator is 1.5 k0 times the
    unit-coefficient stiffness (the latter pinned by the 1D rational Q2 matrices)."""
    dm = mesh.uniform_dofmap(3, LO, HI, 2)
    T = np.full(dm.n_dofs, TB)
    m, kq, conv = asm.heat_coefficients(dm, 4087.0 * 1130.0, 1e-5, K0, TB, T_prev=T)
    assert conv is None
    assert np.allclose(kq, 1.5 * K0, rtol=1e-15, atol=0)
    K = asm.assemble_scalar(dm, 0 * m, diff=kq)
    K1 = _unit_stiffness(dm)
    assert abs(K - 1.5 * K0 * K1).max() <= 1e-14 * abs(K).max()
    # and the mass part is (rho c_p / dt) times the mass matrix, whose entries sum to the volume
    M = asm.assemble_scalar(dm, m)
    vol = np.prod(np.array(HI) - np.array(LO))
    assert abs(M.sum() - 4087.0 * 1130.0 / 1e-5 * vol) < 1e-12 * abs(M.sum())


def test_heat_conductivity_at_the_gauss_points_of_a_quadratic_temperature():
    """Q2 interpolates T^n = a + b z + c z^2 exactly, so k at each Gauss point is the law at the
    exact temperature there; the Gauss points of a cell with lower corner z0 and edge h sit at
    z0 + h (1/2 - sqrt(15)/10, 1/2, 1/2 + sqrt(15)/10)."""
    n = 4
    dm = mesh.uniform_dofmap(n, LO, HI, 2, 1 << 4)
    a, b, c = 500.0, 4e6, 2e9
    z = dm.dof_coords()[:, 2]
    T = a + b * z + c * z * z
    _, kq, _ = asm.heat_coefficients(dm, 1.0, 1.0, K0, TB, T_prev=T)
    h = (HI[2] - LO[2]) / n
    g = np.array([0.5 - math.sqrt(15.0) / 10.0, 0.5, 0.5 + math.sqrt(15.0) / 10.0])
    zq = dm.cell_origin[:, 2][:, None] + h * np.array([g[q // 9] for q in range(27)])[None, :]
    Tq = a + b * zq + c * zq * zq
    want = K0 * (1.0 + 0.5 * Tq / TB)
    assert np.allclose(kq, want, rtol=1e-13, atol=0)
    # the same operator through the per-Gauss-point path
    A1 = asm.heat_matrix(dm, 1.0, 1.0, K0, TB, T_prev=T)
    A2 = asm.heat_matrix(dm, 1.0, 1.0, kq=want)
    assert abs(A1 - A2).max() <= 1e-13 * abs(A1).max()
