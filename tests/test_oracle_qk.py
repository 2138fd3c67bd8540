"""Pins of the oracle's Q3/Q4 elements (Appendix B: continuous Lagrange elements of degree k with
(k+1)^3 Gauss points): Gauss-Lobatto support points in closed form, the Lagrange property, exact
reproduction of polynomials of degree k per axis by the mass and stiffness forms (the Gauss rule is
exact to degree 2k + 1), constants in the kernel of the stiffness, and symmetry."""
import numpy as np
import pytest

import synthetic as syn
from oracle import assemble as asm
from oracle import mesh as omesh
from oracle.basis import lagrange_1d, lagrange_nodes


def test_gauss_lobatto_points_closed_forms():
    r5, r37 = 1.0 / np.sqrt(5.0), np.sqrt(3.0 / 7.0)
    assert np.allclose(lagrange_nodes(3), [0.0, (1 - r5) / 2, (1 + r5) / 2, 1.0], rtol=0, atol=1e-15)
    assert np.allclose(lagrange_nodes(4), [0.0, (1 - r37) / 2, 0.5, (1 + r37) / 2, 1.0], rtol=0, atol=1e-15)
    assert np.array_equal(lagrange_nodes(2), [0.0, 0.5, 1.0])


@pytest.mark.parametrize("k", [3, 4])
def test_lagrange_property(k):
    L, dL = lagrange_1d(k, lagrange_nodes(k))
    assert np.abs(L - np.eye(k + 1)).max() <= 1e-13
    assert np.abs(dL.sum(axis=0)).max() <= 1e-12          # the basis sums to one


def _poly(X, pa, pb, pc):
    return X[:, 0] ** pa * X[:, 1] ** pb * X[:, 2] ** pc


@pytest.mark.parametrize("k", [3, 4])
def test_mass_and_stiffness_reproduce_degree_k_polynomials(k):
    n = 2
    dm = omesh.uniform_dofmap(n, (0, 0, 0), (1, 1, 1), k)
    X = dm.dof_coords()
    phi = np.zeros(dm.n_dofs)
    M = asm.helmholtz_matrix(dm, phi, 1.0, 0.0, 0.0)            # a = 0: mass only
    K = asm.helmholtz_matrix(dm, phi, 0.0, 1.0, 1.0)            # a = 1, no mass
    one = np.ones(dm.n_dofs)
    # int x^k y^(k-1) z = 1/(k+1) 1/k 1/2
    u = _poly(X, k, k - 1, 1)
    assert one @ (M @ u) == pytest.approx(1.0 / ((k + 1) * k * 2), rel=1e-13)
    # int (d/dx x^k)^2 = k^2 / (2k - 1);  grad x^k . grad y^k = 0
    xk, yk = _poly(X, k, 0, 0), _poly(X, 0, k, 0)
    assert xk @ (K @ xk) == pytest.approx(k * k / (2.0 * k - 1.0), rel=1e-12)
    assert abs(xk @ (K @ yk)) <= 1e-12
    # u = x^2 y, v = x y^2: int grad u . grad v = int 2 x y^3 + 2 x^3 y = 1/2
    assert _poly(X, 2, 1, 0) @ (K @ _poly(X, 1, 2, 0)) == pytest.approx(0.5, rel=1e-12)
    assert np.abs(K @ one).max() <= 1e-12 * abs(K).max()


@pytest.mark.parametrize("k", [3, 4])
def test_variable_coefficient_operator_is_symmetric_with_constant_kernel(k):
    dm = omesh.uniform_dofmap(2, (0, 0, 0), (1, 1, 1), k)
    X = dm.dof_coords()
    phi = syn.initial_level_set(syn.sphere_distance(*X.T), 0.25)
    A = asm.helmholtz_matrix(dm, phi, 0.0, 1000.0, 1.0)
    assert abs(A - A.T).max() <= 1e-15 * abs(A).max() * 10
    assert np.abs(A @ np.ones(dm.n_dofs)).max() <= 1e-12 * abs(A).max()
