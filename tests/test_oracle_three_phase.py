"""Pins of the three-phase coefficients, the Darcy damping and the trace-corrected viscous stress
in the oracle's Oseen operator (Sections 3.1-3.3 of the melt-pool model and the stress of
Section 2.1), by closed forms and reductions to the two-phase operator."""
import numpy as np
import pytest

import synthetic as syn
from oracle import assemble as asm
from oracle import coeffs as co
from oracle import mesh as omesh

TI = syn.TI64
TS, TL = 1933.0, 2200.0


def test_solid_fraction_and_smooth_heaviside():
    assert co.solid_fraction(np.array([1000.0, TS, 0.5 * (TS + TL), TL, 3000.0]), TS, TL).tolist() == \
        [1.0, 1.0, 0.5, 0.0, 0.0]
    assert co.heaviside_solid(np.array([0.0, 0.5, 1.0])).tolist() == [0.0, 0.5, 1.0]
    # dH_s/dT vanishes at both isotherms (the point of the cubic)
    h = 1e-6
    for f in (0.0, 1.0):
        d = (co.heaviside_solid(f + h) - co.heaviside_solid(f - h)) / (2 * h)
        assert abs(d) < 1e-9


def test_three_phase_laws_reduce_to_the_two_phase_ones():
    H = np.linspace(0, 1, 11)
    assert np.allclose(co.three_phase_mix(H, 0.0, 7.0, 3.0, 0.5), co.arithmetic_mix(H, 3.0, 0.5), rtol=0, atol=1e-15)
    assert np.allclose(co.three_phase_density(H, 0.0, 9.0, 4087.0, 4.087), co.reciprocal_density(H, 4087.0, 4.087),
                       rtol=1e-15)
    assert co.three_phase_mix(1.0, 1.0, 7.0, 3.0, 0.5) == 7.0
    assert co.three_phase_density(1.0, 1.0, 9.0, 4087.0, 4.087) == pytest.approx(9.0, rel=1e-15)


def test_darcy_coefficient_values():
    # eq. (darcy_damping_force): K(f_s = 1) = C / b, K(0) = 0.  (The text quotes 1e13 for C = 1e12,
    # b = 1, which the formula does not give; the formula is followed.)
    assert co.darcy_coefficient(1.0, 1e12, 1.0) == 1e12
    assert co.darcy_coefficient(0.0, 1e12, 1.0) == 0.0
    assert co.darcy_coefficient(0.5, 8.0, 1.0) == pytest.approx(8.0 * 0.25 / 1.125, rel=1e-15)


def _maps(n, faces=0):
    return omesh.uniform_dofmap(n, (0, 0, 0), (1, 1, 1), 2, faces), omesh.uniform_dofmap(n, (0, 0, 0), (1, 1, 1), 1, 0)


def _fields(dmu, seed=3):
    x = dmu.dof_coords()
    t1, t2 = syn.wavy_plane_phases(seed)
    phi = syn.initial_level_set(syn.wavy_plane_distance(*x.T, t1, t2), 0.25)
    beta = np.array(syn.convection_field(*x.T, seed, (0, 0, 0), (1, 1, 1)))
    return x, phi, beta


SOLID = dict(rho_s=5000.0, mu_s=2e-2, t_solidus=TS, t_liquidus=TL)
DARCY = dict(C=1e6, b=1.0, t_solidus=TS, t_liquidus=TL)


def test_hot_melt_reduces_to_the_two_phase_operator():
    dmu, dmp = _maps(3, 0b011111)
    x, phi, beta = _fields(dmu)
    T = np.full(dmu.n_dofs, 2500.0)                       # above T_l: f_s = 0 everywhere
    base = asm.oseen_matrix(dmu, dmp, phi, beta, 8.0, TI["rho_l"], TI["rho_g"], TI["mu_l"], TI["mu_g"])
    three = asm.oseen_matrix(dmu, dmp, phi, beta, 8.0, TI["rho_l"], TI["rho_g"], TI["mu_l"], TI["mu_g"], T=T,
                             solid=SOLID, darcy=DARCY)
    assert abs(three - base).max() <= 1e-15 * abs(base).max()


def test_darcy_in_a_frozen_dense_block_is_C_over_b_times_the_mass():
    dmu, dmp = _maps(3)
    x = dmu.dof_coords()
    phi = np.ones(dmu.n_dofs)                             # dense everywhere: H = 1
    beta = np.zeros((3, dmu.n_dofs))
    T = np.full(dmu.n_dofs, 1500.0)                       # below T_s: f_s = 1
    args = (dmu, dmp, phi, beta, 8.0, TI["rho_l"], TI["rho_g"], TI["mu_l"], TI["mu_g"])
    diff = (asm.oseen_matrix(*args, T=T, darcy=DARCY) - asm.oseen_matrix(*args)).tocsr()
    nu = dmu.n_dofs
    for c in range(3):
        blk = diff[c * nu:(c + 1) * nu, c * nu:(c + 1) * nu]
        assert blk.sum() == pytest.approx(DARCY["C"] / DARCY["b"] * 1.0, rel=1e-13)   # C/b |Omega|
        off = diff[c * nu:(c + 1) * nu, :]
        assert abs(off.sum() - blk.sum()) <= 1e-12 * abs(blk.sum())
    assert abs(diff - diff.T).max() <= 1e-15 * abs(diff).max()    # a mass term: symmetric


def test_trace_correction_vanishes_on_divergence_free_fields():
    dmu, dmp = _maps(3)            # no Dirichlet rows: they would cut the field at the walls
    x, phi, beta = _fields(dmu)
    args = (dmu, dmp, phi, beta, 8.0, TI["rho_l"], TI["rho_g"], TI["mu_l"], TI["mu_g"])
    A0, A1 = asm.oseen_matrix(*args), asm.oseen_matrix(*args, trace_correction=True)
    # (y, z, x) and a rigid rotation: div = 0, reproduced exactly by Q2
    for u3 in (np.stack([x[:, 1], x[:, 2], x[:, 0]]), np.stack([-x[:, 1], x[:, 0], np.zeros(len(x))])):
        u = np.concatenate([u3.ravel(), np.zeros(dmp.n_dofs)])
        r0, r1 = A0 @ u, A1 @ u
        assert np.abs(r1 - r0).max() <= 1e-13 * np.abs(A0).max() * np.abs(u).max()
    assert abs(A1 - A1.T).max() > 1e-6 * abs(A1).max()     # the correction is not symmetric


def test_trace_correction_on_a_flat_interface_is_a_boundary_flux():
    """phi = phi(z) decreasing: n = -e_z at every Gauss point.  With u = (x, 0, 0) (div u = 1) and
    constant mu, the correction of the z-rows is -2 mu int d_z N_i = -2 mu (int_top N_i - int_bottom N_i);
    over the top-face nodes it sums to -2 mu, over the bottom-face nodes to +2 mu, elsewhere 0, and
    the x- and y-rows do not change."""
    n = 4
    dmu, dmp = _maps(n)
    x = dmu.dof_coords()
    phi = np.tanh((0.5 - x[:, 2]) / 0.5)
    beta = np.zeros((3, dmu.n_dofs))
    mu = 0.7
    args = (dmu, dmp, phi, beta, 8.0, TI["rho_l"], TI["rho_g"], mu, mu)
    d = (asm.oseen_matrix(*args, trace_correction=True) - asm.oseen_matrix(*args)) @ np.concatenate(
        [x[:, 0], np.zeros(2 * dmu.n_dofs + dmp.n_dofs)])
    nu = dmu.n_dofs
    assert np.abs(d[:2 * nu]).max() <= 1e-13
    dz = d[2 * nu:3 * nu]
    top, bottom = np.isclose(x[:, 2], 1.0), np.isclose(x[:, 2], 0.0)
    assert dz[top].sum() == pytest.approx(-2 * mu, rel=1e-12)
    assert dz[bottom].sum() == pytest.approx(2 * mu, rel=1e-12)
    assert np.abs(dz[~(top | bottom)]).max() <= 1e-13
