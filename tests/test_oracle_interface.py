"""Pins of the oracle's interface source terms (Section 2.4 and the evaporation model of Section
5.2) against closed forms: mass-flux laws, the unit integrals of the regularised delta functions,
and an exact identity for delta on a flat interface."""
import numpy as np
import pytest
from scipy import integrate

import synthetic as syn
from oracle import coeffs as co
from oracle import interface as oi
from oracle import mesh as omesh

EV = syn.EVAPORATION
TI = syn.TI64


def params(model="tanasawa", heaviside="tanh", eps=None, recoil=True):
    return dict(rho_l=TI["rho_l"], rho_g=TI["rho_g"], rhocp_l=TI["rho_l"] * TI["cp_l"],
                rhocp_g=TI["rho_g"] * TI["cp_g"], heaviside=heaviside, eps=eps, model=model, recoil=recoil, **EV)


def test_mass_flux_laws_at_and_around_the_boiling_point():
    Tv, M, R = EV["t_boil"], EV["molar_mass"], oi.R_GAS
    # Clausius-Clapeyron is anchored at p_sat(T_v) = p_amb
    assert oi.saturated_vapour_pressure(Tv, EV["p_amb"], EV["h_v"], M, Tv) == pytest.approx(EV["p_amb"], rel=1e-15)
    ref = 0.82 * EV["sticking"] * EV["p_amb"] * np.sqrt(M / (2 * np.pi * R * Tv))
    assert oi.mass_flux_knight(Tv, EV["p_amb"], EV["h_v"], M, Tv, EV["sticking"]) == pytest.approx(ref, rel=1e-15)
    assert oi.recoil_anisimov(Tv, EV["p_amb"], EV["h_v"], M, Tv) == pytest.approx(0.54 * EV["p_amb"], rel=1e-15)
    assert oi.mass_flux_tanasawa(Tv + 2.0, 0.25, Tv) == 0.5
    # d ln p_sat / dT = h_v M / (R T^2) (Clausius-Clapeyron), by central differences
    for T in (2500.0, 3133.0, 3700.0):
        dT = 1e-3
        lp = lambda t: np.log(oi.saturated_vapour_pressure(t, EV["p_amb"], EV["h_v"], M, Tv))
        fd = (lp(T + dT) - lp(T - dT)) / (2 * dT)
        assert fd == pytest.approx(EV["h_v"] * M / (R * T * T), rel=1e-7)
    # the Anisimov pressure is 0.54 p_sat at every temperature (same exponent)
    T = np.array([2000.0, 3133.0, 4000.0])
    assert np.allclose(oi.recoil_anisimov(T, EV["p_amb"], EV["h_v"], M, Tv),
                       0.54 * oi.saturated_vapour_pressure(T, EV["p_amb"], EV["h_v"], M, Tv), rtol=1e-14)


def test_delta_weights_have_unit_integral_across_the_interface():
    rl, rg = TI["rho_l"], TI["rho_g"]
    cl, cg = TI["rho_l"] * TI["cp_l"], TI["rho_g"] * TI["cp_g"]
    # delta dn = dH: int delta_rho = c_rho int_0^1 rho(H) dH = 1
    v, _ = integrate.quad(lambda H: co.reciprocal_density(H, rl, rg), 0.0, 1.0, epsabs=0, epsrel=1e-12, limit=200)
    assert oi.c_rho(rl, rg) * v == pytest.approx(1.0, rel=1e-11)
    # reading: delta_rhocp carries (rho c_p)(H)^2; c_rhocp normalises exactly that weight
    v2, _ = integrate.quad(lambda H: co.arithmetic_mix(H, cl, cg) ** 2, 0.0, 1.0, epsabs=0, epsrel=1e-12)
    assert oi.c_rhocp(cl, cg) * v2 == pytest.approx(1.0, rel=1e-12)
    # the printed single power would not integrate to one for these contrasts
    v1, _ = integrate.quad(lambda H: co.arithmetic_mix(H, cl, cg), 0.0, 1.0)
    assert abs(oi.c_rhocp(cl, cg) * v1 * cl - 1.0) > 0.1


def flat_interface(n, dirichlet_faces=0, eps=None):
    dmu = omesh.uniform_dofmap(n, (0, 0, 0), (1, 1, 1), 2, dirichlet_faces)
    dmp = omesh.uniform_dofmap(n, (0, 0, 0), (1, 1, 1), 1, 0)
    eps = 2.0 / n if eps is None else eps
    z = dmu.dof_coords()[:, 2]
    phi = np.tanh((0.5 - z) / (2 * eps))
    return dmu, dmp, phi, eps


@pytest.mark.parametrize("n", [6, 8, 10])
def test_delta_integral_on_a_flat_interface_is_exact(n):
    """phi_h depends on z only and decreases monotonically, so delta = -d_z phi_h / 2 is a linear
    polynomial per cell, which the 3-point rule integrates exactly: int delta = (phi(0) - phi(1))/2 =
    tanh(1 / (4 eps)).  The pressure loads sum it through the Q1 partition of unity."""
    dmu, dmp, phi, eps = flat_interface(n)
    T = np.full(dmu.n_dofs, EV["t_boil"] + 1.0)
    p = params("tanasawa", eps=eps)
    f_u, f_p, f_T = oi.interface_sources(dmu, dmp, phi, T, p)
    mdot = EV["tanasawa"]
    exact = mdot * (1 / TI["rho_l"] - 1 / TI["rho_g"]) * np.tanh(1.0 / (4.0 * eps))
    assert f_p.sum() == pytest.approx(exact, rel=1e-13)


def _closed_form_weights(eps):
    """int delta_rho and int delta_rhocp across z in (0, 1) for phi = tanh((0.5 - z)/(2 eps)):
    c int_{H(1)}^{H(0)} w(H) dH in closed form."""
    rl, rg = TI["rho_l"], TI["rho_g"]
    cl, cg = TI["rho_l"] * TI["cp_l"], TI["rho_g"] * TI["cp_g"]
    t = np.tanh(1.0 / (4.0 * eps))
    Ht, Hb = 0.5 * (1 + t), 0.5 * (1 - t)
    a, b = 1 / rl, 1 / rg            # 1/rho = a H + b (1 - H)
    F = lambda H: np.log(b + (a - b) * H) / (a - b)
    w_rho = oi.c_rho(rl, rg) * (F(Ht) - F(Hb))
    G = lambda H: (cg + (cl - cg) * H) ** 3 / (3 * (cl - cg))
    w_cp = oi.c_rhocp(cl, cg) * (G(Ht) - G(Hb))
    return w_rho, w_cp


def test_recoil_and_cooling_loads_converge_to_the_closed_form():
    errs = []
    for n in (8, 16, 32):     # fixed interface width, refined mesh
        dmu, dmp, phi, eps = flat_interface(n, eps=0.1)
        T = np.full(dmu.n_dofs, EV["t_boil"] + 40.0)
        p = params("knight", eps=eps)
        f_u, f_p, f_T = oi.interface_sources(dmu, dmp, phi, T, p)
        nu = dmu.n_dofs
        Tq = EV["t_boil"] + 40.0
        mdot = oi.mass_flux_knight(Tq, EV["p_amb"], EV["h_v"], EV["molar_mass"], EV["t_boil"], EV["sticking"])
        p_an = oi.recoil_anisimov(Tq, EV["p_amb"], EV["h_v"], EV["molar_mass"], EV["t_boil"])
        w_rho, w_cp = _closed_form_weights(eps)
        w_delta = np.tanh(1.0 / (4.0 * eps))
        # n_Gamma = grad phi / |grad phi| = -e_z: the net recoil load points down, into the liquid
        fz = -(p_an * w_rho - mdot * mdot * (1 / TI["rho_g"] - 1 / TI["rho_l"]) * w_delta)
        assert f_u[2 * nu:].sum() < 0
        assert abs(f_u[:nu].sum()) <= 1e-12 * abs(fz) and abs(f_u[nu:2 * nu].sum()) <= 1e-12 * abs(fz)
        cool = -mdot * EV["h_v"] * w_cp
        errs.append((abs(f_u[2 * nu:].sum() / fz - 1), abs(f_T.sum() / cool - 1)))
    assert errs[-1][0] < 1e-5 and errs[-1][1] < 1e-5
    assert errs[-1][0] < errs[0][0] and errs[-1][1] < errs[0][1]


def test_sine_heaviside_delta_converges_to_the_jump_of_H():
    """With eq. (heaviside), int delta = H(phi(0)) - H(phi(1)) in the limit; the 3-point rule on
    the composed profile converges to it."""
    errs = []
    for n in (8, 16, 32):     # fixed interface width, refined mesh
        dmu, dmp, phi, eps = flat_interface(n, eps=0.1)
        T = np.full(dmu.n_dofs, EV["t_boil"] + 1.0)
        p = params("tanasawa", heaviside="sine", eps=eps)
        _, f_p, _ = oi.interface_sources(dmu, dmp, phi, T, p)
        t = np.tanh(1.0 / (4.0 * eps))
        jump = co.heaviside_sine(np.array(t), eps) - co.heaviside_sine(np.array(-t), eps)
        errs.append(abs(f_p.sum() / (EV["tanasawa"] * (1 / TI["rho_l"] - 1 / TI["rho_g"]) * jump) - 1))
    assert errs[-1] < 1e-3 and errs[2] < errs[0]


def test_velocity_dirichlet_rows_are_zero_and_absolute_bound_dominates():
    dmu, dmp, phi, eps = flat_interface(6, dirichlet_faces=0b011111)
    x = dmu.dof_coords()
    T = syn.interface_temperature(*x.T)
    p = params("knight", eps=eps)
    f_u, f_p, f_T = oi.interface_sources(dmu, dmp, phi, T, p)
    b_u, b_p, b_T = oi.interface_sources(dmu, dmp, phi, T, p, absolute=True)
    assert np.all(f_u[np.tile(dmu.dirichlet, 3)] == 0.0)
    for f, b in ((f_u, b_u), (f_p, b_p), (f_T, b_T)):
        assert np.all(np.abs(f) <= b * (1 + 1e-14) + 1e-300)
