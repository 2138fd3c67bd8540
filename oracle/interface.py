"""Interface source terms as load vectors (test infrastructure: only tests, smoke() and the
bench's CPU leg use this package).

Section 2.4 of the paper couples the phases through regularised interface terms built from the
smoothed delta function delta = ||grad H_phi(phi)|| (eq. delta):
  * evaporative dilation rate  mdot (1/rho_l - 1/rho_g) delta           -> continuity, eq. (evaporDil)
  * evaporative cooling        -mdot h_v delta_rhocp                     -> energy, eq. (vapor_heat_loss)
  * hybrid recoil force        (p_An(T) delta_rho - mdot^2 (1/rho_g - 1/rho_l) delta) n_Gamma
                                                                         -> momentum, eqs. (anisimov_regularized),
                                                                            (recoilPressureEvaporDil), (hybrid_recoil_pressure)
with delta_rho = delta rho(phi) c_rho (Section 2.4) and the evaporative mass flux of Knight,
mdot = 0.82 c_s p_sat(T) sqrt(M / (2 pi R T)) (eq. mDotPSat), p_sat from Clausius-Clapeyron
(p_sat = p_amb exp(h_v M / (R T_v) (1 - T_v / T)), Appendix on the recoil pressure), or
Tanasawa's mdot = h_e (T - T_v) (eq. mDotTanasawa).  p_An(T) = 0.54 p_amb exp(-h_v M / R
(1/T - 1/T_v)) is eq. (anisimov).

Readings (listed in the design notes):
* delta_rhocp.  As printed, delta_rhocp = delta (rho c_p)(phi) c_rhocp with c_rhocp =
  3 / ((rho c_p)_g^2 + (rho c_p)_l (rho c_p)_g + (rho c_p)_l^2) has units of 1/(m rho c_p), which
  does not make eq. (laser_gauss) a volumetric heat source, and c_rhocp is exactly
  1 / int_0^1 (rho c_p)(H)^2 dH for the linear (rho c_p)(H).  Read: delta_rhocp = delta
  (rho c_p)(phi)^2 c_rhocp, a weight of unit integral across the interface (like delta and
  delta_rho).
* The temperature in mdot is the finite element interpolant T_h at the Gauss point (the
  paper evaluates it at the interface projection with its extension algorithm, which is out
  of scope).
* n_Gamma = grad phi_h / ||grad phi_h|| (the paper filters phi first; n = 0 where ||grad phi_h||
  vanishes).
* The loads are full-quadrature integrals f_i = sum_q w_q |J| s(x_q) N_i(x_q) over every cell, with
  every basis function evaluated directly; velocity Dirichlet rows of f_u are zero, f_p and f_T are
  natural load vectors (no Dirichlet rows).
"""
import numpy as np

from .basis import tensor_tables
from . import coeffs as co
from .assemble import field_at_qpoints

R_GAS = 8.314  # J/(mol K), the paper's molar gas constant


def saturated_vapour_pressure(T, p_amb, h_v, molar_mass, t_boil, gas_constant=R_GAS):
    """Clausius-Clapeyron: p_sat(T) = p_amb exp(h_v M / (R T_v) (1 - T_v / T))."""
    return p_amb * np.exp(h_v * molar_mass / (gas_constant * t_boil) * (1.0 - t_boil / T))


def mass_flux_knight(T, p_amb, h_v, molar_mass, t_boil, sticking=1.0, gas_constant=R_GAS):
    """Eq. (mDotPSat): mdot = 0.82 c_s p_sat(T) sqrt(M / (2 pi R T))."""
    ps = saturated_vapour_pressure(T, p_amb, h_v, molar_mass, t_boil, gas_constant)
    return 0.82 * sticking * ps * np.sqrt(molar_mass / (2.0 * np.pi * gas_constant * T))


def mass_flux_tanasawa(T, coefficient, t_boil):
    """Eq. (mDotTanasawa): mdot = h_e (T - T_v)."""
    return coefficient * (T - t_boil)


def recoil_anisimov(T, p_amb, h_v, molar_mass, t_boil, gas_constant=R_GAS):
    """Eq. (anisimov): p_An(T) = 0.54 p_amb exp(-h_v M / R (1/T - 1/T_v))."""
    return 0.54 * p_amb * np.exp(-h_v * molar_mass / gas_constant * (1.0 / T - 1.0 / t_boil))


def delta_smoothed(phi, grad_phi, heaviside="tanh", eps=None):
    """Eq. (delta): ||grad H_phi(phi_h)|| at points with values phi and gradients grad_phi (..., 3).
    tanh reading: H = clamp((1 + phi)/2), so delta = ||grad phi||/2 where 0 < H < 1, else 0.
    Eq. (heaviside): H(d) with d = 2 eps atanh(phi), dH/dd = (1 + cos(pi d / (3 eps))) / (6 eps)
    on |d| < 3 eps, grad d = 2 eps grad phi / (1 - phi^2)."""
    g = np.sqrt(np.sum(grad_phi ** 2, axis=-1))
    if heaviside == "tanh":
        H = 0.5 * (1.0 + phi)
        return np.where((H > 0.0) & (H < 1.0), 0.5 * g, 0.0)
    lim = 1.0 - 2.0 ** -52
    p = np.clip(phi, -lim, lim)
    d = 2.0 * eps * np.arctanh(p)
    dH = (1.0 + np.cos(np.pi * d / (3.0 * eps))) / (6.0 * eps)
    inside = np.abs(d) < 3.0 * eps
    return np.where(inside, dH * 2.0 * eps * g / (1.0 - p * p), 0.0)


def c_rho(rho_l, rho_g):
    """Normalisation of delta_rho (Section 2.4): (rho_g - rho_l) / (rho_l rho_g ln(rho_g / rho_l))."""
    return (rho_g - rho_l) / (rho_l * rho_g * np.log(rho_g / rho_l))


def c_rhocp(rhocp_l, rhocp_g):
    """Eq. (deltaRhoCp)'s constant 3 / ((rho c_p)_g^2 + (rho c_p)_l (rho c_p)_g + (rho c_p)_l^2)."""
    return 3.0 / (rhocp_g ** 2 + rhocp_l * rhocp_g + rhocp_l ** 2)


def source_densities(phi, grad_phi, T, p):
    """Pointwise densities (s_u (..., 3), s_p, s_T) of the three interface terms; p is a dict with
    rho_l, rho_g, rhocp_l, rhocp_g, heaviside, eps, model ('knight' | 'tanasawa'), p_amb, h_v,
    molar_mass, t_boil, sticking, tanasawa, recoil (bool)."""
    dl = delta_smoothed(phi, grad_phi, p["heaviside"], p["eps"])
    H = co.heaviside_tanh(phi) if p["heaviside"] == "tanh" else co.heaviside_sine(phi, p["eps"])
    rho = co.reciprocal_density(H, p["rho_l"], p["rho_g"])
    rhocp = co.arithmetic_mix(H, p["rhocp_l"], p["rhocp_g"])
    d_rho = dl * rho * c_rho(p["rho_l"], p["rho_g"])
    d_rhocp = dl * rhocp * rhocp * c_rhocp(p["rhocp_l"], p["rhocp_g"])
    if p["model"] == "knight":
        mdot = mass_flux_knight(T, p["p_amb"], p["h_v"], p["molar_mass"], p["t_boil"], p["sticking"])
    else:
        mdot = mass_flux_tanasawa(T, p["tanasawa"], p["t_boil"])
    s_p = mdot * (1.0 / p["rho_l"] - 1.0 / p["rho_g"]) * dl
    s_T = -mdot * p["h_v"] * d_rhocp
    g = np.sqrt(np.sum(grad_phi ** 2, axis=-1))
    n = np.where(g[..., None] > 0.0, grad_phi / np.where(g > 0.0, g, 1.0)[..., None], 0.0)
    if p["recoil"]:
        p_an = recoil_anisimov(T, p["p_amb"], p["h_v"], p["molar_mass"], p["t_boil"])
        net = p_an * d_rho - mdot * mdot * (1.0 / p["rho_g"] - 1.0 / p["rho_l"]) * dl
    else:
        net = np.zeros_like(dl)
    return net[..., None] * n, s_p, s_T


def interface_sources(dmu, dmp, phi, T, p, absolute=False):
    """Load vectors (f_u of length 3 n_u, f_p of n_p, f_T of n_u) of the densities above, by full
    quadrature with directly evaluated basis functions.  With ``absolute`` the integrands are
    replaced by their absolute values (|s| |N_i|): the componentwise scale for parity checks."""
    N, _, w = tensor_tables(2, 3)
    P, _, _ = tensor_tables(1, 3)
    ph, gph = field_at_qpoints(dmu, phi)
    Tq, _ = field_at_qpoints(dmu, T)
    s_u, s_p, s_T = source_densities(ph, gph, Tq, p)
    jw = w[None, :] * dmu.cell_h[:, None] ** 3
    Nn, Pn = (np.abs(N), np.abs(P)) if absolute else (N, P)
    if absolute:
        s_u, s_p, s_T = np.abs(s_u), np.abs(s_p), np.abs(s_T)
    M = dmu.points.shape[0]
    f_T = np.bincount(dmu.cell_points.ravel(), weights=np.einsum("cq,qi->ci", jw * s_T, Nn).ravel(), minlength=M)
    f_T = (np.abs(dmu.C.T) if absolute else dmu.C.T) @ f_T
    f_u = []
    for c in range(3):
        fc = np.bincount(dmu.cell_points.ravel(), weights=np.einsum("cq,qi->ci", jw * s_u[..., c], Nn).ravel(),
                         minlength=M)
        fc = (np.abs(dmu.C.T) if absolute else dmu.C.T) @ fc
        fc[dmu.dirichlet] = 0.0
        f_u.append(fc)
    Mp = dmp.points.shape[0]
    f_p = np.bincount(dmp.cell_points.ravel(), weights=np.einsum("cq,qi->ci", jw * s_p, Pn).ravel(), minlength=Mp)
    f_p = (np.abs(dmp.C.T) if absolute else dmp.C.T) @ f_p
    return np.concatenate(f_u), f_p, f_T
