"""Pointwise coefficient laws (Section 2.3 and Section 4.3 of the paper).

Readings (stated once here, listed in the design notes):
* The default Heaviside is the tanh-regularised one implied by eq. (initial_phi):
  phi = tanh(d / 2 eps) gives H = (1 + phi) / 2 = 1 / (1 + exp(-d / eps)); the
  interpolated phi_h can overshoot [-1, 1], so H is clamped to [0, 1].
* The paper's own eq. (heaviside) is written in d(phi); d is recovered by inverting
  eq. (initial_phi): d = 2 eps atanh(phi), with phi clamped to +-(1 - 2^-52).
* k(T) = k0 (1 + 0.5 T / T_b) is the temperature law of the heat workloads (the paper
  keeps properties temperature independent; it is a workload input, not a paper law).
* Darcy damping acts in the dense phase only: K_eff = H_phi K(f_s(T)).  Eq. (darcy_damping_force)
  computes f_s from T everywhere, but the solid fraction is defined "in the dense part of the
  domain" (Section 3.1), and cold gas must not be frozen.
"""
import numpy as np


def heaviside_tanh(phi):
    """H = clamp((1 + phi) / 2, 0, 1)."""
    return np.clip(0.5 * (1.0 + phi), 0.0, 1.0)


def heaviside_sine(phi, eps):
    """Eq. (heaviside): 0 below -3 eps, 1 above 3 eps, else 1/2 + d/(6 eps) + sin(pi d/(3 eps))/(2 pi)."""
    lim = 1.0 - 2.0 ** -52
    d = 2.0 * eps * np.arctanh(np.clip(phi, -lim, lim))
    mid = 0.5 + d / (6.0 * eps) + np.sin(np.pi * d / (3.0 * eps)) / (2.0 * np.pi)
    return np.where(d <= -3.0 * eps, 0.0, np.where(d >= 3.0 * eps, 1.0, mid))


def arithmetic_mix(H, a_liquid, a_gas):
    """Eq. (muEff): a = H a_l + (1 - H) a_g (viscosity, conductivity, rho c_p)."""
    return H * a_liquid + (1.0 - H) * a_gas


def reciprocal_density(H, rho_liquid, rho_gas):
    """Eq. (rhoEff): 1 / rho = H / rho_l + (1 - H) / rho_g."""
    return 1.0 / (H / rho_liquid + (1.0 - H) / rho_gas)


def conductivity_of_temperature(T, k0, t_boil):
    """k(T) = k0 (1 + 0.5 T / T_b)."""
    return k0 * (1.0 + 0.5 * T / t_boil)


def laser_flux(x, y, power, radius, x0, y0, absorptivity):
    """Eq. (laser_gauss) on a flat top surface with the beam along -z, so that
    <-n . e_L> = 1 and the flux is the surface density 2 chi P / (pi r^2) exp(-2 rho^2 / r^2),
    rho the distance to the beam axis through (x0, y0)."""
    r2 = (x - x0) ** 2 + (y - y0) ** 2
    return 2.0 * absorptivity * power / (np.pi * radius ** 2) * np.exp(-2.0 * r2 / radius ** 2)


def laser_flux_parameter_derivatives(x, y, power, radius, x0, y0, absorptivity):
    """Closed-form derivatives of eq. (laser_gauss) w.r.t. (P, r, x0, y0):
    dq/dP = q/P, dq/dr = q (-2/r + 4 rho^2 / r^3), dq/dx0 = 4 q (x - x0)/r^2, dq/dy0 = 4 q (y - y0)/r^2."""
    q = laser_flux(x, y, power, radius, x0, y0, absorptivity)
    r2 = (x - x0) ** 2 + (y - y0) ** 2
    return np.stack([q / power,
                     q * (-2.0 / radius + 4.0 * r2 / radius ** 3),
                     4.0 * q * (x - x0) / radius ** 2,
                     4.0 * q * (y - y0) / radius ** 2])


def solid_fraction(T, t_solidus, t_liquidus):
    """Eq. (solid_fraction): 1 below T_s, 0 above T_l, linear (T_l - T)/(T_l - T_s) between."""
    return np.clip((t_liquidus - T) / (t_liquidus - t_solidus), 0.0, 1.0)


def heaviside_solid(fs):
    """Eq. (heaviside_sl): H_s = 3 f_s^2 - 2 f_s^3."""
    return 3.0 * fs * fs - 2.0 * fs * fs * fs


def three_phase_mix(H, Hs, a_solid, a_liquid, a_gas):
    """Eq. (solid_liquid_gas_property): H (H_s a_s + (1 - H_s) a_l) + (1 - H) a_g."""
    return H * (Hs * a_solid + (1.0 - Hs) * a_liquid) + (1.0 - H) * a_gas


def three_phase_density(H, Hs, rho_solid, rho_liquid, rho_gas):
    """Eq. (solid_liquid_gas_density): 1/rho = H / rho_sl + (1 - H) / rho_g, rho_sl = H_s rho_s + (1 - H_s) rho_l."""
    rho_sl = Hs * rho_solid + (1.0 - Hs) * rho_liquid
    return 1.0 / (H / rho_sl + (1.0 - H) / rho_gas)


def darcy_coefficient(fs, C, b):
    """Magnitude of eq. (darcy_damping_force)'s K: C f_s^2 / ((1 - f_s)^3 + b) (the force is -that u)."""
    return C * fs * fs / ((1.0 - fs) ** 3 + b)
