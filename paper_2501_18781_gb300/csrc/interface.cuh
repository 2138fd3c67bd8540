// Pointwise interface quantities of Section 2.4 shared by the source-term and time-step kernels:
// the smoothed delta function and the evaporative mass flux, evaluated in fp64.
#pragma once

#include <cmath>

#include "scalar_local.cuh"

namespace mf {

// eq. (delta) at a Gauss point from phi_h and its physical gradient
__device__ __forceinline__ double delta_at(double phi, double g, int kind, double eps) {
  if (kind == 0) {
    const double H = 0.5 * (1.0 + phi);
    return (H > 0.0 && H < 1.0) ? 0.5 * g : 0.0;
  }
  const double lim = 1.0 - 2.220446049250313e-16;
  const double p = phi > lim ? lim : (phi < -lim ? -lim : phi);
  const double d = 2.0 * eps * atanh(p);
  if (!(fabs(d) < 3.0 * eps)) return 0.0;
  const double pi = 3.141592653589793;
  return (1.0 + cos(pi * d / (3.0 * eps))) / (6.0 * eps) * 2.0 * eps * g / (1.0 - p * p);
}

// Evaporative mass flux mdot(T): Knight's eq. (mDotPSat) with the Clausius-Clapeyron saturated
// pressure, mdot = 0.82 c_s p_amb e^{kappa (1/T_v - 1/T)} sqrt(M / (2 pi R T)), kappa = h_v M / R, or
// Tanasawa's eq. (mDotTanasawa), mdot = h_e (T - T_v).
struct MassFlux {
  int knight;
  double knight_coef;  // 0.82 c_s p_amb sqrt(M / (2 pi R))
  double kappa, inv_t_boil, tanasawa, t_boil;
};

inline MassFlux make_mass_flux(const mf_evaporation& ev) {
  MassFlux m{};
  const double gas = ev.gas_constant > 0 ? ev.gas_constant : 8.314;
  m.knight = ev.mass_flux == MF_MASS_FLUX_KNIGHT ? 1 : 0;
  m.knight_coef = 0.82 * ev.sticking * ev.p_ambient * std::sqrt(ev.molar_mass / (2.0 * 3.141592653589793 * gas));
  m.kappa = ev.latent_heat * ev.molar_mass / gas;
  m.inv_t_boil = ev.t_boil > 0 ? 1.0 / ev.t_boil : 0.0;
  m.tanasawa = ev.tanasawa_coef;
  m.t_boil = ev.t_boil;
  return m;
}

__device__ __forceinline__ double mass_flux_at(const MassFlux& m, double T) {
  if (m.knight) {
    const double iT = 1.0 / T;
    return m.knight_coef * exp(m.kappa * (m.inv_t_boil - iT)) * sqrt(iT);
  }
  return m.tanasawa * (T - m.t_boil);
}

}  // namespace mf
