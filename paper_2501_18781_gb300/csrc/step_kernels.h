// Launchers of the melt-pool time-step kernels (step.cu), used by the step driver (step.cpp).
#pragma once

#include "ops.h"

namespace mf {

// eq. (laser_gauss): q0 = 2 chi P / (pi r^2), beam axis through focus along the unit dir
struct StepLaser {
  double q0, radius;
  double focus[3], dir[3];
  double lo[3];  // box origin (Gauss-point coordinates)
};

// eq. (surface_tension) with the residual coefficient alpha_res, and gravity
struct StepForces {
  double alpha0, alpha1, t_alpha, alpha_res;
  double g[3];
  double rho_l, rho_g, c_rho;
  int hv;
  double eps;
};

// out = 2 x - xp
mf_status launch_extrapolate(mf_ctx* ctx, int64_t n, const double* x, const double* xp, double* out);
// u_G = u_h + mdot(T_h) / rho(phi_h) n_G(phi_h) at the Gauss points, out[cell][27][3]
mf_status launch_transport_velocity(mf_ctx* ctx, const mf_dofmap* m, const double* u, const double* T,
                                    const double* phi, const mf_evaporation& ev, double rho_l, double rho_g, int hv,
                                    double eps, double* out);
// two-phase k and rho_cp at the Gauss points, [cell][27]
mf_status launch_heat_coefficients(mf_ctx* ctx, const mf_dofmap* m, const double* phi, int hv, double eps,
                                   double rhocp_l, double rhocp_g, double k_l, double k_g, double* kq, double* rhocp);
// dst += int c u_h N_i, c = c0 or c0 tab[q qs + cell cs]; mask: skip the map's Dirichlet rows
mf_status launch_mass_load(mf_ctx* ctx, const mf_dofmap* m, const double* src, const double* tab, int64_t qs,
                           int64_t cs, double c0, bool mask, double* dst);
// dst += int (1 - psi_h^2)/2 n(phi_h) . grad N_i
mf_status launch_compressive_flux(mf_ctx* ctx, const mf_dofmap* m, const double* psi, const double* phi,
                                  double* dst);
// dst += int q_L N_i
mf_status launch_laser_interface(mf_ctx* ctx, const mf_dofmap* m, const StepLaser& L, const double* phi, int hv,
                                 double eps, double rhocp_l, double rhocp_g, double* dst);
// dst_u (3 blocks) += surface tension and gravity loads, Dirichlet rows skipped
mf_status launch_flow_forces(mf_ctx* ctx, const mf_dofmap* mu, const StepForces& F, const double* phi,
                             const double* T, const double* rho_tab, double* dst);

}  // namespace mf
