// Interface source terms of Section 2.4 as load vectors, fused in one pass over the cells of a
// uniform Oseen mesh: the smoothed delta function delta = ||grad H(phi_h)|| (eq. delta), its
// density- and heat-capacity-weighted forms, the evaporative mass flux (Knight's eq. mDotPSat with
// the Clausius-Clapeyron saturated pressure, or Tanasawa's eq. mDotTanasawa), and from them
//   f_p = int mdot (1/rho_l - 1/rho_g) delta psi          (evaporative dilation, eq. evaporDil)
//   f_T = int -mdot h_v delta_rhocp N                      (evaporative cooling, eq. vapor_heat_loss)
//   f_u = int (p_An delta_rho - mdot^2 (1/rho_g - 1/rho_l) delta) n_Gamma . v
//                                                          (hybrid recoil force, eq. hybrid_recoil_pressure)
// Every value is evaluated in fp64 at the 27 Gauss points of a cell from the nodal phi and T.
#include <cmath>

#include "interface.cuh"

namespace mf {

MF_DEFINE_TABLE_UPLOAD

UniformGeom uniform_geom(const mf_dofmap* m);

namespace {

struct SourceArgs {
  const double* phi;  // nodal level set on the velocity map
  const double* T;    // nodal temperature on the velocity map
  double *fu, *fp, *fT;
  int64_t nu;
  double rho_l, rho_g, rhocp_l, rhocp_g, eps;
  int heaviside;
  int knight;  // 1: Knight / Clausius-Clapeyron, 0: Tanasawa
  double p_amb, h_v, t_boil, tanasawa, gas;
  double c_rho, c_rhocp;
  double kappa, inv_t_boil, knight_coef;  // h_v M / R, 1 / T_v, 0.82 c_s p_amb sqrt(M / (2 pi R))
};

template <bool RECOIL>
__global__ void __launch_bounds__(128) k_interface_sources(SourceArgs A, UniformGeom ug) {
  int i, j, k;
  if (!brick_cell(ug, i, j, k)) return;
  const int64_t base = 2 * int64_t(i) + ug.sx * (2 * int64_t(j)) + ug.sy * (2 * int64_t(k));
  const uint32_t dmask = dirichlet_mask(ug, i, j, k);
  const int64_t px = ug.nx + 1, pxy = px * (ug.ny + 1);
  const int64_t pbase = i + px * (j + (ug.ny + 1) * int64_t(k));
  const double h = ug.h, ih = 1.0 / ug.h, h3 = h * h * h;
  double P[27], TT[27];
  gather_uniform<double>(A.phi, base, ug.sx, ug.sy, 0u, P);
  gather_uniform<double>(A.T, base, ug.sx, ug.sy, 0u, TT);
  to_qpoints<double>(P);
  to_qpoints<double>(TT);
  double Rp[8], R0[27], R1[27], R2[27];
#pragma unroll
  for (int n = 0; n < 8; ++n) Rp[n] = 0.0;
  const double drho = 1.0 / A.rho_l - 1.0 / A.rho_g;
#pragma unroll
  for (int qc = 0; qc < 3; ++qc)
#pragma unroll
    for (int qb = 0; qb < 3; ++qb)
#pragma unroll
      for (int qa = 0; qa < 3; ++qa) {
        const int q = qa + 3 * qb + 9 * qc;
        double gx, gy, gz;
        grad_at<double>(P, qa, qb, qc, gx, gy, gz);
        gx *= ih;
        gy *= ih;
        gz *= ih;
        const double g = sqrt(gx * gx + gy * gy + gz * gz);
        const double phi = P[q], T = TT[q];
        const double dl = delta_at(phi, g, A.heaviside, A.eps);
        const double H = heaviside<double>(phi, A.heaviside, A.eps);
        const double rhocp = H * A.rhocp_l + (1.0 - H) * A.rhocp_g;
        // Clausius-Clapeyron and eq. (anisimov) share the exponent kappa (1/T_v - 1/T), kappa =
        // h_v M / R: p_sat = p_amb e^x and p_An = 0.54 p_amb e^x (one exp per Gauss point)
        const double iT = 1.0 / T;
        const double ex = (A.knight || RECOIL) ? exp(A.kappa * (A.inv_t_boil - iT)) : 0.0;
        const double mdot = A.knight ? A.knight_coef * ex * sqrt(iT) : A.tanasawa * (T - A.t_boil);
        const double w = Tb<double>::W3(q) * h3;
        const double sp = w * mdot * drho * dl;
#pragma unroll
        for (int n = 0; n < 8; ++n) Rp[n] += Tb<double>::PW(q, n) * sp;
        TT[q] = w * (-mdot * A.h_v * dl * rhocp * rhocp * A.c_rhocp);  // T at q is consumed
        if constexpr (RECOIL) {
          const double rho = 1.0 / (H / A.rho_l + (1.0 - H) / A.rho_g);
          const double p_an = 0.54 * A.p_amb * ex;
          const double net = p_an * dl * rho * A.c_rho + mdot * mdot * drho * dl;
          const double s = g > 0.0 ? w * net / g : 0.0;
          R0[q] = s * gx;
          R1[q] = s * gy;
          R2[q] = s * gz;
        }
      }
  if (A.fT) {
    to_nodes<double>(TT);
    scatter_uniform<double>(A.fT, base, ug.sx, ug.sy, 0u, TT);
  }
  if (A.fp) {
#pragma unroll
    for (int n = 0; n < 8; ++n) atomicAdd(A.fp + pbase + (n & 1) + px * ((n >> 1) & 1) + pxy * (n >> 2), Rp[n]);
  }
  if constexpr (RECOIL) {
    to_nodes<double>(R0);
    scatter_uniform<double>(A.fu, base, ug.sx, ug.sy, dmask, R0);
    to_nodes<double>(R1);
    scatter_uniform<double>(A.fu + A.nu, base, ug.sx, ug.sy, dmask, R1);
    to_nodes<double>(R2);
    scatter_uniform<double>(A.fu + 2 * A.nu, base, ug.sx, ug.sy, dmask, R2);
  }
}

}  // namespace

mf_status launch_interface_sources(mf_ctx* ctx, const mf_dofmap* mu, const mf_dofmap* mp, const mf_op_params& p,
                                   const double* phi, const mf_evaporation& ev, const double* T, double* fu,
                                   double* fp, double* fT) {
  MF_CUDA_TRY(upload_tables_here());
  UniformGeom ug = uniform_geom(mu);
  SourceArgs a{};
  a.phi = phi;
  a.T = T;
  a.fu = fu;
  a.fp = fp;
  a.fT = fT;
  a.nu = mu->n_dofs;
  a.rho_l = p.rho_l;
  a.rho_g = p.rho_g;
  a.rhocp_l = ev.rhocp_liquid;
  a.rhocp_g = ev.rhocp_gas;
  a.eps = p.eps;
  a.heaviside = p.heaviside;
  a.knight = ev.mass_flux == MF_MASS_FLUX_KNIGHT ? 1 : 0;
  a.p_amb = ev.p_ambient;
  a.h_v = ev.latent_heat;
  a.t_boil = ev.t_boil;
  a.tanasawa = ev.tanasawa_coef;
  a.gas = ev.gas_constant > 0 ? ev.gas_constant : 8.314;
  a.c_rho = (p.rho_g - p.rho_l) / (p.rho_l * p.rho_g * std::log(p.rho_g / p.rho_l));
  a.kappa = ev.latent_heat * ev.molar_mass / a.gas;
  a.inv_t_boil = ev.t_boil > 0 ? 1.0 / ev.t_boil : 0.0;
  a.knight_coef = 0.82 * ev.sticking * ev.p_ambient * std::sqrt(ev.molar_mass / (2.0 * 3.141592653589793 * a.gas));
  a.c_rhocp = 3.0 / (ev.rhocp_gas * ev.rhocp_gas + ev.rhocp_liquid * ev.rhocp_gas + ev.rhocp_liquid * ev.rhocp_liquid);
  if (fu) MF_CUDA_TRY(cudaMemsetAsync(fu, 0, sizeof(double) * 3 * mu->n_dofs, ctx->stream));
  if (fp) MF_CUDA_TRY(cudaMemsetAsync(fp, 0, sizeof(double) * mp->n_dofs, ctx->stream));
  if (fT) MF_CUDA_TRY(cudaMemsetAsync(fT, 0, sizeof(double) * mu->n_dofs, ctx->stream));
  const int nb = brick_blocks(ug.nx, ug.ny, ug.nz);
  if (fu)
    k_interface_sources<true><<<nb, 128, 0, ctx->stream>>>(a, ug);
  else
    k_interface_sources<false><<<nb, 128, 0, ctx->stream>>>(a, ug);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

}  // namespace mf
