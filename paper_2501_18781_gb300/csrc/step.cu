// Kernels of one melt-pool time step (Algorithm algo:meltpooldg) on a uniform Q2 mesh: the
// predictors, the Gauss-point transport velocity of variant 1 (eq. transport_vel_local_continuous),
// the two-phase heat coefficients (eq. muEff), and the load vectors of the level-set, heat and flow
// systems (mass-weighted previous step, Olsson's compressive flux, the interface laser flux of eq.
// laser_gauss, surface tension of eq. surface_tension with gravity).  One thread owns one cell, as
// in the operator kernels; every value is evaluated in fp64 from the nodal fields.
#include "interface.cuh"
#include "step_kernels.h"

namespace mf {

MF_DEFINE_TABLE_UPLOAD

UniformGeom uniform_geom(const mf_dofmap* m);

namespace {

__global__ void k_extrapolate(int64_t n, const double* __restrict__ x, const double* __restrict__ xp,
                              double* __restrict__ out) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = 2.0 * x[i] - xp[i];
}

__device__ __forceinline__ int64_t cell_base(const UniformGeom& ug, int i, int j, int k) {
  return 2 * int64_t(i) + ug.sx * (2 * int64_t(j)) + ug.sy * (2 * int64_t(k));
}

__device__ __forceinline__ int64_t cell_index(const UniformGeom& ug, int i, int j, int k) {
  return i + int64_t(ug.nx) * (j + int64_t(ug.ny) * k);
}

// Unit normal from a reference gradient (0 where |g| < 1e-12, i.e. |grad phi_h| < 1e-12 / h);
// returns |g|.
__device__ __forceinline__ double unit_normal(double gx, double gy, double gz, double& nx, double& ny, double& nz) {
  const double nn = sqrt(gx * gx + gy * gy + gz * gz);
  const double inv = nn < 1e-12 ? 0.0 : 1.0 / nn;
  nx = gx * inv;
  ny = gy * inv;
  nz = gz * inv;
  return nn;
}

// Reference Hessian (xx, yy, zz, xy, xz, yz) at Gauss point (qa, qb, qc) of the collocation values
// U of a Q2 function.  Along every Gauss line the function is quadratic, so its second derivative
// is the constant 2 f[g0, g1, g2] = (u0 - 2 u1 + u2) / r^2 (points 1/2 - r, 1/2, 1/2 + r); the mixed
// terms are two collocation derivatives.
__device__ __forceinline__ void hessian_at(const double* U, int qa, int qb, int qc, double* H) {
  const double r = cG64[1] - cG64[0];
  const double i2 = 1.0 / (r * r);
  const int q = qa + 3 * qb + 9 * qc;
  const int bx = q - qa, by = q - 3 * qb, bz = q - 9 * qc;
  H[0] = (U[bx] - 2.0 * U[bx + 1] + U[bx + 2]) * i2;
  H[1] = (U[by] - 2.0 * U[by + 3] + U[by + 6]) * i2;
  H[2] = (U[bz] - 2.0 * U[bz + 9] + U[bz + 18]) * i2;
  double t[3];
  for (int a = 0; a < 3; ++a) t[a] = dline<double>(qb, U[a + 9 * qc], U[a + 3 + 9 * qc], U[a + 6 + 9 * qc]);
  H[3] = dline<double>(qa, t[0], t[1], t[2]);
  for (int a = 0; a < 3; ++a) t[a] = dline<double>(qc, U[a + 3 * qb], U[a + 3 * qb + 9], U[a + 3 * qb + 18]);
  H[4] = dline<double>(qa, t[0], t[1], t[2]);
  for (int b = 0; b < 3; ++b) t[b] = dline<double>(qc, U[qa + 3 * b], U[qa + 3 * b + 9], U[qa + 3 * b + 18]);
  H[5] = dline<double>(qb, t[0], t[1], t[2]);
}

// u_G = u_h + mdot(T_h) / rho(phi_h) n_G(phi_h) at the Gauss points, out[cell][27][3]
__global__ void __launch_bounds__(128) k_transport_velocity(UniformGeom ug, const double* u, int64_t nu,
                                                            const double* T, const double* phi, MassFlux mflux,
                                                            double rho_l, double rho_g, int hv, double eps,
                                                            double* out) {
  int i, j, k;
  if (!brick_cell(ug, i, j, k)) return;
  const int64_t base = cell_base(ug, i, j, k), cell = cell_index(ug, i, j, k);
  double* o = out + cell * 81;
  double U[27];
  for (int c = 0; c < 3; ++c) {
    gather_uniform<double>(u + c * nu, base, ug.sx, ug.sy, 0u, U);
    to_qpoints<double>(U);
    for (int q = 0; q < 27; ++q) o[3 * q + c] = U[q];
  }
  double P[27];
  gather_uniform<double>(phi, base, ug.sx, ug.sy, 0u, P);
  gather_uniform<double>(T, base, ug.sx, ug.sy, 0u, U);
  to_qpoints<double>(P);
  to_qpoints<double>(U);
#pragma unroll 1
  for (int q = 0; q < 27; ++q) {
    const int qa = q % 3, qb = (q / 3) % 3, qc = q / 9;
    double gx, gy, gz, nx, ny, nz;
    grad_at<double>(P, qa, qb, qc, gx, gy, gz);
    unit_normal(gx, gy, gz, nx, ny, nz);
    const double H = heaviside<double>(P[q], hv, eps);
    const double s = mass_flux_at(mflux, U[q]) * (H / rho_l + (1.0 - H) / rho_g);  // mdot / rho
    o[3 * q] += s * nx;
    o[3 * q + 1] += s * ny;
    o[3 * q + 2] += s * nz;
  }
}

// k = H k_l + (1 - H) k_g and rho_cp = H rho_cp_l + (1 - H) rho_cp_g at the Gauss points, [cell][27]
__global__ void __launch_bounds__(128) k_heat_coefficients(UniformGeom ug, const double* phi, int hv, double eps,
                                                           double rhocp_l, double rhocp_g, double k_l, double k_g,
                                                           double* kq, double* rhocp) {
  int i, j, k;
  if (!brick_cell(ug, i, j, k)) return;
  const int64_t base = cell_base(ug, i, j, k), cell = cell_index(ug, i, j, k);
  double P[27];
  gather_uniform<double>(phi, base, ug.sx, ug.sy, 0u, P);
  to_qpoints<double>(P);
  for (int q = 0; q < 27; ++q) {
    const double H = heaviside<double>(P[q], hv, eps);
    kq[cell * 27 + q] = H * k_l + (1.0 - H) * k_g;
    rhocp[cell * 27 + q] = H * rhocp_l + (1.0 - H) * rhocp_g;
  }
}

// dst += int c u_h N_i with c = c0 (tab NULL) or c0 tab[q qs + cell cs]; Dirichlet rows of the map
// are skipped when mask is set.
__global__ void __launch_bounds__(128) k_mass_load(UniformGeom ug, const double* src, const double* tab, int64_t qs,
                                                   int64_t cs, double c0, int mask, double* dst) {
  int i, j, k;
  if (!brick_cell(ug, i, j, k)) return;
  const int64_t base = cell_base(ug, i, j, k), cell = cell_index(ug, i, j, k);
  const double h3 = ug.h * ug.h * ug.h;
  double U[27];
  gather_uniform<double>(src, base, ug.sx, ug.sy, 0u, U);
  to_qpoints<double>(U);
  for (int q = 0; q < 27; ++q) {
    const double c = tab ? c0 * __ldg(tab + q * qs + cell * cs) : c0;
    U[q] = Tb<double>::W3(q) * h3 * (c * U[q]);
  }
  to_nodes<double>(U);
  scatter_uniform<double>(dst, base, ug.sx, ug.sy, mask ? dirichlet_mask(ug, i, j, k) : 0u, U);
}

// dst += F(psi), F_i = int (1 - psi_h^2)/2 n . grad N_i with n the unit normal of phi_h
__global__ void __launch_bounds__(128) k_compressive_flux(UniformGeom ug, const double* psi, const double* phi,
                                                          double* dst) {
  int i, j, k;
  if (!brick_cell(ug, i, j, k)) return;
  const int64_t base = cell_base(ug, i, j, k);
  const double h2 = ug.h * ug.h;
  double S[27], P[27], R[27];
  gather_uniform<double>(psi, base, ug.sx, ug.sy, 0u, S);
  gather_uniform<double>(phi, base, ug.sx, ug.sy, 0u, P);
  to_qpoints<double>(S);
  to_qpoints<double>(P);
  for (int q = 0; q < 27; ++q) R[q] = 0.0;
#pragma unroll
  for (int qc = 0; qc < 3; ++qc)
#pragma unroll
    for (int qb = 0; qb < 3; ++qb)
#pragma unroll
      for (int qa = 0; qa < 3; ++qa) {
        const int q = qa + 3 * qb + 9 * qc;
        double gx, gy, gz, nx, ny, nz;
        grad_at<double>(P, qa, qb, qc, gx, gy, gz);
        unit_normal(gx, gy, gz, nx, ny, nz);
        const double v = Tb<double>::W3(q) * h2 * (0.5 * (1.0 - S[q] * S[q]));
        add_grad_test<double>(R, qa, qb, qc, v * nx, v * ny, v * nz);
      }
  to_nodes<double>(R);
  scatter_uniform<double>(dst, base, ug.sx, ug.sy, 0u, R);
}

// dst += int q_L N_i, q_L of eq. (laser_gauss) with <n_G . e_L>, d_L the distance to the beam
// axis and delta_rhocp = delta (rho c_p)(phi)^2 c_rhocp
__global__ void __launch_bounds__(128) k_laser_load(UniformGeom ug, StepLaser L, const double* phi, int hv,
                                                    double eps, double rhocp_l, double rhocp_g, double c_rhocp,
                                                    double* dst) {
  int i, j, k;
  if (!brick_cell(ug, i, j, k)) return;
  const int64_t base = cell_base(ug, i, j, k);
  const double h = ug.h, h3 = h * h * h;
  double P[27], R[27];
  gather_uniform<double>(phi, base, ug.sx, ug.sy, 0u, P);
  to_qpoints<double>(P);
#pragma unroll 1
  for (int q = 0; q < 27; ++q) {
    const int qa = q % 3, qb = (q / 3) % 3, qc = q / 9;
    double gx, gy, gz, nx, ny, nz;
    grad_at<double>(P, qa, qb, qc, gx, gy, gz);
    const double g = unit_normal(gx, gy, gz, nx, ny, nz) / h;
    const double cos_in = nx * L.dir[0] + ny * L.dir[1] + nz * L.dir[2];
    double f = 0.0;
    if (cos_in > 0.0) {
      const double dl = delta_at(P[q], g, hv, eps);
      const double H = heaviside<double>(P[q], hv, eps);
      const double rc = H * rhocp_l + (1.0 - H) * rhocp_g;
      const double x[3] = {L.lo[0] + h * (i + cG64[qa]), L.lo[1] + h * (j + cG64[qb]), L.lo[2] + h * (k + cG64[qc])};
      double r[3], along = 0.0;
      for (int d = 0; d < 3; ++d) {
        r[d] = x[d] - L.focus[d];
        along += r[d] * L.dir[d];
      }
      double d2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        const double p = r[d] - along * L.dir[d];  // off the axis
        d2 += p * p;
      }
      f = L.q0 * cos_in * exp(-2.0 * d2 / (L.radius * L.radius)) * (dl * rc * rc * c_rhocp);
    }
    R[q] = Tb<double>::W3(q) * h3 * f;
  }
  to_nodes<double>(R);
  scatter_uniform<double>(dst, base, ug.sx, ug.sy, 0u, R);
}

// dst_u += int ((alpha kappa n + (I - n n) grad alpha) delta_rho + rho g) . v (eq. surface_tension
// and gravity), kappa = -div n from the Hessian of phi_h, rho from the flow operator's table
// (rho_tab[q][cell]), delta_rho with the two-phase rho of eq. (rhoEff); Dirichlet rows skipped.
__global__ void __launch_bounds__(128) k_flow_forces(UniformGeom ug, StepForces F, const double* phi,
                                                     const double* T, const double* rho_tab, int64_t ncells,
                                                     int64_t nu, double* dst) {
  int i, j, k;
  if (!brick_cell(ug, i, j, k)) return;
  const int64_t base = cell_base(ug, i, j, k), cell = cell_index(ug, i, j, k);
  const uint32_t dmask = dirichlet_mask(ug, i, j, k);
  const double h = ug.h, h3 = h * h * h;
  double P[27], TT[27], R0[27], R1[27], R2[27];
  gather_uniform<double>(phi, base, ug.sx, ug.sy, 0u, P);
  gather_uniform<double>(T, base, ug.sx, ug.sy, 0u, TT);
  to_qpoints<double>(P);
  to_qpoints<double>(TT);
#pragma unroll 1
  for (int q = 0; q < 27; ++q) {
    const int qa = q % 3, qb = (q / 3) % 3, qc = q / 9;
    double gx, gy, gz, n[3];
    grad_at<double>(P, qa, qb, qc, gx, gy, gz);
    const double nn = unit_normal(gx, gy, gz, n[0], n[1], n[2]);
    double Hs[6];
    hessian_at(P, qa, qb, qc, Hs);
    // kappa = -(tr Hess - n^T Hess n) / |grad phi| in physical units (Hess / h^2, |grad| = nn / h)
    const double nHn = n[0] * n[0] * Hs[0] + n[1] * n[1] * Hs[1] + n[2] * n[2] * Hs[2] +
                       2.0 * (n[0] * n[1] * Hs[3] + n[0] * n[2] * Hs[4] + n[1] * n[2] * Hs[5]);
    const double kappa = nn < 1e-12 ? 0.0 : -((Hs[0] + Hs[1] + Hs[2]) - nHn) / (h * nn);
    const double H = heaviside<double>(P[q], F.hv, F.eps);
    const double drho = delta_at(P[q], nn / h, F.hv, F.eps) / (H / F.rho_l + (1.0 - H) / F.rho_g) * F.c_rho;
    double tx, ty, tz;
    grad_at<double>(TT, qa, qb, qc, tx, ty, tz);
    const double lin = F.alpha0 - F.alpha1 * (TT[q] - F.t_alpha);
    const bool active = lin > F.alpha_res;
    const double alpha = active ? lin : F.alpha_res;
    const double ga[3] = {active ? -F.alpha1 * tx / h : 0.0, active ? -F.alpha1 * ty / h : 0.0,
                          active ? -F.alpha1 * tz / h : 0.0};
    const double ng = n[0] * ga[0] + n[1] * ga[1] + n[2] * ga[2];
    const double rho = __ldg(rho_tab + q * ncells + cell);
    const double w = Tb<double>::W3(q) * h3;
    double f[3];
    for (int d = 0; d < 3; ++d) f[d] = (alpha * kappa * n[d] + (ga[d] - ng * n[d])) * drho + rho * F.g[d];
    R0[q] = w * f[0];
    R1[q] = w * f[1];
    R2[q] = w * f[2];
  }
  to_nodes<double>(R0);
  scatter_uniform<double>(dst, base, ug.sx, ug.sy, dmask, R0);
  to_nodes<double>(R1);
  scatter_uniform<double>(dst + nu, base, ug.sx, ug.sy, dmask, R1);
  to_nodes<double>(R2);
  scatter_uniform<double>(dst + 2 * nu, base, ug.sx, ug.sy, dmask, R2);
}

int grid_for(int64_t n) { return int(std::min<int64_t>((n + 255) / 256, 152 * 16)); }

}  // namespace

#define MF_STEP_LAUNCH_END  \
  ctx->launches++;          \
  MF_CUDA_TRY(cudaGetLastError()); \
  return MF_OK

mf_status launch_extrapolate(mf_ctx* ctx, int64_t n, const double* x, const double* xp, double* out) {
  if (n == 0) return MF_OK;
  k_extrapolate<<<grid_for(n), 256, 0, ctx->stream>>>(n, x, xp, out);
  MF_STEP_LAUNCH_END;
}

mf_status launch_transport_velocity(mf_ctx* ctx, const mf_dofmap* m, const double* u, const double* T,
                                    const double* phi, const mf_evaporation& ev, double rho_l, double rho_g, int hv,
                                    double eps, double* out) {
  MF_CUDA_TRY(upload_tables_here());
  UniformGeom ug = uniform_geom(m);
  k_transport_velocity<<<brick_blocks(ug.nx, ug.ny, ug.nz), 128, 0, ctx->stream>>>(
      ug, u, m->n_dofs, T, phi, make_mass_flux(ev), rho_l, rho_g, hv, eps, out);
  MF_STEP_LAUNCH_END;
}

mf_status launch_heat_coefficients(mf_ctx* ctx, const mf_dofmap* m, const double* phi, int hv, double eps,
                                   double rhocp_l, double rhocp_g, double k_l, double k_g, double* kq, double* rhocp) {
  MF_CUDA_TRY(upload_tables_here());
  UniformGeom ug = uniform_geom(m);
  k_heat_coefficients<<<brick_blocks(ug.nx, ug.ny, ug.nz), 128, 0, ctx->stream>>>(ug, phi, hv, eps, rhocp_l, rhocp_g,
                                                                                  k_l, k_g, kq, rhocp);
  MF_STEP_LAUNCH_END;
}

mf_status launch_mass_load(mf_ctx* ctx, const mf_dofmap* m, const double* src, const double* tab, int64_t qs,
                           int64_t cs, double c0, bool mask, double* dst) {
  MF_CUDA_TRY(upload_tables_here());
  UniformGeom ug = uniform_geom(m);
  k_mass_load<<<brick_blocks(ug.nx, ug.ny, ug.nz), 128, 0, ctx->stream>>>(ug, src, tab, qs, cs, c0, mask ? 1 : 0,
                                                                          dst);
  MF_STEP_LAUNCH_END;
}

mf_status launch_compressive_flux(mf_ctx* ctx, const mf_dofmap* m, const double* psi, const double* phi,
                                  double* dst) {
  MF_CUDA_TRY(upload_tables_here());
  UniformGeom ug = uniform_geom(m);
  k_compressive_flux<<<brick_blocks(ug.nx, ug.ny, ug.nz), 128, 0, ctx->stream>>>(ug, psi, phi, dst);
  MF_STEP_LAUNCH_END;
}

mf_status launch_laser_interface(mf_ctx* ctx, const mf_dofmap* m, const StepLaser& L, const double* phi, int hv,
                                 double eps, double rhocp_l, double rhocp_g, double* dst) {
  MF_CUDA_TRY(upload_tables_here());
  UniformGeom ug = uniform_geom(m);
  const double c_rhocp = 3.0 / (rhocp_g * rhocp_g + rhocp_l * rhocp_g + rhocp_l * rhocp_l);
  k_laser_load<<<brick_blocks(ug.nx, ug.ny, ug.nz), 128, 0, ctx->stream>>>(ug, L, phi, hv, eps, rhocp_l, rhocp_g,
                                                                           c_rhocp, dst);
  MF_STEP_LAUNCH_END;
}

mf_status launch_flow_forces(mf_ctx* ctx, const mf_dofmap* mu, const StepForces& F, const double* phi,
                             const double* T, const double* rho_tab, double* dst) {
  MF_CUDA_TRY(upload_tables_here());
  UniformGeom ug = uniform_geom(mu);
  k_flow_forces<<<brick_blocks(ug.nx, ug.ny, ug.nz), 128, 0, ctx->stream>>>(ug, F, phi, T, rho_tab, mu->n_cells,
                                                                            mu->n_dofs, dst);
  MF_STEP_LAUNCH_END;
}

}  // namespace mf
