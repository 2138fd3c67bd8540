// One time step of the overall solution algorithm (Algorithm algo:meltpooldg) on one uniform mesh:
// the operators of its four solves, their Gauss-point fields, and the order of the stages
// (predictors; level-set advection with the variant-1 transport velocity and Olsson's
// reinitialisation; the two-phase heat equation with the interface laser and evaporative cooling;
// the melt-pool Navier-Stokes step with surface tension, recoil, dilation and gravity).  Every
// field stays on the device; the host only sequences launches and solves.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <memory>
#include <new>
#include <utility>

#include "step_kernels.h"
#include "vec.cuh"

namespace mf {
mf_status ensure_tables(mf_op* op);
}

struct mf_meltpool_step {
  mf_ctx* ctx = nullptr;
  mf_meltpool_params p{};
  mf_evaporation ev{};
  const mf_dofmap *mu = nullptr, *mp = nullptr, *mphi = nullptr, *mT = nullptr;
  int64_t nu = 0, np = 0, nc = 0;
  // advection (heat form with rho_cp = 1, k = 0, Gauss-point velocity), reinitialisation, heat on
  // the temperature map and on the Dirichlet-free map (for A T^n), flow
  mf_op *adv = nullptr, *re = nullptr, *heat = nullptr, *heat_all = nullptr, *flow = nullptr;
  mf::DevBuf us, Ts, phis, ug, kzero, kq, rhocp, b, phia, psi, psi2, r, d, zero, fu, fp, bflow;
  mf::StepLaser laser{};
  mf::StepForces forces{};
  ~mf_meltpool_step() {
    for (mf_op* o : {adv, re, heat, heat_all, flow})
      if (o) mf_operator_destroy(o);
  }
};

namespace {

using clk = std::chrono::steady_clock;
using mf::fail;

mf_status make_op(mf_ctx* c, const mf_op_params& p, const mf_dofmap* m0, const mf_dofmap* m1, mf_op** out) {
  const mf_dofmap* maps[2] = {m0, m1};
  return mf_operator_create(c, &p, maps, m1 ? 2 : 1, out);
}

mf_solver_params scalar_solver(int solver, double tol, int maxit) {
  mf_solver_params s{};
  s.solver = solver;
  s.precond = MF_PREC_JACOBI;
  s.restart = 30;
  s.maxit = maxit;
  s.tol = tol;
  return s;
}

// solve and record; a stage that stops at maxit still hands its iterate on
mf_status run_solve(mf_op* op, const mf_solver_params& sp, const double* b, double* x, int* its, double* res,
                    mf_status* worst) {
  mf_solve_info si{};
  const mf_status st = mf_solve(op, &sp, b, x, 1, &si);
  if (st != MF_OK && st != MF_ENOTCONV) return st;
  if (st == MF_ENOTCONV) *worst = MF_ENOTCONV;
  *its += si.iterations;
  *res = si.rel_residual;
  return MF_OK;
}

mf_status copy_out(mf_ctx* c, double* dst, const double* src, int64_t n) {
  if (dst) MF_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
  return MF_OK;
}

mf_status check_params(const mf_meltpool_params& p) {
  if (!(p.dt > 0) || !(p.eps > 0)) return fail(MF_EINVAL, "dt and eps must be > 0");
  if (!(p.rho_l > 0) || !(p.rho_g > 0) || !(p.mu_l > 0) || !(p.mu_g > 0))
    return fail(MF_EINVAL, "densities and viscosities must be > 0");
  if (!(p.rhocp_l > 0) || !(p.rhocp_g > 0) || !(p.k_l >= 0) || !(p.k_g >= 0))
    return fail(MF_EINVAL, "rho_cp must be > 0 and k >= 0");
  if (p.reinit_steps < 0 || (p.reinit_steps > 0 && !(p.dtau > 0)))
    return fail(MF_EINVAL, "reinit_steps must be >= 0 (with dtau > 0)");
  if (!(p.tol > 0) || !(p.flow_tol > 0)) return fail(MF_EINVAL, "tolerances must be > 0");
  if (p.laser_on) {
    const double dn = std::sqrt(p.laser_direction[0] * p.laser_direction[0] + p.laser_direction[1] * p.laser_direction[1] +
                                p.laser_direction[2] * p.laser_direction[2]);
    if (!(p.laser_radius > 0) || !(dn > 0)) return fail(MF_EINVAL, "laser radius and direction must be nonzero");
  }
  return MF_OK;
}

}  // namespace

extern "C" {

mf_status mf_meltpool_create(mf_ctx* c, const mf_meltpool_params* params, const mf_dofmap* u_map,
                             const mf_dofmap* p_map, const mf_dofmap* phi_map, const mf_dofmap* T_map,
                             mf_meltpool_step** out) {
  try {
    if (!c || !params || !u_map || !p_map || !phi_map || !T_map || !out) return fail(MF_EINVAL, "NULL argument");
    const mf_mesh* mesh = u_map->mesh;
    for (const mf_dofmap* m : {u_map, p_map, phi_map, T_map})
      if (m->mesh != mesh || !m->uniform || mesh->ctx != c)
        return fail(MF_EINVAL, "all maps must be uniform maps of one mesh of this context");
    if (u_map->degree != 2 || p_map->degree != 1 || phi_map->degree != 2 || T_map->degree != 2)
      return fail(MF_EINVAL, "maps must be Q2 velocity, Q1 pressure, Q2 level set, Q2 temperature");
    if (phi_map->dirichlet_faces != 0) return fail(MF_EINVAL, "the level-set map has no Dirichlet faces");
    MF_TRY(check_params(*params));
    std::unique_ptr<mf_meltpool_step> s(new mf_meltpool_step);
    mf_meltpool_step& S = *s;
    const mf_meltpool_params& p = *params;
    S.ctx = c;
    S.p = p;
    S.mu = u_map;
    S.mp = p_map;
    S.mphi = phi_map;
    S.mT = T_map;
    S.nu = u_map->n_dofs;
    S.np = p_map->n_dofs;
    S.nc = u_map->n_cells;
    S.ev = p.evaporation;
    S.ev.rhocp_liquid = p.rhocp_l;
    S.ev.rhocp_gas = p.rhocp_g;
    // operators
    mf_op_params a{};
    a.kind = MF_OP_HEAT;
    a.coef_mode = MF_COEF_QPOINT;
    a.rhocp = 1.0;
    a.dt = p.dt;
    MF_TRY(make_op(c, a, phi_map, nullptr, &S.adv));
    mf_op_params r{};
    r.kind = MF_OP_REINIT;
    r.coef_mode = MF_COEF_QPOINT;
    r.eps = p.eps;
    r.dtau = p.reinit_steps > 0 ? p.dtau : 1.0;
    MF_TRY(make_op(c, r, phi_map, nullptr, &S.re));
    mf_op_params h{};
    h.kind = MF_OP_HEAT;
    h.coef_mode = MF_COEF_QPOINT;
    h.rhocp = p.rhocp_l;  // replaced per Gauss point
    h.dt = p.dt;
    MF_TRY(make_op(c, h, T_map, nullptr, &S.heat));
    MF_TRY(make_op(c, h, phi_map, nullptr, &S.heat_all));
    mf_op_params f{};
    f.kind = MF_OP_OSEEN;
    f.sigma = 1.0 / p.dt;
    f.rho_l = p.rho_l;
    f.rho_g = p.rho_g;
    f.mu_l = p.mu_l;
    f.mu_g = p.mu_g;
    f.eps = p.eps;
    f.rho_s = p.rho_s;
    f.mu_s = p.mu_s;
    f.t_solidus = p.t_solidus;
    f.t_liquidus = p.t_liquidus;
    f.darcy_c = p.darcy_c;
    f.darcy_b = p.darcy_b;
    f.oseen_flags = p.oseen_flags;
    MF_TRY(make_op(c, f, u_map, p_map, &S.flow));
    // work vectors and Gauss-point tables
    const int64_t nu = S.nu, nq = 27 * S.nc;
    MF_TRY(S.us.alloc(sizeof(double) * 3 * nu));
    for (mf::DevBuf* v : {&S.Ts, &S.phis, &S.b, &S.phia, &S.psi, &S.psi2, &S.r, &S.d, &S.zero})
      MF_TRY(v->alloc(sizeof(double) * nu));
    MF_TRY(S.ug.alloc(sizeof(double) * 3 * nq));
    for (mf::DevBuf* v : {&S.kzero, &S.kq, &S.rhocp}) MF_TRY(v->alloc(sizeof(double) * nq));
    MF_TRY(S.fu.alloc(sizeof(double) * 3 * nu));
    MF_TRY(S.fp.alloc(sizeof(double) * S.np));
    MF_TRY(S.bflow.alloc(sizeof(double) * (3 * nu + S.np)));
    MF_CUDA_TRY(cudaMemsetAsync(S.kzero.p, 0, sizeof(double) * nq, c->stream));
    MF_CUDA_TRY(cudaMemsetAsync(S.zero.p, 0, sizeof(double) * nu, c->stream));
    // laser and forces
    if (p.laser_on) {
      const double* e = p.laser_direction;
      const double dn = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
      S.laser.q0 = 2.0 * p.laser_absorptivity * p.laser_power / (3.141592653589793 * p.laser_radius * p.laser_radius);
      S.laser.radius = p.laser_radius;
      for (int d = 0; d < 3; ++d) {
        S.laser.focus[d] = p.laser_focus[d];
        S.laser.dir[d] = e[d] / dn;
        S.laser.lo[d] = mesh->lo[d];
      }
    }
    mf::StepForces& F = S.forces;
    F.alpha0 = p.alpha0;
    F.alpha1 = p.alpha1;
    F.t_alpha = p.t_alpha;
    F.alpha_res = p.alpha_res;
    for (int d = 0; d < 3; ++d) F.g[d] = p.gravity[d];
    F.rho_l = p.rho_l;
    F.rho_g = p.rho_g;
    F.c_rho = (p.rho_g - p.rho_l) / (p.rho_l * p.rho_g * std::log(p.rho_g / p.rho_l));
    F.hv = 0;
    F.eps = p.eps;
    MF_CUDA_TRY(cudaStreamSynchronize(c->stream));
    *out = s.release();
    return MF_OK;
  } catch (const std::bad_alloc&) {
    return fail(MF_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(MF_EINVAL, "internal exception");
  }
}

void mf_meltpool_destroy(mf_meltpool_step* step) { delete step; }

mf_status mf_meltpool_advance(mf_meltpool_step* step, const double* u_prev, const double* u, const double* T_prev,
                              const double* T, const double* phi_prev, const double* phi, double* up, double* T_out,
                              double* phi_out, mf_meltpool_trace* trace, mf_meltpool_info* info) {
  try {
    if (!step || !u_prev || !u || !T_prev || !T || !phi_prev || !phi || !up || !T_out || !phi_out)
      return fail(MF_EINVAL, "NULL argument");
    mf_meltpool_step& S = *step;
    mf_ctx* c = S.ctx;
    const mf_meltpool_params& p = S.p;
    const int64_t nu = S.nu, np = S.np;
    const int maxit = p.maxit > 0 ? p.maxit : 5000;
    double* us = S.us.as<double>();
    double* Ts = S.Ts.as<double>();
    double* phis = S.phis.as<double>();
    double* b = S.b.as<double>();
    double* phia = S.phia.as<double>();
    mf_meltpool_info inf{};
    mf_status worst = MF_OK;
    const auto t0 = clk::now();
    auto lap = [&](int k, clk::time_point& t) -> mf_status {
      MF_CUDA_TRY(cudaStreamSynchronize(c->stream));
      const auto now = clk::now();
      inf.seconds[k] = std::chrono::duration<double>(now - t).count();
      t = now;
      return MF_OK;
    };
    clk::time_point t = t0;

    // 1. predictors
    MF_TRY(mf::launch_extrapolate(c, 3 * nu, u, u_prev, us));
    MF_TRY(mf::launch_extrapolate(c, nu, T, T_prev, Ts));
    MF_TRY(mf::launch_extrapolate(c, nu, phi, phi_prev, phis));
    // 2. level set: advection with the variant-1 transport velocity
    MF_TRY(mf::launch_transport_velocity(c, S.mphi, us, Ts, phis, S.ev, p.rho_l, p.rho_g, 0, p.eps, S.ug.as<double>()));
    MF_TRY(mf_operator_set_field(S.adv, MF_FIELD_BETA_QPOINT, S.ug.p, MF_F64, 81 * S.nc));
    MF_TRY(mf_operator_set_field(S.adv, MF_FIELD_K_QPOINT, S.kzero.p, MF_F64, 27 * S.nc));
    MF_CUDA_TRY(cudaMemsetAsync(b, 0, sizeof(double) * nu, c->stream));
    MF_TRY(mf::launch_mass_load(c, S.mphi, phi, nullptr, 0, 0, 1.0 / p.dt, false, b));
    if (trace) {
      MF_TRY(copy_out(c, trace->u_star, us, 3 * nu));
      MF_TRY(copy_out(c, trace->T_star, Ts, nu));
      MF_TRY(copy_out(c, trace->phi_star, phis, nu));
      MF_TRY(copy_out(c, trace->u_gamma, S.ug.as<double>(), 81 * S.nc));
      MF_TRY(copy_out(c, trace->b_advection, b, nu));
    }
    // defect correction: fp32 inner GMRES, the outer residuals with double-float applies
    mf_solver_params as = scalar_solver(MF_SOLVER_DEFECT_CORRECTION, p.tol, maxit);
    as.inner_dtype = MF_F32;
    as.fp64_arith = 1;
    MF_TRY(run_solve(S.adv, as, b, phia, &inf.advection_iterations, &inf.advection_residual, &worst));
    if (trace) MF_TRY(copy_out(c, trace->phi_advected, phia, nu));
    MF_TRY(lap(0, t));

    // 2. level set: reinitialisation with the normal of phi_a
    MF_TRY(mf_operator_set_field(S.re, MF_FIELD_PHI, phia, MF_F64, nu));
    MF_CUDA_TRY(cudaMemcpyAsync(S.psi.p, phia, sizeof(double) * nu, cudaMemcpyDeviceToDevice, c->stream));
    for (int k = 0; k < p.reinit_steps; ++k) {
      MF_CUDA_TRY(cudaMemsetAsync(b, 0, sizeof(double) * nu, c->stream));
      MF_TRY(mf::launch_mass_load(c, S.mphi, S.psi.as<double>(), nullptr, 0, 0, 1.0 / p.dtau, false, b));
      MF_TRY(mf::launch_compressive_flux(c, S.mphi, S.psi.as<double>(), phia, b));
      mf_solver_params rs = scalar_solver(MF_SOLVER_CG, p.tol, maxit);
      if (p.reinit_mixed) {  // fp32 Chebyshev-CG inner solves, fp64 residuals
        rs.solver = MF_SOLVER_DEFECT_CORRECTION;
        rs.precond = MF_PREC_CHEBYSHEV;
        rs.inner_dtype = MF_F32;
        rs.maxit = 100;
      }
      MF_TRY(run_solve(S.re, rs, b, S.psi2.as<double>(), &inf.reinit_iterations, &inf.reinit_residual, &worst));
      std::swap(S.psi.p, S.psi2.p);
    }
    MF_CUDA_TRY(cudaMemcpyAsync(phi_out, S.psi.p, sizeof(double) * nu, cudaMemcpyDeviceToDevice, c->stream));
    MF_TRY(lap(1, t));

    // 3. heat: two-phase coefficients of phi^(n+1), sources, update T^(n+1) - T^n
    MF_TRY(mf::launch_heat_coefficients(c, S.mphi, phi_out, 0, p.eps, p.rhocp_l, p.rhocp_g, p.k_l, p.k_g,
                                        S.kq.as<double>(), S.rhocp.as<double>()));
    for (mf_op* o : {S.heat, S.heat_all}) {
      MF_TRY(mf_operator_set_field(o, MF_FIELD_K_QPOINT, S.kq.p, MF_F64, 27 * S.nc));
      MF_TRY(mf_operator_set_field(o, MF_FIELD_RHOCP_QPOINT, S.rhocp.p, MF_F64, 27 * S.nc));
      MF_TRY(mf_operator_set_field(o, MF_FIELD_BETA, us, MF_F64, 3 * nu));
    }
    MF_CUDA_TRY(cudaMemsetAsync(b, 0, sizeof(double) * nu, c->stream));
    MF_TRY(mf::launch_mass_load(c, S.mphi, T, S.rhocp.as<double>(), 1, 27, 1.0 / p.dt, false, b));
    MF_TRY(mf::launch_interface_sources(c, S.mu, S.mp, S.flow->p, phi_out, S.ev, Ts, nullptr, nullptr,
                                        S.d.as<double>()));
    MF_TRY(mf::axpby<double, double>(c, nu, 1.0, S.d.as<double>(), 1.0, b));
    if (p.laser_on) MF_TRY(mf::launch_laser_interface(c, S.mphi, S.laser, phi_out, 0, p.eps, p.rhocp_l, p.rhocp_g, b));
    double* r = S.r.as<double>();
    MF_TRY(mf_apply(S.heat_all, T, r, 1, nu, MF_F64));
    MF_TRY(mf::axpby<double, double>(c, nu, 1.0, b, -1.0, r));
    MF_TRY(mf::launch_dirichlet_copy(c, S.mT, S.zero.p, r, 1, nu, 0, false));
    if (trace) MF_TRY(copy_out(c, trace->r_heat, r, nu));
    mf_solver_params hs = scalar_solver(MF_SOLVER_DEFECT_CORRECTION, p.tol, maxit);  // as the advection
    hs.inner_dtype = MF_F32;
    hs.fp64_arith = 1;
    MF_TRY(run_solve(S.heat, hs, r, S.d.as<double>(), &inf.heat_iterations, &inf.heat_residual, &worst));
    if (trace) MF_TRY(copy_out(c, trace->T_update, S.d.as<double>(), nu));
    MF_CUDA_TRY(cudaMemcpyAsync(T_out, T, sizeof(double) * nu, cudaMemcpyDeviceToDevice, c->stream));
    MF_TRY(mf::axpby<double, double>(c, nu, 1.0, S.d.as<double>(), 1.0, T_out));
    MF_TRY(lap(2, t));

    // 4. flow: the melt-pool Oseen system about u*
    MF_TRY(mf_operator_set_field(S.flow, MF_FIELD_PHI, phi_out, MF_F64, nu));
    MF_TRY(mf_operator_set_field(S.flow, MF_FIELD_BETA, us, MF_F64, 3 * nu));
    MF_TRY(mf_operator_set_field(S.flow, MF_FIELD_T_PREV, T_out, MF_F64, nu));
    MF_TRY(mf::ensure_tables(S.flow));
    double* bf = S.bflow.as<double>();
    MF_CUDA_TRY(cudaMemsetAsync(bf, 0, sizeof(double) * (3 * nu + np), c->stream));
    for (int k = 0; k < 3; ++k)
      MF_TRY(mf::launch_mass_load(c, S.mu, u + k * nu, S.flow->rho64.as<double>(), S.nc, 1, 1.0 / p.dt, true,
                                  bf + k * nu));
    MF_TRY(mf::launch_flow_forces(c, S.mu, S.forces, phi_out, T_out, S.flow->rho64.as<double>(), bf));
    MF_TRY(mf::launch_interface_sources(c, S.mu, S.mp, S.flow->p, phi_out, S.ev, T_out, S.fu.as<double>(),
                                        S.fp.as<double>(), nullptr));
    MF_TRY(mf::axpby<double, double>(c, 3 * nu, 1.0, S.fu.as<double>(), 1.0, bf));
    MF_TRY(mf::axpby<double, double>(c, np, -1.0, S.fp.as<double>(), 0.0, bf + 3 * nu));
    if (trace) MF_TRY(copy_out(c, trace->b_flow, bf, 3 * nu + np));
    mf_solver_params fs{};
    fs.solver = MF_SOLVER_GMRES;
    fs.precond = MF_PREC_BLOCK_TRIANGULAR;
    fs.restart = 50;
    fs.maxit = maxit;
    fs.tol = p.flow_tol;
    fs.velocity_steps = p.flow_velocity_steps;
    fs.schur_maxit = p.flow_schur_maxit;
    fs.schur_tol = p.flow_schur_tol;
    fs.use_graph = 1;
    fs.fp64_arith = 1;   // the outer Oseen applies in double-float (fp64-accurate, 1.14x the fp64 pipes at 64^3)
    MF_TRY(run_solve(S.flow, fs, bf, up, &inf.flow_iterations, &inf.flow_residual, &worst));
    MF_TRY(lap(3, t));
    inf.seconds[4] = std::chrono::duration<double>(clk::now() - t0).count();
    if (info) *info = inf;
    if (worst != MF_OK) return fail(worst, "a solve of the step stopped at maxit");
    return MF_OK;
  } catch (const std::bad_alloc&) {
    return fail(MF_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(MF_EINVAL, "internal exception");
  }
}

}  // extern "C"
