// Operator state and kernel launchers (internal).
#pragma once

#include "cellops.cuh"
#include "internal.h"

namespace mf {

enum ScalarKind { K_HELM = 0, K_HEAT = 1, K_REINIT = 2, K_MASS = 3 };
// arithmetic of an apply: fp64, fp32, or double-float (fp64 storage, pairs of fp32 in the kernel)
enum ApplyPrec { PREC_F64 = 0, PREC_F32 = 1, PREC_DF64 = 2, PREC_F16 = 3, PREC_BF16 = 4, PREC_TC = 5 };

// Arguments of the scalar cell kernels.  Vector fields are in the apply precision T.
template <typename T> struct ScalarArgs {
  const T* src;
  T* dst;
  int nrhs;
  int64_t ld;
  const T* field;   // nodal phi (Helmholtz, reinit) or T^n (heat) for in-kernel coefficients
  const T* qcoef;   // [27][ncp] scalar coefficient per Gauss point (a, k) when tabulated
  const T* qvec;    // [3][27][ncp] rho_cp beta (heat) or n (reinit) per Gauss point
  const T* qmass;   // [27][ncp] value-term coefficient per Gauss point (heat with rho_cp,q), or NULL
  int64_t ncp;      // stride of the Gauss-point tables (number of cells)
  T mass;           // value-term coefficient
  T a_l, a_g;       // Helmholtz: a = a_g + (a_l - a_g) H
  T k0, k_slope;    // heat: k = k0 + k_slope T
  T eps;            // reinit diffusion / sine Heaviside width
  int heaviside;    // 0 tanh, 1 sine
  // K_MASS only: restrict to cells whose centre lies in a box (|x|,|y| <= bx, z >= bz)
  int use_box;
  double box_half, box_zmin, lo[3];
  // launch shape (autotuned): octree cells per block (64 or 128) and, if > 0, a persistent
  // grid of persistent_blocks blocks per SM striding over the work units
  int block;
  int persistent_blocks;
};

template <typename T> struct OseenArgs {
  const T* src;
  T* dst;
  int64_t nu, np;   // velocity DoFs per component, pressure DoFs
  const T* rho;     // [27][ncells]
  const T* mu;      // [27][ncells]
  const T* beta;    // [3][27][ncells]
  T sigma;
  int qouter;       // 1: Gauss-point loop outside the velocity components (autotuned variant)
  // melt-pool extensions (ext = 1): extra mass coefficient (Darcy) and interface normal per Gauss
  // point; kd and nrm hold zeros for a term that is switched off
  int ext;
  const T* kd;      // [27][ncells]
  const T* nrm;     // [3][27][ncells]
  // Gauss-point coefficients with the weight and the powers of h folded in (Gauss-point-outer
  // kernel): cm = w h^3 (sigma rho + Darcy), cv = w h mu, each [27][ncells], and the convection
  // velocity times w h^2 rho, cb [3][27][ncells]
  const T* cm;
  const T* cb;
  const T* cv;
};

// scalar apply: kind, coefficient mode (0 in-kernel, 1 tabulated), convection, transpose
mf_status launch_scalar_apply(mf_ctx* ctx, const mf_dofmap* m, int kind, int mode, bool beta, bool transpose,
                              int prec, const void* args);
mf_status launch_oseen_apply(mf_ctx* ctx, const mf_dofmap* mu, int prec, const void* args);
// Oseen coupling blocks alone: which 0 dst_u = B^T src_p, which 1 dst_p = B src_u (dst zeroed)
mf_status launch_oseen_coupling_f64(mf_ctx* ctx, const mf_dofmap* mu, int which, const double* src, double* dst);
mf_status launch_oseen_coupling_f32(mf_ctx* ctx, const mf_dofmap* mu, int which, const float* src, float* dst);
// S~ = B D^-1 B^T as a 125-point stencil on the pressure grid (uniform Q2 velocity map; blk: fp32
// inverses of the 3 x 3 nodal blocks, entry-major; S: stencil_halves(n_p) fp16 entries in the
// scaled tiled layout of stencil_at, scale: n_p row factors; both overwritten)
mf_status launch_schur_assemble_f32(mf_ctx* ctx, const mf_dofmap* mu, const float* blk, void* S, float* scale);
// Gauss-point tables from nodal fp64 fields (always evaluated in fp64, stored in both precisions)
// (heat: rhocp_q / beta_q are the optional per-Gauss-point fields; qmass gets rhocp_q / dt)
mf_status launch_scalar_qtables(mf_ctx* ctx, const mf_dofmap* m, int kind, const double* field, const double* kq_user,
                                const double* beta, double k0, double k_slope, double a_l, double a_g, int heaviside,
                                double eps, double rhocp, double* qcoef64, float* qcoef32, double* qvec64, float* qvec32,
                                const double* rhocp_q = nullptr, const double* beta_q = nullptr, double dt = 1.0,
                                double* qmass64 = nullptr, float* qmass32 = nullptr);
mf_status launch_oseen_qtables(mf_ctx* ctx, const mf_dofmap* mu, const double* phi, const double* beta, double rho_l,
                               double rho_g, double mu_l, double mu_g, int heaviside, double eps, double* rho64,
                               float* rho32, double* muq64, float* muq32, double* beta64, float* beta32);
// folded coefficients cm, cv, cb of the Gauss-point-outer Oseen kernel from rho, mu, beta (and kd)
mf_status launch_oseen_fold(mf_ctx* ctx, const mf_dofmap* mu, double sigma, const double* rho, const double* muq,
                            const double* kd, const double* beta, double* cm64, float* cm32, double* cb64, float* cb32,
                            double* cv64,
                            float* cv32);
// melt-pool extension tables (three-phase rho/mu overwrite the two-phase ones; Darcy mass; normal)
mf_status launch_oseen_ext_tables(mf_ctx* ctx, const mf_dofmap* mu, const mf_op_params& p, const double* phi,
                                  const double* T, double* rho64, float* rho32, double* muq64, float* muq32,
                                  double* kd64, float* kd32, double* nrm64, float* nrm32);
// diagonal (scalar ops) in fp64 from tabulated coefficients
mf_status launch_scalar_diag(mf_ctx* ctx, const mf_dofmap* m, int kind, bool beta, const ScalarArgs<double>& a,
                             double* diag);
// Oseen block-Jacobi: 3x3 velocity blocks (inverted in place) and pressure scaling
mf_status launch_oseen_blockdiag(mf_ctx* ctx, const mf_dofmap* mu, const mf_dofmap* mp, const OseenArgs<double>& a,
                                 double* blk, double* pdiag);
// the same in fp32 from the folded fp32 tables (a: oseen_args<float>): blk = the inverted blocks,
// entry-major (blk[e nu + node], identity at Dirichlet nodes), pinv = the inverse pressure scaling
mf_status launch_oseen_blockdiag32(mf_ctx* ctx, const mf_dofmap* mu, const mf_dofmap* mp, const OseenArgs<float>& a,
                                   float* blk, float* pinv);
// dst[dir] = src[dir] for nrhs vectors (Dirichlet identity rows)
mf_status launch_dirichlet_copy(mf_ctx* ctx, const mf_dofmap* m, const void* src, void* dst, int nrhs, int64_t ld,
                                int64_t offset, bool f32);
// scalar operators in packed 16-bit arithmetic on fp32 vectors (prec PREC_F16 / PREC_BF16)
mf_status launch_scalar_apply_h16(mf_ctx* ctx, const mf_dofmap* m, int kind, int prec, const ScalarArgs<float>& a,
                                  float scale, float cnorm);
mf_status abs_max_f32(mf_ctx* ctx, const float* x, int64_t n, float* out);
// interface source terms (evaporative dilation, cooling, hybrid recoil) on an Oseen mesh
mf_status launch_interface_sources(mf_ctx* ctx, const mf_dofmap* mu, const mf_dofmap* mp, const mf_op_params& p,
                                   const double* phi, const mf_evaporation& ev, const double* T, double* fu,
                                   double* fp, double* fT);
// Q3 / Q4 Helmholtz (uniform maps): Gauss-point coefficient table [cell][q], apply, diagonal
mf_status launch_qk_coef(mf_ctx* ctx, const mf_dofmap* m, const double* phi, double a_l, double a_g, int heaviside,
                         double eps, double* c64, float* c32);
template <typename T>
mf_status launch_helmholtz_qk(mf_ctx* ctx, const mf_dofmap* m, const T* src, T* dst, const T* coef, double mass);
// Q2 Helmholtz / heat (no convection) on a uniform map by the line-per-thread kernel of degree 2:
// coef the [q][cell] Gauss-point table of the scalar coefficient, mass the value coefficient; dst is
// accumulated (zero it first); Dirichlet rows receive nothing
template <typename T>
mf_status launch_q2_line(mf_ctx* ctx, const mf_dofmap* m, const T* src, T* dst, const T* coef, double mass);
mf_status launch_qk_diag(mf_ctx* ctx, const mf_dofmap* m, const double* coef, double mass, double* diag);
// Q3 Helmholtz on the tensor cores (fp32 vectors, dst accumulated; coef per tile of 128 cells,
// [tile][q][row], from launch_tc_coef_layout).  A launch returns MF_ETIMEOUT when an earlier one
// stopped at its bounded wait.
mf_status launch_tc_coef_layout(mf_ctx* ctx, const mf_dofmap* m, const float* in, float* out);
mf_status launch_helmholtz_q3_tc(mf_ctx* ctx, const mf_dofmap* m, const float* src, float* dst, const float* coef,
                                 double mass);
// MF_ETIMEOUT (once, then the flag is cleared) if a tensor-core launch timed out; read it after
// the stream has synchronised to cover the launches of the last call
mf_status tc_take_error();
// double-float scalar apply on uniform meshes (Helmholtz, heat without convection or Gauss-point
// rho_cp): the tabulated coefficient split into float pairs of w_q h c_q, then the apply (dst
// accumulated, nrhs vectors ld apart)
mf_status launch_df_coef_split(mf_ctx* ctx, const mf_dofmap* m, const double* qcoef64, float* ch, float* cl);
// the convective heat operator (transpose: its adjoint) in double-float on a uniform mesh; bh, bl the
// float pairs of w_q h^2 rho_cp beta_d ([3][27][ncells], from launch_df_vec_split)
mf_status launch_scalar_df_uniform_conv(mf_ctx* ctx, const mf_dofmap* m, const double* src, double* dst, int nrhs,
                                        int64_t ld, const float* ch, const float* cl, const float* bh, const float* bl,
                                        double mass, bool transpose, const float* mh = nullptr,
                                        const float* ml = nullptr);
mf_status launch_df_vec_split(mf_ctx* ctx, const mf_dofmap* m, const double* qvec64, float* bh, float* bl);
// [27][ncells] value coefficients m_q -> w_q h^3 m_q as float pairs (the mh, ml of the kernel above)
mf_status launch_df_mass_split(mf_ctx* ctx, const mf_dofmap* m, const double* qmass64, float* mh, float* ml);
// the reinitialisation operator in double-float on an octree map (normals from the float pairs of
// the fp64 Gauss-point table, [3][27][ncells]); dst zeroed by the caller, Dirichlet rows left alone
mf_status launch_reinit_df_octree(mf_ctx* ctx, const mf_dofmap* m, const double* src, double* dst, int nrhs,
                                  int64_t ld, const float* nh, const float* nl, double eps, double mass);
mf_status launch_scalar_df_uniform(mf_ctx* ctx, const mf_dofmap* m, const double* src, double* dst, int nrhs,
                                   int64_t ld, const float* ch, const float* cl, double mass);
// double-float Oseen apply on uniform meshes: the folded coefficient tables cm, cv (27 per cell) and
// cb (81 per cell) as float pairs (high parts, then low parts); nr: the melt-pool interface normal
// table (81 per cell, pairs) for the trace correction, or NULL without the melt-pool terms
mf_status launch_split_pairs(mf_ctx* ctx, const double* c, int64_t n, float* h, float* l);
mf_status launch_oseen_df_uniform(mf_ctx* ctx, const mf_dofmap* mu, const double* src, double* dst, const float* cm,
                                  const float* cv, const float* cb, const float* nr);
// laser top-face load and its parameter derivatives (uniform maps)
mf_status launch_laser(mf_ctx* ctx, const mf_dofmap* m, const double lz[5], double* f, double* dF);
// dJ/dk_q = -w_q h grad(lambda) . grad(theta), [cell][27]
mf_status launch_grad_kq(mf_ctx* ctx, const mf_dofmap* m, const double* lam, const double* theta, double* out);

}  // namespace mf

struct mf_op {
  mf_ctx* ctx = nullptr;
  mf_op_params p{};
  const mf_dofmap* map[2] = {nullptr, nullptr};
  int nmaps = 1;
  int64_t n = 0;        // vector length
  int64_t ncells = 0;
  // borrowed nodal fields (fp64)
  const double* phi = nullptr;
  const double* tprev = nullptr;
  const double* beta = nullptr;
  const double* kq_user = nullptr;
  const double* rhocp_user = nullptr;   // heat: rho_cp per Gauss point [cell][27]
  const double* betaq_user = nullptr;   // heat: convection velocity per Gauss point [cell][27][3]
  // owned copies / tables
  mf::DevBuf field32;             // float copy of the in-kernel nodal field
  mf::DevBuf qcoef64, qcoef32;    // [27][ncells]
  mf::DevBuf qvec64, qvec32;      // [3][27][ncells]
  mf::DevBuf qmass64, qmass32;    // [27][ncells] heat value term rho_cp,q / dt
  mf::DevBuf qmass_dfh, qmass_dfl;  // the same times w_q h^3 as float pairs (double-float applies)
  mf::DevBuf qcoef_tc;            // Q3 tensor-core apply: fp32 coefficients [tile of 128 cells][q][row]
  bool tc_ready = false;
  int qk_f32_tc = 0;              // Q3: plain fp32 applies run on the tensor cores (autotuned)
  mf::DevBuf rho64, rho32, mu64, mu32;  // Oseen
  mf::DevBuf kd64, kd32, nrm64, nrm32;  // Oseen melt-pool extensions
  mf::DevBuf cm64, cm32, cb64, cb32, cv64, cv32;  // Oseen folded Gauss-point coefficients
  mf::DevBuf diag64;              // cached diagonal (fp64)
  mf::DevBuf blk64, pdiag64;      // Oseen block Jacobi
  bool tables_ready = false;
  mf::DevBuf qcoef_dfh, qcoef_dfl;  // [27][ncells] float pairs of w_q h c_q for the double-float kernel
  mf::DevBuf qvec_dfh, qvec_dfl;    // [3][27][ncells] float pairs of w_q h^2 rho_cp beta (convection)
  bool df_ready = false;
  mf::DevBuf cm_df, cv_df, cb_df;   // Oseen: folded coefficients as float pairs (high, then low parts)
  mf::DevBuf nrm_df;                // Oseen melt-pool terms: the interface normal table as float pairs
  bool diag_ready = false;
  // Chebyshev bounds: lambda_max of D^-1 A from the first solve's Lanczos run, kept until a field
  // changes (the same number of steps from the same start vector gives the same estimate)
  bool lanczos_ready = false;
  int lanczos_steps = 0, lanczos_prec = 0;   // its step count and the arithmetic of its fp32 applies
  double lanczos_lmax = 0.0;
  int mode64 = 1, mode32 = 0;     // coefficient mode per precision (autotuned)
  int f64_prec = 0;               // arithmetic of fp64 applies inside solvers (PREC_F64 or PREC_DF64)
  int f32_prec = 1;               // arithmetic of fp32 applies inside solvers (PREC_F32, PREC_F16, PREC_BF16, PREC_TC)
  float h16_cnorm = 0.0f;         // 16-bit applies: power of two >= every coefficient (0: not computed)
  int block = 128;                // octree cells per block (autotuned: 64 or 128)
  int persistent_blocks = 0;      // > 0: persistent launch with this many blocks per SM (autotuned)
  bool df64_faster = false;
  int q2_line64 = 0, q2_line32 = 0;  // uniform Q2 Helmholtz / heat: the line-per-thread kernel (autotuned)       // autotuned: double-float beats the fp64 pipes (used when fp64_arith = 2)
  int oseen_qouter64 = 0;         // Oseen fp64 kernel variant (autotuned)
  std::string tune_record;        // JSON of the last autotuning
  std::string variant;
};
