// double instantiation of the apply kernels.
#include "apply_kernels.cuh"

namespace mf {

mf_status launch_scalar_apply_f64(mf_ctx* ctx, const mf_dofmap* m, int kind, int mode, bool beta, bool tr,
                                   const ScalarArgs<double>& a) {
  return dispatch_scalar<double>(ctx, m, kind, mode, beta, tr, a);
}

mf_status launch_oseen_apply_f64(mf_ctx* ctx, const mf_dofmap* mu, const OseenArgs<double>& a) {
  MF_CUDA_TRY(upload_tables_here());
  UniformGeom ug = uniform_geom(mu);
  if (a.ext)  // melt-pool terms (three-phase tables, Darcy, trace correction)
    k_oseen_qouter<double, true><<<brick_blocks(ug.nx, ug.ny, ug.nz), 128, 0, ctx->stream>>>(a, ug);
  else if (a.qouter)  // fewer fp64 operations per cell, at the price of register spills
    k_oseen_qouter<double><<<brick_blocks(ug.nx, ug.ny, ug.nz), 128, 0, ctx->stream>>>(a, ug);
  else
    k_oseen<double><<<brick_blocks(ug.nx, ug.ny, ug.nz), 128, 0, ctx->stream>>>(a, ug);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

// which = 0: dst_u = B^T src_p; which = 1: dst_p = B src_u (dst zeroed by the caller)
mf_status launch_oseen_coupling_f64(mf_ctx* ctx, const mf_dofmap* mu, int which, const double* src, double* dst) {
  MF_CUDA_TRY(upload_tables_here());
  UniformGeom ug = uniform_geom(mu);
  const int nb = brick_blocks(ug.nx, ug.ny, ug.nz);
  if (which == 0)
    k_oseen_bt<double><<<nb, 128, 0, ctx->stream>>>(src, dst, mu->n_dofs, ug);
  else
    k_oseen_div<double><<<nb, 128, 0, ctx->stream>>>(src, mu->n_dofs, dst, ug);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

}  // namespace mf
