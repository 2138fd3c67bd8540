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
  if (a.qouter)  // fewer fp64 operations per cell, at the price of register spills
    k_oseen_qouter<double><<<brick_blocks(ug.nx, ug.ny, ug.nz), 128, 0, ctx->stream>>>(a, ug);
  else
    k_oseen<double><<<brick_blocks(ug.nx, ug.ny, ug.nz), 128, 0, ctx->stream>>>(a, ug);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

}  // namespace mf
