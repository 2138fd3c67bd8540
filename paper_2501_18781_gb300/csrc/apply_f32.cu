// float instantiation of the apply kernels.
#include "apply_kernels.cuh"

namespace mf {

mf_status launch_scalar_apply_f32(mf_ctx* ctx, const mf_dofmap* m, int kind, int mode, bool beta, bool tr,
                                   const ScalarArgs<float>& a) {
  return dispatch_scalar<float>(ctx, m, kind, mode, beta, tr, a);
}

mf_status launch_oseen_apply_f32(mf_ctx* ctx, const mf_dofmap* mu, const OseenArgs<float>& a) {
  MF_CUDA_TRY(upload_tables_here());
  UniformGeom ug = uniform_geom(mu);
  // fp32: all three velocity components fit in registers (Gauss-point loop outside)
  if (a.ext)
    k_oseen_qouter<float, true><<<brick_blocks(ug.nx, ug.ny, ug.nz), 128, 0, ctx->stream>>>(a, ug);
  else
    k_oseen_qouter<float><<<brick_blocks(ug.nx, ug.ny, ug.nz), 128, 0, ctx->stream>>>(a, ug);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

// which = 0: dst_u = B^T src_p; which = 1: dst_p = B src_u (dst zeroed by the caller)
mf_status launch_oseen_coupling_f32(mf_ctx* ctx, const mf_dofmap* mu, int which, const float* src, float* dst) {
  MF_CUDA_TRY(upload_tables_here());
  UniformGeom ug = uniform_geom(mu);
  const int nb = brick_blocks(ug.nx, ug.ny, ug.nz);
  if (which == 0)
    k_oseen_bt<float><<<nb, 128, 0, ctx->stream>>>(src, dst, mu->n_dofs, ug);
  else
    k_oseen_div<float><<<nb, 128, 0, ctx->stream>>>(src, mu->n_dofs, dst, ug);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

}  // namespace mf
