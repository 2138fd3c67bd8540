// Apply launchers: dispatch on the arithmetic to the per-precision translation units, plus
// the Dirichlet-row copy.
#include "ops.h"

namespace mf {

mf_status launch_scalar_apply_f64(mf_ctx*, const mf_dofmap*, int, int, bool, bool, const ScalarArgs<double>&);
mf_status launch_scalar_apply_f32(mf_ctx*, const mf_dofmap*, int, int, bool, bool, const ScalarArgs<float>&);
mf_status launch_scalar_apply_df64(mf_ctx*, const mf_dofmap*, int, int, bool, bool, const ScalarArgs<double>&);
mf_status launch_oseen_apply_f64(mf_ctx*, const mf_dofmap*, const OseenArgs<double>&);
mf_status launch_oseen_apply_f32(mf_ctx*, const mf_dofmap*, const OseenArgs<float>&);
mf_status launch_oseen_apply_df64(mf_ctx*, const mf_dofmap*, const OseenArgs<double>&);

namespace {

template <typename T>
__global__ void k_dirichlet_copy(const T* src, T* dst, const int32_t* list, int64_t nlist, int nrhs, int64_t ld,
                                 int64_t offset) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= nlist * nrhs) return;
  int64_t r = t / nlist, i = list[t % nlist] + offset;
  dst[r * ld + i] = src[r * ld + i];
}


}  // namespace

UniformGeom uniform_geom(const mf_dofmap* m) {
  UniformGeom g;
  g.nx = m->mesh->n[0];
  g.ny = m->mesh->n[1];
  g.nz = m->mesh->n[2];
  g.sx = m->R[0] + 1;
  g.sy = (m->R[0] + 1) * (m->R[1] + 1);
  g.n_dofs = m->n_dofs;
  g.dir_faces = m->dirichlet_faces;
  g.h = m->mesh->h0;
  return g;
}

OctGeom oct_geom(const mf_dofmap* m) {
  OctGeom g{};
  if (m->uniform) return g;
  g.cmap = m->d_cell_map.as<int32_t>();
  g.level = m->d_cell_level.as<uint8_t>();
  g.order = m->d_order.as<int32_t>();
  g.rowptr = m->d_con_rowptr.as<int32_t>();
  g.cols = m->d_con_cols.as<int32_t>();
  g.w64 = m->d_con_w.as<double>();
  g.w32 = m->d_con_wf.as<float>();
  g.dflag = m->dirichlet_list.empty() ? nullptr : m->d_dir_flag.as<uint8_t>();
  g.ncp = m->n_cells_pad;
  g.ncells = m->n_cells;
  g.n_dofs = m->n_dofs;
  g.h0 = m->mesh->h0;
  return g;
}

mf_status launch_scalar_apply(mf_ctx* ctx, const mf_dofmap* m, int kind, int mode, bool beta, bool tr, int prec,
                              const void* args) {
  if (prec == PREC_F32)
    return launch_scalar_apply_f32(ctx, m, kind, mode, beta, tr, *static_cast<const ScalarArgs<float>*>(args));
  if (prec == PREC_DF64)
    return launch_scalar_apply_df64(ctx, m, kind, 1, beta, tr, *static_cast<const ScalarArgs<double>*>(args));
  return launch_scalar_apply_f64(ctx, m, kind, mode, beta, tr, *static_cast<const ScalarArgs<double>*>(args));
}

mf_status launch_oseen_apply(mf_ctx* ctx, const mf_dofmap* mu, int prec, const void* args) {
  if (prec == PREC_F32) return launch_oseen_apply_f32(ctx, mu, *static_cast<const OseenArgs<float>*>(args));
  if (prec == PREC_DF64) return launch_oseen_apply_df64(ctx, mu, *static_cast<const OseenArgs<double>*>(args));
  return launch_oseen_apply_f64(ctx, mu, *static_cast<const OseenArgs<double>*>(args));
}

mf_status launch_dirichlet_copy(mf_ctx* ctx, const mf_dofmap* m, const void* src, void* dst, int nrhs, int64_t ld,
                                int64_t offset, bool f32) {
  int64_t nl = int64_t(m->dirichlet_list.size());
  if (nl == 0 || nrhs == 0) return MF_OK;
  int64_t tot = nl * nrhs;
  int nb = int((tot + 255) / 256);
  if (f32)
    k_dirichlet_copy<float><<<nb, 256, 0, ctx->stream>>>(static_cast<const float*>(src), static_cast<float*>(dst),
                                                         m->d_dir_list.as<int32_t>(), nl, nrhs, ld, offset);
  else
    k_dirichlet_copy<double><<<nb, 256, 0, ctx->stream>>>(static_cast<const double*>(src), static_cast<double*>(dst),
                                                          m->d_dir_list.as<int32_t>(), nl, nrhs, ld, offset);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

}  // namespace mf
