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

namespace {

// Couplings of a 1D Q2 hat (lattice index a of 0..2n) with the Q1 hats of pressure nodes lo,
// lo + 1, lo + 2 (entries outside 0..n are 0): M = int phi_a psi_i / h, D = int phi_a' psi_i.
// On a cell [0, 1] with phi = (2x^2 - 3x + 1, 4x - 4x^2, 2x^2 - x), psi = (1 - x, x):
//   int phi psi  = [[1/6, 0], [1/3, 1/3], [0, 1/6]],
//   int phi' psi = [[-5/6, -1/6], [2/3, -2/3], [1/6, 5/6]],
// summed over the one cell (odd a) or two cells (even a) that hold node a.
__device__ __forceinline__ void hat_couplings(int a, int n, int& lo, float M[3], float D[3]) {
  const float s = 1.0f / 6.0f, t = 1.0f / 3.0f;
  if (a & 1) {
    lo = a >> 1;
    M[0] = t, M[1] = t, M[2] = 0.0f;
    D[0] = 2.0f * t, D[1] = -2.0f * t, D[2] = 0.0f;
    return;
  }
  const int i = a >> 1;
  lo = i - 1;
  M[0] = 0.0f, M[2] = 0.0f;
  if (i == 0) {
    M[1] = s;
    D[0] = 0.0f, D[1] = -5.0f * s, D[2] = -s;
  } else if (i == n) {
    M[1] = s;
    D[0] = s, D[1] = 5.0f * s, D[2] = 0.0f;
  } else {
    M[1] = t;
    D[0] = s, D[1] = 0.0f, D[2] = -s;
  }
}

// ub = D^-1 B^T p at every velocity node, node by node (no scatter, no atomics): on a uniform
// mesh the coupling factors into 1D couplings, (B^T p)_{v,x} = -h^2 sum_ijk D_a,i M_b,j M_c,k
// p_ijk (and likewise along y and z), which the cellwise Gauss quadrature evaluates exactly;
// here it is summed dimension by dimension over the 3 x 3 x 3 pressure nodes around the node.
// One grid row per lattice plane c (blockIdx.y), so the index arithmetic stays in 32 bits.
// blk: the fp32 inverses of the 3 x 3 nodal blocks of A_uu, entry-major (e * nu + node).
// Dirichlet nodes receive 0.
__global__ void __launch_bounds__(256) k_oseen_bt_dinv(const float* __restrict__ p, const float* __restrict__ blk,
                                                       float* __restrict__ ub, int64_t nu, UniformGeom ug) {
  const uint32_t sx = uint32_t(ug.sx), plane = uint32_t(ug.sy);
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= plane) return;
  const int a = int(t % sx), b = int(t / sx), c = int(blockIdx.y);
  const int64_t v = int64_t(c) * plane + t;
  const uint32_t f = ug.dir_faces;
  if (((f & 1u) && a == 0) || ((f & 2u) && a == 2 * ug.nx) || ((f & 4u) && b == 0) ||
      ((f & 8u) && b == 2 * ug.ny) || ((f & 16u) && c == 0) || ((f & 32u) && c == 2 * ug.nz)) {
    ub[v] = 0.0f;
    ub[nu + v] = 0.0f;
    ub[2 * nu + v] = 0.0f;
    return;
  }
  int lx, ly, lz;
  float Mx[3], Dx[3], My[3], Dy[3], Mz[3], Dz[3];
  hat_couplings(a, ug.nx, lx, Mx, Dx);
  hat_couplings(b, ug.ny, ly, My, Dy);
  hat_couplings(c, ug.nz, lz, Mz, Dz);
  const int px = ug.nx + 1, pxy = px * (ug.ny + 1);
  int oi[3], oj[3], ok[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    oi[s] = min(max(lx + s, 0), ug.nx);
    oj[s] = px * min(max(ly + s, 0), ug.ny);
    ok[s] = pxy * min(max(lz + s, 0), ug.nz);
  }
  float Qmm[3], Qdm[3], Qmd[3];
#pragma unroll
  for (int si = 0; si < 3; ++si) {
    Qmm[si] = 0.0f, Qdm[si] = 0.0f, Qmd[si] = 0.0f;
#pragma unroll
    for (int sj = 0; sj < 3; ++sj) {
      float pm = 0.0f, pd = 0.0f;
#pragma unroll
      for (int sk = 0; sk < 3; ++sk) {
        const float pv = __ldg(p + (oi[si] + oj[sj] + ok[sk]));
        pm = fmaf(Mz[sk], pv, pm);
        pd = fmaf(Dz[sk], pv, pd);
      }
      Qmm[si] = fmaf(My[sj], pm, Qmm[si]);
      Qdm[si] = fmaf(Dy[sj], pm, Qdm[si]);
      Qmd[si] = fmaf(My[sj], pd, Qmd[si]);
    }
  }
  const float sc = -float(ug.h * ug.h);
  float gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll
  for (int si = 0; si < 3; ++si) {
    gx = fmaf(Dx[si], Qmm[si], gx);
    gy = fmaf(Mx[si], Qdm[si], gy);
    gz = fmaf(Mx[si], Qmd[si], gz);
  }
  gx *= sc, gy *= sc, gz *= sc;
  ub[v] = blk[v] * gx + blk[nu + v] * gy + blk[2 * nu + v] * gz;
  ub[nu + v] = blk[3 * nu + v] * gx + blk[4 * nu + v] * gy + blk[5 * nu + v] * gz;
  ub[2 * nu + v] = blk[6 * nu + v] * gx + blk[7 * nu + v] * gy + blk[8 * nu + v] * gz;
}

}  // namespace

mf_status launch_oseen_bt_dinv_f32(mf_ctx* ctx, const mf_dofmap* mu, const float* p, const float* blk, float* ub) {
  UniformGeom ug = uniform_geom(mu);
  const int64_t nu = mu->n_dofs;
  // 32-bit plane and pressure indices; the grid's y extent is limited to 65535 planes
  if (ug.sy >= (int64_t(1) << 31) || int64_t(ug.nx + 1) * (ug.ny + 1) * (ug.nz + 1) >= (int64_t(1) << 31) ||
      2 * ug.nz + 1 > 65535)
    return fail(MF_EUNSUPPORTED, "node-wise coupling kernel: mesh too large for 32-bit plane indices");
  const dim3 grid(unsigned((ug.sy + 255) / 256), unsigned(2 * ug.nz + 1));
  k_oseen_bt_dinv<<<grid, 256, 0, ctx->stream>>>(p, blk, ub, nu, ug);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

}  // namespace mf
