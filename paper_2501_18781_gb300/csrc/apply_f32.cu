// float instantiation of the apply kernels.
#include "apply_kernels.cuh"
#include <cuda_fp16.h>

#include "vec.cuh"

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

constexpr int kSchurRows = 64;  // pressure rows per block of the assembly

// S~ = B D^-1 B^T on the pressure grid as a 5 x 5 x 5 stencil (the scaled fp16 tiled layout of
// stencil_at; scale[i] = the row's largest magnitude, 1 for an empty row):
// entry o of row i couples pressure node i with node i + (ox, oy, oz), o = (ox + 2) + 5 (oy + 2) +
// 25 (oz + 2), 0 where that node lies outside the grid.  With b(v, i) the column of B^T of pressure node i at velocity
// node v (on a uniform mesh, (B^T)_{v,x; i} = -h^2 D_{a,ix} M_{b,iy} M_{c,iz} and likewise along y
// and z, from the 1D couplings above), S~_{i,i'} = sum over the non-Dirichlet velocity nodes v
// within two lattice steps of i of b(v, i)^T D_v^-1 b(v, i').  One thread per pressure row; its
// 125 sums live in shared memory as [o][thread].  blk: the fp32 nodal block inverses,
// entry-major (e nu + v, e = 3 row + column); fp32 arithmetic (the result is the operator of an
// inner preconditioner solve).
__global__ void __launch_bounds__(kSchurRows) k_schur_assemble(const float* __restrict__ blk, __half* __restrict__ S,
                                                               float* __restrict__ scale, int64_t nu, UniformGeom ug) {
  __shared__ float acc[125 * kSchurRows];
  const int px = ug.nx + 1, py = ug.ny + 1;
  const int64_t np = int64_t(px) * py * (ug.nz + 1);
  const int64_t row = int64_t(blockIdx.x) * kSchurRows + threadIdx.x;
  for (int o = 0; o < 125; ++o) acc[o * kSchurRows + threadIdx.x] = 0.0f;
  if (row >= np) return;
  const int ix = int(row % px), iy = int((row / px) % py), iz = int(row / (int64_t(px) * py));
  const float sc = -float(ug.h * ug.h);
  const uint32_t f = ug.dir_faces;
  for (int c = max(0, 2 * iz - 2); c <= min(2 * ug.nz, 2 * iz + 2); ++c) {
    int lz;
    float Mz[3], Dz[3];
    hat_couplings(c, ug.nz, lz, Mz, Dz);
    const int qz = iz - lz;  // the slot of row i in node c's couplings: 0..2
    if (((f & 16u) && c == 0) || ((f & 32u) && c == 2 * ug.nz)) continue;
    for (int b = max(0, 2 * iy - 2); b <= min(2 * ug.ny, 2 * iy + 2); ++b) {
      int ly;
      float My[3], Dy[3];
      hat_couplings(b, ug.ny, ly, My, Dy);
      const int qy = iy - ly;
      if (((f & 4u) && b == 0) || ((f & 8u) && b == 2 * ug.ny)) continue;
      for (int a = max(0, 2 * ix - 2); a <= min(2 * ug.nx, 2 * ix + 2); ++a) {
        if (((f & 1u) && a == 0) || ((f & 2u) && a == 2 * ug.nx)) continue;
        int lx;
        float Mx[3], Dx[3];
        hat_couplings(a, ug.nx, lx, Mx, Dx);
        const int qx = ix - lx;
        const float bx = sc * Dx[qx] * My[qy] * Mz[qz];
        const float by = sc * Mx[qx] * Dy[qy] * Mz[qz];
        const float bz = sc * Mx[qx] * My[qy] * Dz[qz];
        if (bx == 0.0f && by == 0.0f && bz == 0.0f) continue;
        const int64_t v = a + ug.sx * b + ug.sy * c;
        // w^T = b(v, i)^T D_v^-1
        const float w0 = bx * blk[v] + by * blk[3 * nu + v] + bz * blk[6 * nu + v];
        const float w1 = bx * blk[nu + v] + by * blk[4 * nu + v] + bz * blk[7 * nu + v];
        const float w2 = bx * blk[2 * nu + v] + by * blk[5 * nu + v] + bz * blk[8 * nu + v];
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            const float myz = My[t] * Mz[u], dyz = Dy[t] * Mz[u], mdz = My[t] * Dz[u];
            const int oyz = 5 * (ly + t - iy + 2) + 25 * (lz + u - iz + 2);
#pragma unroll
            for (int s2 = 0; s2 < 3; ++s2) {
              const float val = sc * (w0 * (Dx[s2] * myz) + w1 * (Mx[s2] * dyz) + w2 * (Mx[s2] * mdz));
              acc[(oyz + lx + s2 - ix + 2) * kSchurRows + threadIdx.x] += val;
            }
          }
      }
    }
  }
  float big = 0.0f;
  for (int o = 0; o < 125; ++o) big = fmaxf(big, fabsf(acc[o * kSchurRows + threadIdx.x]));
  const float sr = big > 0.0f ? big : 1.0f;
  scale[row] = sr;
  for (int o = 0; o < 125; ++o) S[stencil_at(o, row)] = __float2half_rn(acc[o * kSchurRows + threadIdx.x] / sr);
  for (int o = 125; o < 128; ++o) S[stencil_at(o, row)] = __float2half_rn(0.0f);
}

}  // namespace

mf_status launch_schur_assemble_f32(mf_ctx* ctx, const mf_dofmap* mu, const float* blk, void* S, float* scale) {
  UniformGeom ug = uniform_geom(mu);
  const int64_t np = int64_t(ug.nx + 1) * (ug.ny + 1) * (ug.nz + 1);
  k_schur_assemble<<<unsigned((np + kSchurRows - 1) / kSchurRows), kSchurRows, 0, ctx->stream>>>(
      blk, static_cast<__half*>(S), scale, mu->n_dofs, ug);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

}  // namespace mf
