// Scalar operator applies in packed 16-bit arithmetic (fp16x2 or bf16x2): two right-hand sides
// share one thread's instructions, lane r and lane r+1 of every value.  Vectors stay fp32 in memory
// (gathered, packed, computed, unpacked, scattered with fp32 atomics); the Gauss-point
// coefficients are the fp32 tables, broadcast into both lanes.  This is the reduced-precision
// variant for smoothers: ~3 decimal digits (fp16) or ~2 (bf16) per operation.
//
// fp16 has a narrow exponent range (6e-5 .. 65504): the values are multiplied by a power of two
// (`scale`, chosen by the caller from the vector length so that unit-norm vectors have O(1)
// entries) before packing, every coefficient is divided by a power of two `cnorm` at or above the
// largest of them, and the result is multiplied by h cnorm / scale in fp32 after unpacking.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "apply_kernels.cuh"

namespace mf {

namespace {

// the same 1D tables in both 16-bit formats (uploaded with the other tables of this unit)
__constant__ __half2 cS_f16[9], cD_f16[9], cW3_f16[27];
__constant__ __nv_bfloat162 cS_b16[9], cD_b16[9], cW3_b16[27];

template <typename P> struct Pk;
template <> struct Pk<__half2> {
  static __device__ __forceinline__ __half2 two(float a, float b) { return __floats2half2_rn(a, b); }
  static __device__ __forceinline__ __half2 one(float a) { return __float2half2_rn(a); }
  static __device__ __forceinline__ float lo(__half2 v) { return __low2float(v); }
  static __device__ __forceinline__ float hi(__half2 v) { return __high2float(v); }
};
template <> struct Pk<__nv_bfloat162> {
  static __device__ __forceinline__ __nv_bfloat162 two(float a, float b) { return __floats2bfloat162_rn(a, b); }
  static __device__ __forceinline__ __nv_bfloat162 one(float a) { return __float2bfloat162_rn(a); }
  static __device__ __forceinline__ float lo(__nv_bfloat162 v) { return __low2float(v); }
  static __device__ __forceinline__ float hi(__nv_bfloat162 v) { return __high2float(v); }
};

}  // namespace

template <> struct Tb<__half2> {
  static __device__ __forceinline__ __half2 S(int q, int a) { return cS_f16[3 * q + a]; }
  static __device__ __forceinline__ __half2 D(int q, int p) { return cD_f16[3 * q + p]; }
  static __device__ __forceinline__ __half2 W3(int q) { return cW3_f16[q]; }
};
template <> struct Tb<__nv_bfloat162> {
  static __device__ __forceinline__ __nv_bfloat162 S(int q, int a) { return cS_b16[3 * q + a]; }
  static __device__ __forceinline__ __nv_bfloat162 D(int q, int p) { return cD_b16[3 * q + p]; }
  static __device__ __forceinline__ __nv_bfloat162 W3(int q) { return cW3_b16[q]; }
};

namespace {

cudaError_t upload_h16_tables() {
  static bool done = false;
  if (done) return cudaSuccess;
  Tables t = make_tables();
  __half2 h[27];
  __nv_bfloat162 b[27];
  cudaError_t e = cudaSuccess;
  auto up = [&](const void* sh, const void* sb, const double* src, int n) {
    for (int i = 0; i < n; ++i) {
      h[i] = __float2half2_rn(float(src[i]));
      b[i] = __float2bfloat162_rn(float(src[i]));
    }
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(sh, h, n * sizeof(__half2));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(sb, b, n * sizeof(__nv_bfloat162));
  };
  up(cS_f16, cS_b16, t.S, 9);
  up(cD_f16, cD_b16, t.D, 9);
  up(cW3_f16, cW3_b16, t.W3, 27);
  if (e == cudaSuccess) done = true;
  return e;
}

// One cell, right-hand sides r and r + 1 (the second lane idles when r + 1 == nrhs).  KIND:
// K_HELM / K_HEAT (scalar coefficient table) or K_REINIT (normal table); coefficients tabulated.
template <typename P, int KIND, bool OCT>
__device__ __forceinline__ void cell_pair(const ScalarArgs<float>& A, const UniformGeom& ug, const OctGeom& og,
                                          const CellLoc& L, int r, float scale, float inv_cnorm) {
  const bool two = r + 1 < A.nrhs;
  const float h = OCT ? float(L.h) : float(ug.h);
  P U[27];
  {
    float Ua[27], Ub[27];
    gather<float, OCT>(ug, og, L, A.src + r * A.ld, Ua);
    if (two) gather<float, OCT>(ug, og, L, A.src + (r + 1) * A.ld, Ub);
#pragma unroll
    for (int l = 0; l < 27; ++l) U[l] = Pk<P>::two(scale * Ua[l], two ? scale * Ub[l] : 0.0f);
  }
  to_qpoints<P>(U);
  const P mh2 = Pk<P>::one(A.mass * h * h * inv_cnorm);
  const P eps = Pk<P>::one(A.eps * inv_cnorm);
  P R[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) R[q] = Pk<P>::one(0.0f);
#pragma unroll
  for (int qc = 0; qc < 3; ++qc)
#pragma unroll
    for (int qb = 0; qb < 3; ++qb)
#pragma unroll
      for (int qa = 0; qa < 3; ++qa) {
        const int q = qa + 3 * qb + 9 * qc;
        const P w = Tb<P>::W3(q);
        P gx, gy, gz;
        grad_at<P>(U, qa, qb, qc, gx, gy, gz);
        P Fx, Fy, Fz;
        if constexpr (KIND == K_REINIT) {
          const P nx = Pk<P>::one(__ldg(A.qvec + (0 * 27 + q) * A.ncp + L.cell));
          const P ny = Pk<P>::one(__ldg(A.qvec + (1 * 27 + q) * A.ncp + L.cell));
          const P nz = Pk<P>::one(__ldg(A.qvec + (2 * 27 + q) * A.ncp + L.cell));
          const P s = w * (eps * (nx * gx + ny * gy + nz * gz));
          Fx = s * nx;
          Fy = s * ny;
          Fz = s * nz;
        } else {
          const P c = w * Pk<P>::one(__ldg(A.qcoef + q * A.ncp + L.cell) * inv_cnorm);
          Fx = c * gx;
          Fy = c * gy;
          Fz = c * gz;
        }
        R[q] += w * (mh2 * U[q]);
        add_grad_test<P>(R, qa, qb, qc, Fx, Fy, Fz);
      }
  to_nodes<P>(R);
  const float back = h / (scale * inv_cnorm);
  {
    float Ra[27];
#pragma unroll
    for (int l = 0; l < 27; ++l) Ra[l] = back * Pk<P>::lo(R[l]);
    scatter<float, OCT>(ug, og, L, A.dst + r * A.ld, Ra);
  }
  if (two) {
    float Rb[27];
#pragma unroll
    for (int l = 0; l < 27; ++l) Rb[l] = back * Pk<P>::hi(R[l]);
    scatter<float, OCT>(ug, og, L, A.dst + (r + 1) * A.ld, Rb);
  }
}

template <typename P, int KIND, bool OCT>
__global__ void __launch_bounds__(128) k_scalar_h16(ScalarArgs<float> A, UniformGeom ug, OctGeom og, int64_t nwork,
                                                    float scale, float inv_cnorm) {
  for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
    CellLoc L;
    if (!locate<OCT>(ug, og, w, L)) continue;
    for (int r = 0; r < A.nrhs; r += 2) cell_pair<P, KIND, OCT>(A, ug, og, L, r, scale, inv_cnorm);
  }
}

// largest |x| over a float array into *out, compared as bit patterns of |x| (all non-negative)
__global__ void k_absmax(const float* x, int64_t n, unsigned int* out) {
  unsigned int m = 0u;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    m = max(m, __float_as_uint(fabsf(x[i])));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

template <typename P, int KIND>
mf_status launch_kind(mf_ctx* ctx, const mf_dofmap* m, const ScalarArgs<float>& a, float scale, float inv_cnorm) {
  UniformGeom ug = m->uniform ? uniform_geom(m) : UniformGeom{};
  OctGeom og = oct_geom(m);
  const int64_t nwork = m->uniform ? brick_blocks(ug.nx, ug.ny, ug.nz) : (m->n_cells + 127) / 128;
  if (nwork < 1) return MF_OK;
  if (m->uniform)
    k_scalar_h16<P, KIND, false><<<unsigned(nwork), 128, 0, ctx->stream>>>(a, ug, og, nwork, scale, inv_cnorm);
  else
    k_scalar_h16<P, KIND, true><<<unsigned(nwork), 128, 0, ctx->stream>>>(a, ug, og, nwork, scale, inv_cnorm);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

template <typename P>
mf_status launch_packed(mf_ctx* ctx, const mf_dofmap* m, int kind, const ScalarArgs<float>& a, float scale,
                        float inv_cnorm) {
  switch (kind) {
    case K_HELM: return launch_kind<P, K_HELM>(ctx, m, a, scale, inv_cnorm);
    case K_HEAT: return launch_kind<P, K_HEAT>(ctx, m, a, scale, inv_cnorm);
    case K_REINIT: return launch_kind<P, K_REINIT>(ctx, m, a, scale, inv_cnorm);
  }
  return fail(MF_EUNSUPPORTED, "16-bit applies exist for the Helmholtz, heat and reinit operators");
}

}  // namespace

// prec: PREC_F16 or PREC_BF16; coefficients tabulated, no convection.  cnorm: power of two >= every
// coefficient of the operator (mf_op::h16_cnorm).
mf_status launch_scalar_apply_h16(mf_ctx* ctx, const mf_dofmap* m, int kind, int prec, const ScalarArgs<float>& a,
                                  float scale, float cnorm) {
  MF_CUDA_TRY(upload_tables_here());
  MF_CUDA_TRY(upload_h16_tables());
  if (prec == PREC_F16) return launch_packed<__half2>(ctx, m, kind, a, scale, 1.0f / cnorm);
  return launch_packed<__nv_bfloat162>(ctx, m, kind, a, scale, 1.0f / cnorm);
}

// largest |x| over n floats (synchronising; used once per operator)
mf_status abs_max_f32(mf_ctx* ctx, const float* x, int64_t n, float* out) {
  unsigned int* d = reinterpret_cast<unsigned int*>(ctx->scratch.as<double>());
  MF_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(unsigned int), ctx->stream));
  const int64_t nb = std::min<int64_t>((n + 255) / 256, 4 * 152);
  k_absmax<<<unsigned(nb > 0 ? nb : 1), 256, 0, ctx->stream>>>(x, n, d);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  unsigned int h = 0;
  MF_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
  MF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  std::memcpy(out, &h, sizeof(float));
  return MF_OK;
}

}  // namespace mf
