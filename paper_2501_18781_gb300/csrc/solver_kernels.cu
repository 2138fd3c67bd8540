// Small elementwise kernels used by the solvers.
#include "vec.cuh"

namespace mf {

namespace {

inline int grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  return int(g < 2432 ? (g < 1 ? 1 : g) : 2432);
}

__global__ void k_invert(double* v, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    v[i] = 1.0 / v[i];
}
__global__ void k_sqrt(const double* a, double* b, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = sqrt(a[i]);
}
template <typename T> __global__ void k_smul(const double* s, const double* v, T* out, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = T(s[i] * v[i]);
}
template <typename T> __global__ void k_smul_back(const double* s, const T* v, double* out, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = s[i] * double(v[i]);
}
__global__ void k_scale_rhs(const double* in, float* out, const double* sc, int64_t n) {
  const int64_t o = int64_t(blockIdx.y) * n;
  const double s = sc[blockIdx.y];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[o + i] = float(s * in[o + i]);
}
__global__ void k_add_scaled(const float* d, double* x, const double* sc, int64_t n) {
  const int64_t o = int64_t(blockIdx.y) * n;
  const double s = sc[blockIdx.y];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[o + i] += s * double(d[o + i]);
}

}  // namespace

#define LAUNCHED() \
  do { c->launches++; MF_CUDA_TRY(cudaGetLastError()); return MF_OK; } while (0)

mf_status dev_invert(mf_ctx* c, double* v, int64_t n) {
  k_invert<<<grid(n), 256, 0, c->stream>>>(v, n);
  LAUNCHED();
}
mf_status dev_sqrt(mf_ctx* c, const double* in, double* out, int64_t n) {
  k_sqrt<<<grid(n), 256, 0, c->stream>>>(in, out, n);
  LAUNCHED();
}
template <typename T> mf_status dev_scale_mul(mf_ctx* c, const double* s, const double* v, T* out, int64_t n) {
  k_smul<T><<<grid(n), 256, 0, c->stream>>>(s, v, out, n);
  LAUNCHED();
}
template <typename T> mf_status dev_scale_mul_back(mf_ctx* c, const double* s, const T* v, double* out, int64_t n) {
  k_smul_back<T><<<grid(n), 256, 0, c->stream>>>(s, v, out, n);
  LAUNCHED();
}
template mf_status dev_scale_mul<double>(mf_ctx*, const double*, const double*, double*, int64_t);
template mf_status dev_scale_mul<float>(mf_ctx*, const double*, const double*, float*, int64_t);
template mf_status dev_scale_mul_back<double>(mf_ctx*, const double*, const double*, double*, int64_t);
template mf_status dev_scale_mul_back<float>(mf_ctx*, const double*, const float*, double*, int64_t);

mf_status dev_scale_rhs(mf_ctx* c, const double* in, float* out, const double* scale, int64_t n, int nrhs) {
  k_scale_rhs<<<dim3(grid(n), nrhs), 256, 0, c->stream>>>(in, out, scale, n);
  LAUNCHED();
}
mf_status dev_add_scaled(mf_ctx* c, const float* d, double* x, const double* scale, int64_t n, int nrhs) {
  k_add_scaled<<<dim3(grid(n), nrhs), 256, 0, c->stream>>>(d, x, scale, n);
  LAUNCHED();
}

}  // namespace mf
