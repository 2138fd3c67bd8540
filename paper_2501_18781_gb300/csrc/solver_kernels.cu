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

// Inner solves of the Oseen block preconditioner without host round trips: the stopping test
// of a CG and the Givens/back-substitution of a fixed-length GMRES run in one-thread kernels
// on device scalars.
__global__ void k_cg_tol_init(double* S, double tol2) {
  S[S_ACTIVE] = S[S_RR] > 0.0 ? 1.0 : 0.0;
  S[7] = tol2 * S[S_RR];
}
// steps: counts the steps that ran while the CG was still iterating (may be NULL)
__global__ void k_cg_tol_check(double* S, double* steps) {
  if (steps && S[S_ACTIVE] != 0.0) steps[0] += 1.0;
  if (S[S_RR] <= S[7] || !(S[S_PAP] > 0.0)) S[S_ACTIVE] = 0.0;
}
// the same for the nrhs systems of the batched CG (one thread each; a system already stopped by the
// host stays stopped): the threshold tol2 ||r_0||^2 into slot 7, then per iteration the step count
// and the stopping test
__global__ void k_cg_tol_init_batched(double* S, double tol2, int nrhs) {
  const int k = threadIdx.x;
  if (k >= nrhs) return;
  double* s = S + k * S_NSCAL;
  s[7] = tol2 * s[S_RR];
}
__global__ void k_cg_tol_check_batched(double* S, double* steps, int nrhs) {
  const int k = threadIdx.x;
  if (k >= nrhs) return;
  double* s = S + k * S_NSCAL;
  if (s[S_ACTIVE] == 0.0) return;
  steps[k] += 1.0;
  if (s[S_RR] <= s[7] || !(s[S_PAP] > 0.0)) s[S_ACTIVE] = 0.0;
}
// G layout (m = restart): cs[m], sn[m], g[m + 1], inv (1/norm of the newest vector), R[m][m]
__global__ void k_gmres_begin(const double* nrm2, double* G, int m) {
  const double beta = sqrt(nrm2[0]);
  double* g = G + 2 * m;
  g[0] = beta;
  for (int i = 1; i <= m; ++i) g[i] = 0.0;
  G[3 * m + 1] = beta > 0.0 ? 1.0 / beta : 0.0;
}
// h: CGS2 coefficients h[0..j] and h[m+1..m+1+j] (two passes), h[2(m+1)] = |w|^2
__global__ void k_gmres_column(const double* h, double* G, int m, int j) {
  double* cs = G;
  double* sn = G + m;
  double* g = G + 2 * m;
  double* R = G + 3 * m + 2;
  double col[64];
  for (int i = 0; i <= j; ++i) col[i] = h[i] + h[m + 1 + i];
  const double hn = sqrt(h[2 * (m + 1)]);
  col[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double den = hypot(col[j], col[j + 1]);
  cs[j] = den > 0.0 ? col[j] / den : 1.0;
  sn[j] = den > 0.0 ? col[j + 1] / den : 0.0;
  col[j] = den;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  for (int i = 0; i <= j; ++i) R[i * m + j] = col[i];
  G[3 * m + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
}
__global__ void k_gmres_solve(const double* G, int m, int j, double* y) {
  const double* g = G + 2 * m;
  const double* R = G + 3 * m + 2;
  for (int i = j - 1; i >= 0; --i) {
    double s = g[i];
    for (int k = i + 1; k < j; ++k) s -= R[i * m + k] * y[k];
    y[i] = R[i * m + i] != 0.0 ? s / R[i * m + i] : 0.0;
  }
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

mf_status dev_cg_tol_init(mf_ctx* c, double* S, double tol2) {
  k_cg_tol_init<<<1, 1, 0, c->stream>>>(S, tol2);
  LAUNCHED();
}
mf_status dev_cg_tol_check(mf_ctx* c, double* S, double* steps) {
  k_cg_tol_check<<<1, 1, 0, c->stream>>>(S, steps);
  LAUNCHED();
}
mf_status dev_cg_tol_init_batched(mf_ctx* c, double* S, double tol2, int nrhs) {
  k_cg_tol_init_batched<<<1, 64, 0, c->stream>>>(S, tol2, nrhs);
  LAUNCHED();
}
mf_status dev_cg_tol_check_batched(mf_ctx* c, double* S, double* steps, int nrhs) {
  k_cg_tol_check_batched<<<1, 64, 0, c->stream>>>(S, steps, nrhs);
  LAUNCHED();
}
mf_status dev_gmres_begin(mf_ctx* c, const double* nrm2, double* G, int m) {
  k_gmres_begin<<<1, 1, 0, c->stream>>>(nrm2, G, m);
  LAUNCHED();
}
mf_status dev_gmres_column(mf_ctx* c, const double* h, double* G, int m, int j) {
  if (m > 63) return fail(MF_EINVAL, "device GMRES: at most 63 steps");
  k_gmres_column<<<1, 1, 0, c->stream>>>(h, G, m, j);
  LAUNCHED();
}
mf_status dev_gmres_solve(mf_ctx* c, const double* G, int m, int j, double* y) {
  k_gmres_solve<<<1, 1, 0, c->stream>>>(G, m, j, y);
  LAUNCHED();
}

}  // namespace mf
