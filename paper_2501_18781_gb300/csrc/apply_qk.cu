// Q3 and Q4 Helmholtz operators (int c u v + a(phi) grad u . grad v, eq. muEff) on uniform meshes,
// sum-factorised on the CUDA cores: Gauss-Lobatto support points, (k+1)^3 Gauss points (Appendix
// B).  A cell is worked on by (k+1)^2 threads; thread (i, j) keeps the z-line through (i, j) in
// registers, contractions along z run in registers and those along x and y through shared memory.
// The coefficient a is tabulated per Gauss point in fp64 (stored fp64 and fp32, [cell][q]).
// The same kernel at k = 2 (the Gauss-Lobatto points {0, 1/2, 1} are the Q2 nodes) serves the Q2
// Helmholtz and heat operators on small uniform meshes, where one thread per cell leaves most SMs
// idle: 9 threads per cell, the Q2 Gauss-point tables read in their [q][cell] layout, Dirichlet
// nodes read as 0 and left out of the scatter.
#include <cmath>

#include "ops.h"
#include "scalar_local.cuh"

namespace mf {

UniformGeom uniform_geom(const mf_dofmap* m);

namespace {

// 1D tables of degree K (P = K + 1 support points, P Gauss points): S[q][a] = l_a(g_q),
// Sp[q][a] = l_a'(g_q), D[q][p] = lambda_p'(g_q) (Lagrange basis through the Gauss points), W[q].
__constant__ double cQS2[9], cQSp2[9], cQD2[9], cQW2[3];
__constant__ float fQS2[9], fQD2[9], fQW2[3];
__constant__ double cQS3[16], cQSp3[16], cQD3[16], cQW3[4];
__constant__ double cQS4[25], cQSp4[25], cQD4[25], cQW4[5];
__constant__ float fQS3[16], fQD3[16], fQW3[4];
__constant__ float fQS4[25], fQD4[25], fQW4[5];

template <typename T, int K> struct Qt;
template <> struct Qt<double, 2> {
  static __device__ __forceinline__ double S(int q, int a) { return cQS2[3 * q + a]; }
  static __device__ __forceinline__ double D(int q, int p) { return cQD2[3 * q + p]; }
  static __device__ __forceinline__ double W(int q) { return cQW2[q]; }
};
template <> struct Qt<float, 2> {
  static __device__ __forceinline__ float S(int q, int a) { return fQS2[3 * q + a]; }
  static __device__ __forceinline__ float D(int q, int p) { return fQD2[3 * q + p]; }
  static __device__ __forceinline__ float W(int q) { return fQW2[q]; }
};
template <> struct Qt<double, 3> {
  static __device__ __forceinline__ double S(int q, int a) { return cQS3[4 * q + a]; }
  static __device__ __forceinline__ double D(int q, int p) { return cQD3[4 * q + p]; }
  static __device__ __forceinline__ double W(int q) { return cQW3[q]; }
};
template <> struct Qt<double, 4> {
  static __device__ __forceinline__ double S(int q, int a) { return cQS4[5 * q + a]; }
  static __device__ __forceinline__ double D(int q, int p) { return cQD4[5 * q + p]; }
  static __device__ __forceinline__ double W(int q) { return cQW4[q]; }
};
template <> struct Qt<float, 3> {
  static __device__ __forceinline__ float S(int q, int a) { return fQS3[4 * q + a]; }
  static __device__ __forceinline__ float D(int q, int p) { return fQD3[4 * q + p]; }
  static __device__ __forceinline__ float W(int q) { return fQW3[q]; }
};
template <> struct Qt<float, 4> {
  static __device__ __forceinline__ float S(int q, int a) { return fQS4[5 * q + a]; }
  static __device__ __forceinline__ float D(int q, int p) { return fQD4[5 * q + p]; }
  static __device__ __forceinline__ float W(int q) { return fQW4[q]; }
};

struct Tables1D {
  double S[25], Sp[25], D[25], W[5];
};

// Gauss points and weights on [0, 1] (closed forms of the Legendre roots) and Gauss-Lobatto
// support points (the ends and the roots of P_k').
void rule(int k, double* g, double* w, double* x) {
  if (k == 2) {
    const double a = std::sqrt(3.0 / 5.0);
    const double gg[3] = {-a, 0.0, a}, ww[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
    for (int i = 0; i < 3; ++i) {
      g[i] = 0.5 * (1.0 + gg[i]);
      w[i] = 0.5 * ww[i];
    }
    const double xx[3] = {0.0, 0.5, 1.0};
    for (int i = 0; i < 3; ++i) x[i] = xx[i];
  } else if (k == 3) {
    const double a = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
    const double b = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
    const double wa = (18.0 + std::sqrt(30.0)) / 36.0, wb = (18.0 - std::sqrt(30.0)) / 36.0;
    const double gg[4] = {-b, -a, a, b}, ww[4] = {wb, wa, wa, wb};
    for (int i = 0; i < 4; ++i) {
      g[i] = 0.5 * (1.0 + gg[i]);
      w[i] = 0.5 * ww[i];
    }
    const double r = 1.0 / std::sqrt(5.0);
    const double xx[4] = {0.0, 0.5 * (1.0 - r), 0.5 * (1.0 + r), 1.0};
    for (int i = 0; i < 4; ++i) x[i] = xx[i];
  } else {
    const double a = std::sqrt(5.0 - 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
    const double b = std::sqrt(5.0 + 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
    const double wa = (322.0 + 13.0 * std::sqrt(70.0)) / 900.0, wb = (322.0 - 13.0 * std::sqrt(70.0)) / 900.0;
    const double gg[5] = {-b, -a, 0.0, a, b}, ww[5] = {wb, wa, 128.0 / 225.0, wa, wb};
    for (int i = 0; i < 5; ++i) {
      g[i] = 0.5 * (1.0 + gg[i]);
      w[i] = 0.5 * ww[i];
    }
    const double r = std::sqrt(3.0 / 7.0);
    const double xx[5] = {0.0, 0.5 * (1.0 - r), 0.5, 0.5 * (1.0 + r), 1.0};
    for (int i = 0; i < 5; ++i) x[i] = xx[i];
  }
}

// Lagrange polynomial a through the points x (n of them) and its derivative, at t
void lagrange(const double* x, int n, int a, double t, double& v, double& d) {
  v = 1.0;
  d = 0.0;
  for (int b = 0; b < n; ++b)
    if (b != a) v *= (t - x[b]) / (x[a] - x[b]);
  for (int m = 0; m < n; ++m) {
    if (m == a) continue;
    double term = 1.0 / (x[a] - x[m]);
    for (int b = 0; b < n; ++b)
      if (b != a && b != m) term *= (t - x[b]) / (x[a] - x[b]);
    d += term;
  }
}

Tables1D make_qk_tables(int k) {
  Tables1D t{};
  const int P = k + 1;
  double g[5], w[5], x[5];
  rule(k, g, w, x);
  for (int q = 0; q < P; ++q) {
    t.W[q] = w[q];
    for (int a = 0; a < P; ++a) {
      double v, d;
      lagrange(x, P, a, g[q], v, d);
      t.S[P * q + a] = v;
      t.Sp[P * q + a] = d;
      lagrange(g, P, a, g[q], v, d);
      t.D[P * q + a] = d;
    }
  }
  return t;
}

cudaError_t upload_qk_tables() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (int k = 2; k <= 4; ++k) {
    const Tables1D t = make_qk_tables(k);
    const int n = (k + 1) * (k + 1);
    float f[25];
    auto up = [&](const void* sym, const double* src, int cnt) {
      if (e == cudaSuccess) e = cudaMemcpyToSymbol(sym, src, cnt * sizeof(double));
    };
    auto upf = [&](const void* sym, const double* src, int cnt) {
      for (int i = 0; i < cnt; ++i) f[i] = float(src[i]);
      if (e == cudaSuccess) e = cudaMemcpyToSymbol(sym, f, cnt * sizeof(float));
    };
    if (k == 2) {
      up(cQS2, t.S, n); up(cQSp2, t.Sp, n); up(cQD2, t.D, n); up(cQW2, t.W, 3);
      upf(fQS2, t.S, n); upf(fQD2, t.D, n); upf(fQW2, t.W, 3);
    } else if (k == 3) {
      up(cQS3, t.S, n); up(cQSp3, t.Sp, n); up(cQD3, t.D, n); up(cQW3, t.W, 4);
      upf(fQS3, t.S, n); upf(fQD3, t.D, n); upf(fQW3, t.W, 4);
    } else {
      up(cQS4, t.S, n); up(cQSp4, t.Sp, n); up(cQD4, t.D, n); up(cQW4, t.W, 5);
      upf(fQS4, t.S, n); upf(fQD4, t.D, n); upf(fQW4, t.W, 5);
    }
  }
  if (e == cudaSuccess) done = true;
  return e;
}

template <int K> __host__ __device__ constexpr int cells_per_block() { return K == 2 ? 14 : (K == 3 ? 8 : 5); }

struct QkGeom {
  int nx, ny, nz;
  int64_t sx, sy;  // lattice strides (K n + 1 per axis)
  int64_t ncells;
  double h;
  int64_t cq, cc;  // coefficient of Gauss point q of a cell at coef[q cq + cell cc]
  uint32_t dir;    // Dirichlet faces (bits x-, x+, y-, y+, z-, z+): their nodes read as 0, get no update
};

// Cell and in-cell thread coordinates of this thread and the Dirichlet nodes of its z-line (bit z);
// false for the idle tail of the block.
template <int K>
__device__ __forceinline__ bool qk_thread(const QkGeom& g, int& slot, int& i, int& j, int64_t& cell, int64_t& base,
                                          uint32_t& zdir) {
  constexpr int P = K + 1, CPB = cells_per_block<K>();
  const int t = threadIdx.x;
  slot = t / (P * P);
  const int r = t % (P * P);
  i = r % P;
  j = r / P;
  zdir = 0u;
  if (slot >= CPB) return false;
  cell = int64_t(blockIdx.x) * CPB + slot;
  if (cell >= g.ncells) return false;
  const int64_t cx = cell % g.nx, cy = (cell / g.nx) % g.ny, cz = cell / (int64_t(g.nx) * g.ny);
  base = K * cx + i + g.sx * (K * cy + j) + g.sy * (K * cz);
  if (g.dir) {
    const bool side = ((g.dir & 1u) && cx == 0 && i == 0) || ((g.dir & 2u) && cx == g.nx - 1 && i == K) ||
                      ((g.dir & 4u) && cy == 0 && j == 0) || ((g.dir & 8u) && cy == g.ny - 1 && j == K);
    zdir = side ? (1u << P) - 1u : 0u;
    if ((g.dir & 16u) && cz == 0) zdir |= 1u;
    if ((g.dir & 32u) && cz == g.nz - 1) zdir |= 1u << K;
  }
  return true;
}

// dst += A src for one cell per (K+1)^2 threads.  coef[cell * Q^3 + q] = a at Gauss point q
// (x fastest), mass = c.
template <typename T, int K>
__global__ void __launch_bounds__(128) k_helmholtz_qk(QkGeom g, const T* __restrict__ src, T* __restrict__ dst,
                                                      const T* __restrict__ coef, T mass) {
  constexpr int P = K + 1, P2 = P * P, P3 = P2 * P, CPB = cells_per_block<K>();
  __shared__ T s0[CPB][P3], s1[CPB][P3], s2[CPB][P3];
  int slot, i, j;
  int64_t cell = 0, base = 0;
  uint32_t zdir;
  const bool on = qk_thread<K>(g, slot, i, j, cell, base, zdir);
  const int sl = slot < CPB ? slot : 0;
  T r[P], v[P];
  // nodes -> Gauss points: z in registers, then y and x through shared memory
#pragma unroll
  for (int z = 0; z < P; ++z) r[z] = (on && !((zdir >> z) & 1u)) ? __ldg(src + base + g.sy * z) : T(0);
#pragma unroll
  for (int q = 0; q < P; ++q) {
    T s = T(0);
#pragma unroll
    for (int z = 0; z < P; ++z) s += Qt<T, K>::S(q, z) * r[z];
    v[q] = s;
  }
  if (slot < CPB)
#pragma unroll
    for (int q = 0; q < P; ++q) s0[sl][q * P2 + j * P + i] = v[q];
  __syncthreads();
  if (slot < CPB)
#pragma unroll
    for (int qz = 0; qz < P; ++qz) {
      T s = T(0);
#pragma unroll
      for (int b = 0; b < P; ++b) s += Qt<T, K>::S(j, b) * s0[sl][qz * P2 + b * P + i];
      s1[sl][qz * P2 + j * P + i] = s;  // (qx = node i, qy = j)
    }
  __syncthreads();
  T U[P];
  if (slot < CPB)
#pragma unroll
    for (int qz = 0; qz < P; ++qz) {
      T s = T(0);
#pragma unroll
      for (int a = 0; a < P; ++a) s += Qt<T, K>::S(i, a) * s1[sl][qz * P2 + j * P + a];
      U[qz] = s;  // value at Gauss point (qx = i, qy = j, qz)
      s2[sl][qz * P2 + j * P + i] = s;
    }
  __syncthreads();
  // gradients by collocation, pointwise coefficient, test-side fluxes
  const T h = T(g.h), h3 = h * h * h;
  T Fz[P], R[P];
  if (slot < CPB)
#pragma unroll
    for (int qz = 0; qz < P; ++qz) {
      T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        gx += Qt<T, K>::D(i, p) * s2[sl][qz * P2 + j * P + p];
        gy += Qt<T, K>::D(j, p) * s2[sl][qz * P2 + p * P + i];
        gz += Qt<T, K>::D(qz, p) * U[p];
      }
      const int q = i + P * (j + P * qz);
      const T w = Qt<T, K>::W(i) * Qt<T, K>::W(j) * Qt<T, K>::W(qz);
      const T a = on ? coef[q * g.cq + cell * g.cc] : T(0);
      const T c = w * a * h;
      R[qz] = w * mass * h3 * U[qz];
      Fz[qz] = c * gz;
      s0[sl][qz * P2 + j * P + i] = c * gx;  // Fx
      s1[sl][qz * P2 + j * P + i] = c * gy;  // Fy
    }
  __syncthreads();
  if (slot < CPB)
#pragma unroll
    for (int qz = 0; qz < P; ++qz) {
      T s = R[qz];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        s += Qt<T, K>::D(p, i) * s0[sl][qz * P2 + j * P + p];
        s += Qt<T, K>::D(p, j) * s1[sl][qz * P2 + p * P + i];
        s += Qt<T, K>::D(p, qz) * Fz[p];
      }
      s2[sl][qz * P2 + j * P + i] = s;  // R at (qx = i, qy = j, qz)
    }
  __syncthreads();
  // Gauss points -> nodes: x, then y through shared memory, then z in registers
  if (slot < CPB)
#pragma unroll
    for (int qz = 0; qz < P; ++qz) {
      T s = T(0);
#pragma unroll
      for (int q = 0; q < P; ++q) s += Qt<T, K>::S(q, i) * s2[sl][qz * P2 + j * P + q];
      s0[sl][qz * P2 + j * P + i] = s;  // (node a = i, qy = j)
    }
  __syncthreads();
  if (slot < CPB)
#pragma unroll
    for (int qz = 0; qz < P; ++qz) {
      T s = T(0);
#pragma unroll
      for (int q = 0; q < P; ++q) s += Qt<T, K>::S(q, j) * s0[sl][qz * P2 + q * P + i];
      v[qz] = s;  // (a = i, b = j, qz)
    }
  if (!on) return;
#pragma unroll
  for (int z = 0; z < P; ++z) {
    T s = T(0);
#pragma unroll
    for (int q = 0; q < P; ++q) s += Qt<T, K>::S(q, z) * v[q];
    if (!((zdir >> z) & 1u)) atomicAdd(dst + base + g.sy * z, s);
  }
}

// a = a_g + (a_l - a_g) H(phi_h) at the Gauss points from the nodal phi, fp64, one cell per thread
template <int K>
__global__ void k_qk_coef(QkGeom g, const double* phi, double a_l, double a_g, int hv, double eps, double* c64,
                          float* c32) {
  constexpr int P = K + 1, P3 = P * P * P;
  const int64_t cell = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (cell >= g.ncells) return;
  const int64_t cx = cell % g.nx, cy = (cell / g.nx) % g.ny, cz = cell / (int64_t(g.nx) * g.ny);
  const int64_t base = K * cx + g.sx * (K * cy) + g.sy * (K * cz);
  double u[P3], t[P3];
  for (int c = 0; c < P; ++c)
    for (int b = 0; b < P; ++b)
      for (int a = 0; a < P; ++a) u[a + P * (b + P * c)] = phi[base + a + g.sx * b + g.sy * c];
  // x, y, z sweeps (nodes -> Gauss points)
  for (int c = 0; c < P; ++c)
    for (int b = 0; b < P; ++b)
      for (int q = 0; q < P; ++q) {
        double s = 0.0;
        for (int a = 0; a < P; ++a) s += Qt<double, K>::S(q, a) * u[a + P * (b + P * c)];
        t[q + P * (b + P * c)] = s;
      }
  for (int c = 0; c < P; ++c)
    for (int q = 0; q < P; ++q)
      for (int a = 0; a < P; ++a) {
        double s = 0.0;
        for (int b = 0; b < P; ++b) s += Qt<double, K>::S(q, b) * t[a + P * (b + P * c)];
        u[a + P * (q + P * c)] = s;
      }
  for (int q = 0; q < P; ++q)
    for (int b = 0; b < P; ++b)
      for (int a = 0; a < P; ++a) {
        double s = 0.0;
        for (int c = 0; c < P; ++c) s += Qt<double, K>::S(q, c) * u[a + P * (b + P * c)];
        t[a + P * (b + P * q)] = s;
      }
  for (int q = 0; q < P3; ++q) {
    const double a = a_g + (a_l - a_g) * heaviside<double>(t[q], hv, eps);
    c64[cell * P3 + q] = a;
    c32[cell * P3 + q] = float(a);
  }
}

// diagonal: diag_l += sum_q w_q (c h^3 N_l(q)^2 + a_q h |grad_ref N_l(q)|^2), one (cell, l) per thread
template <int K>
__global__ void k_qk_diag(QkGeom g, const double* coef, double mass, double* diag) {
  constexpr int P = K + 1, P3 = P * P * P;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= g.ncells * P3) return;
  const int64_t cell = t / P3;
  const int l = int(t % P3), la = l % P, lb = (l / P) % P, lc = l / (P * P);
  const double* S = K == 3 ? cQS3 : cQS4;
  const double* Sp = K == 3 ? cQSp3 : cQSp4;
  const double* W = K == 3 ? cQW3 : cQW4;
  const double h = g.h;
  double acc = 0.0;
  for (int qc = 0; qc < P; ++qc)
    for (int qb = 0; qb < P; ++qb)
      for (int qa = 0; qa < P; ++qa) {
        const double sa = S[P * qa + la], sb = S[P * qb + lb], sc = S[P * qc + lc];
        const double gx = Sp[P * qa + la] * sb * sc, gy = sa * Sp[P * qb + lb] * sc, gz = sa * sb * Sp[P * qc + lc];
        const double n = sa * sb * sc;
        const double w = W[qa] * W[qb] * W[qc];
        const double a = coef[cell * P3 + qa + P * (qb + P * qc)];
        acc += w * (mass * h * h * h * n * n + a * h * (gx * gx + gy * gy + gz * gz));
      }
  const int64_t cx = cell % g.nx, cy = (cell / g.nx) % g.ny, cz = cell / (int64_t(g.nx) * g.ny);
  atomicAdd(diag + (K * cx + la) + g.sx * (K * cy + lb) + g.sy * (K * cz + lc), acc);
}

}  // namespace

// host copies of the degree-k 1D tables (S, Sp: (k+1) x (k+1), W: k+1)
void qk_host_tables(int k, double* S, double* Sp, double* W) {
  const Tables1D t = make_qk_tables(k);
  const int n = (k + 1) * (k + 1);
  for (int i = 0; i < n; ++i) {
    S[i] = t.S[i];
    Sp[i] = t.Sp[i];
  }
  for (int i = 0; i <= k; ++i) W[i] = t.W[i];
}

namespace {

QkGeom qk_geom(const mf_dofmap* m) {
  QkGeom g{};
  g.nx = m->mesh->n[0];
  g.ny = m->mesh->n[1];
  g.nz = m->mesh->n[2];
  g.sx = m->R[0] + 1;
  g.sy = g.sx * (m->R[1] + 1);
  g.ncells = m->n_cells;
  g.h = m->mesh->h0;
  g.cq = 1;
  g.cc = int64_t(m->degree + 1) * (m->degree + 1) * (m->degree + 1);
  g.dir = 0u;
  return g;
}

}  // namespace

mf_status launch_qk_coef(mf_ctx* ctx, const mf_dofmap* m, const double* phi, double a_l, double a_g, int hv,
                         double eps, double* c64, float* c32) {
  MF_CUDA_TRY(upload_qk_tables());
  const QkGeom g = qk_geom(m);
  const int nb = int((g.ncells + 127) / 128);
  if (m->degree == 3)
    k_qk_coef<3><<<nb, 128, 0, ctx->stream>>>(g, phi, a_l, a_g, hv, eps, c64, c32);
  else
    k_qk_coef<4><<<nb, 128, 0, ctx->stream>>>(g, phi, a_l, a_g, hv, eps, c64, c32);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

template <typename T>
mf_status launch_helmholtz_qk(mf_ctx* ctx, const mf_dofmap* m, const T* src, T* dst, const T* coef, double mass) {
  MF_CUDA_TRY(upload_qk_tables());
  const QkGeom g = qk_geom(m);
  if (m->degree == 3) {
    const int nb = int((g.ncells + cells_per_block<3>() - 1) / cells_per_block<3>());
    k_helmholtz_qk<T, 3><<<nb, 128, 0, ctx->stream>>>(g, src, dst, coef, T(mass));
  } else {
    const int nb = int((g.ncells + cells_per_block<4>() - 1) / cells_per_block<4>());
    k_helmholtz_qk<T, 4><<<nb, 128, 0, ctx->stream>>>(g, src, dst, coef, T(mass));
  }
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}
template mf_status launch_helmholtz_qk<double>(mf_ctx*, const mf_dofmap*, const double*, double*, const double*,
                                               double);
template mf_status launch_helmholtz_qk<float>(mf_ctx*, const mf_dofmap*, const float*, float*, const float*, double);

template <typename T>
mf_status launch_q2_line(mf_ctx* ctx, const mf_dofmap* m, const T* src, T* dst, const T* coef, double mass) {
  if (m->degree != 2 || !m->uniform) return fail(MF_EINVAL, "the line kernel takes uniform Q2 maps");
  MF_CUDA_TRY(upload_qk_tables());
  QkGeom g = qk_geom(m);
  g.cq = m->n_cells;   // the Q2 Gauss-point tables are [q][cell]
  g.cc = 1;
  g.dir = m->dirichlet_faces;
  const int nb = int((g.ncells + cells_per_block<2>() - 1) / cells_per_block<2>());
  k_helmholtz_qk<T, 2><<<nb, 128, 0, ctx->stream>>>(g, src, dst, coef, T(mass));
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}
template mf_status launch_q2_line<double>(mf_ctx*, const mf_dofmap*, const double*, double*, const double*, double);
template mf_status launch_q2_line<float>(mf_ctx*, const mf_dofmap*, const float*, float*, const float*, double);

mf_status launch_qk_diag(mf_ctx* ctx, const mf_dofmap* m, const double* coef, double mass, double* diag) {
  MF_CUDA_TRY(upload_qk_tables());
  const QkGeom g = qk_geom(m);
  MF_CUDA_TRY(cudaMemsetAsync(diag, 0, sizeof(double) * m->n_dofs, ctx->stream));
  const int64_t P3 = int64_t(m->degree + 1) * (m->degree + 1) * (m->degree + 1);
  const int nb = int((g.ncells * P3 + 255) / 256);
  if (m->degree == 3)
    k_qk_diag<3><<<nb, 256, 0, ctx->stream>>>(g, coef, mass, diag);
  else
    k_qk_diag<4><<<nb, 256, 0, ctx->stream>>>(g, coef, mass, diag);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

}  // namespace mf
