// Cell-level building blocks of the sum-factorised Q2 operators (device side).
//
// A cell of edge h maps the reference cube by x = x0 + h xi.  Values at the 3^3 Gauss
// points come from three 1D sweeps with S[q][a] = l_a(g_q) (nodal Q2 basis at the Gauss
// points g = 1/2 -+ sqrt(15)/10, 1/2).  Reference gradients at the Gauss points come from
// the collocation derivative D[q][p] = lambda_p'(g_q) of the Lagrange basis through the
// Gauss points, applied along each line; the test side accumulates, in the same
// collocation space, R[q'] = JxW f(q') + sum_e D_e^T (JxW F_e / h), and three transposed
// S sweeps bring R back to the nodes.  One thread owns one cell; all 27 values, 27
// accumulators and the unrolled index arithmetic stay in registers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "df64.cuh"

namespace mf {

// 1D tables, filled once per translation unit by upload_tables().
struct Tables {
  double S[9], D[9], W[3], P[6], Sp[9], W3[27];
  double SS[9], SSp[9], SpSp[9], PP[6], PpPp[6];
  double G[3];     // Gauss points on [0, 1]
  double PW[216];  // PW[8 q + n] = Q1 basis function n at Gauss point q (n: x fastest)
  double PWW[216]; // PWW[8 q + n] = W3[q] PW[8 q + n]
};

static __constant__ double cS64[9], cD64[9], cW64[3], cP64[6], cSp64[9], cW364[27];
static __constant__ float cS32[9], cD32[9], cW32[3], cP32[6], cSp32[9], cW332[27];
static __constant__ double cSS64[9], cSSp64[9], cSpSp64[9], cPP64[6], cPpPp64[6];
static __constant__ float cSS32[9], cSSp32[9], cSpSp32[9];
static __constant__ double cPW64[216], cG64[3], cPWW64[216];
static __constant__ float cPW32[216], cPWW32[216];
// double-float copies (hi, lo) for the df64 kernels
static __constant__ float cSh[9], cSl[9], cDh[9], cDl[9], cW3h[27], cW3l[27], cPWh[216], cPWl[216];

template <typename T> struct Tb;
template <> struct Tb<double> {
  static __device__ __forceinline__ double S(int q, int a) { return cS64[3 * q + a]; }
  static __device__ __forceinline__ double D(int q, int p) { return cD64[3 * q + p]; }
  static __device__ __forceinline__ double W(int q) { return cW64[q]; }
  static __device__ __forceinline__ double W3(int q) { return cW364[q]; }
  static __device__ __forceinline__ double P(int q, int a) { return cP64[2 * q + a]; }
  static __device__ __forceinline__ double Sp(int q, int a) { return cSp64[3 * q + a]; }
  static __device__ __forceinline__ double PW(int q, int n) { return cPW64[8 * q + n]; }
  static __device__ __forceinline__ double PWW(int q, int n) { return cPWW64[8 * q + n]; }
};
template <> struct Tb<float> {
  static __device__ __forceinline__ float S(int q, int a) { return cS32[3 * q + a]; }
  static __device__ __forceinline__ float D(int q, int p) { return cD32[3 * q + p]; }
  static __device__ __forceinline__ float W(int q) { return cW32[q]; }
  static __device__ __forceinline__ float W3(int q) { return cW332[q]; }
  static __device__ __forceinline__ float P(int q, int a) { return cP32[2 * q + a]; }
  static __device__ __forceinline__ float Sp(int q, int a) { return cSp32[3 * q + a]; }
  static __device__ __forceinline__ float PW(int q, int n) { return cPW32[8 * q + n]; }
  static __device__ __forceinline__ float PWW(int q, int n) { return cPWW32[8 * q + n]; }
};

template <> struct Tb<df64> {
  static __device__ __forceinline__ df64 S(int q, int a) { return df64(cSh[3 * q + a], cSl[3 * q + a]); }
  static __device__ __forceinline__ df64 D(int q, int p) { return df64(cDh[3 * q + p], cDl[3 * q + p]); }
  static __device__ __forceinline__ df64 W3(int q) { return df64(cW3h[q], cW3l[q]); }
  static __device__ __forceinline__ df64 PW(int q, int n) { return df64(cPWh[8 * q + n], cPWl[8 * q + n]); }
};

Tables make_tables();           // host: closed forms (cellops_host.cpp)
// upload_tables_here(): per translation unit, defined by MF_DEFINE_TABLE_UPLOAD

#define MF_DEFINE_TABLE_UPLOAD                                                            \
  static cudaError_t upload_tables_here() {                                                    \
    static bool done = false;                                                             \
    if (done) return cudaSuccess;                                                         \
    Tables t = make_tables();                                                             \
    float f[216], fl[216];                                                                \
    cudaError_t e = cudaSuccess;                                                          \
    auto up64 = [&](const void* sym, const double* src, int n) {                          \
      if (e == cudaSuccess) e = cudaMemcpyToSymbol(sym, src, n * sizeof(double));         \
    };                                                                                    \
    auto up32 = [&](const void* sym, const double* src, int n) {                          \
      for (int i = 0; i < n; ++i) f[i] = float(src[i]);                                   \
      if (e == cudaSuccess) e = cudaMemcpyToSymbol(sym, f, n * sizeof(float));            \
    };                                                                                    \
    up64(cS64, t.S, 9); up64(cD64, t.D, 9); up64(cW64, t.W, 3); up64(cP64, t.P, 6);       \
    up64(cSp64, t.Sp, 9); up64(cW364, t.W3, 27);                                          \
    up64(cSS64, t.SS, 9); up64(cSSp64, t.SSp, 9); up64(cSpSp64, t.SpSp, 9);               \
    up64(cPP64, t.PP, 6); up64(cPpPp64, t.PpPp, 6); up64(cPW64, t.PW, 216); up64(cG64, t.G, 3);\
    up32(cPW32, t.PW, 216); up64(cPWW64, t.PWW, 216); up32(cPWW32, t.PWW, 216);           \
    up32(cS32, t.S, 9); up32(cD32, t.D, 9); up32(cW32, t.W, 3); up32(cP32, t.P, 6);       \
    up32(cSp32, t.Sp, 9); up32(cW332, t.W3, 27);                                          \
    up32(cSS32, t.SS, 9); up32(cSSp32, t.SSp, 9); up32(cSpSp32, t.SpSp, 9);               \
    auto updf = [&](const void* sh, const void* sl, const double* src, int n) {           \
      for (int i = 0; i < n; ++i) {                                                       \
        f[i] = float(src[i]);                                                             \
        fl[i] = float(src[i] - double(f[i]));                                             \
      }                                                                                   \
      if (e == cudaSuccess) e = cudaMemcpyToSymbol(sh, f, n * sizeof(float));             \
      if (e == cudaSuccess) e = cudaMemcpyToSymbol(sl, fl, n * sizeof(float));            \
    };                                                                                    \
    updf(cSh, cSl, t.S, 9); updf(cDh, cDl, t.D, 9); updf(cW3h, cW3l, t.W3, 27);           \
    updf(cPWh, cPWl, t.PW, 216);                                                          \
    if (e == cudaSuccess) done = true;                                                    \
    return e;                                                                             \
  }

// ------------------------------------------------------------------------ 1D sweeps
// Stride of direction DIR in the 27-array (x fastest).
template <int DIR> struct Dir { static constexpr int s = DIR == 0 ? 1 : (DIR == 1 ? 3 : 9); };
// Base index of line j (0..8) in direction DIR.
template <int DIR> __device__ __forceinline__ constexpr int line_base(int j) {
  return DIR == 0 ? 3 * j : (DIR == 1 ? (j % 3) + 9 * (j / 3) : j);
}

// Two exact properties of the 3-point Gauss rule with the Q2 nodes {0, 1/2, 1} (both point sets
// are symmetric about 1/2) shape the sweeps below: the middle Gauss point is the middle node, so
// the middle row of S is (0, 1, 0); and the derivative of the middle Lagrange polynomial through
// the Gauss points vanishes at the middle point, D[1][1] = 0.  Leaving out those terms removes a
// third of the interpolation work and a ninth of the derivative work from every cell (the fp64
// kernels are bound by the fp64 pipe, so every instruction counts).

// U[.. q ..] = sum_a S[q][a] U[.. a ..] along DIR (nodes -> Gauss points), in place.
template <typename T, int DIR> __device__ __forceinline__ void sweep_S(T* U) {
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    const int b = line_base<DIR>(j), s = Dir<DIR>::s;
    T u0 = U[b], u1 = U[b + s], u2 = U[b + 2 * s];
    U[b] = Tb<T>::S(0, 0) * u0 + Tb<T>::S(0, 1) * u1 + Tb<T>::S(0, 2) * u2;
    // middle point = middle node: U[b + s] keeps u1
    U[b + 2 * s] = Tb<T>::S(2, 0) * u0 + Tb<T>::S(2, 1) * u1 + Tb<T>::S(2, 2) * u2;
  }
}
// U[.. a ..] = sum_q S[q][a] U[.. q ..] along DIR (Gauss points -> nodes, transposed), in place.
template <typename T, int DIR> __device__ __forceinline__ void sweep_St(T* U) {
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    const int b = line_base<DIR>(j), s = Dir<DIR>::s;
    T u0 = U[b], u1 = U[b + s], u2 = U[b + 2 * s];
    U[b] = Tb<T>::S(0, 0) * u0 + Tb<T>::S(2, 0) * u2;
    U[b + s] = Tb<T>::S(0, 1) * u0 + u1 + Tb<T>::S(2, 1) * u2;
    U[b + 2 * s] = Tb<T>::S(0, 2) * u0 + Tb<T>::S(2, 2) * u2;
  }
}
template <typename T> __device__ __forceinline__ void to_qpoints(T* U) {
  sweep_S<T, 0>(U);
  sweep_S<T, 1>(U);
  sweep_S<T, 2>(U);
}
template <typename T> __device__ __forceinline__ void to_nodes(T* R) {
  sweep_St<T, 0>(R);
  sweep_St<T, 1>(R);
  sweep_St<T, 2>(R);
}

// Collocation derivative along one line at point qd (values u0, u1, u2 at the Gauss points).
template <typename T> __device__ __forceinline__ T dline(int qd, T u0, T u1, T u2) {
  if (qd == 1) return Tb<T>::D(1, 0) * u0 + Tb<T>::D(1, 2) * u2;  // D[1][1] = 0
  return Tb<T>::D(qd, 0) * u0 + Tb<T>::D(qd, 1) * u1 + Tb<T>::D(qd, 2) * u2;
}

// Reference gradient at Gauss point (qa, qb, qc) of the collocation values U.
template <typename T>
__device__ __forceinline__ void grad_at(const T* U, int qa, int qb, int qc, T& gx, T& gy, T& gz) {
  const int q = qa + 3 * qb + 9 * qc;
  const int bx = q - qa, by = q - 3 * qb, bz = q - 9 * qc;
  gx = dline<T>(qa, U[bx], U[bx + 1], U[bx + 2]);
  gy = dline<T>(qb, U[by], U[by + 3], U[by + 6]);
  gz = dline<T>(qc, U[bz], U[bz + 9], U[bz + 18]);
}
// R += D_dir^T f along direction DIR through (qa, qb, qc).
template <typename T, int DIR>
__device__ __forceinline__ void add_dir_test(T* R, int qa, int qb, int qc, T f) {
  const int q = qa + 3 * qb + 9 * qc;
  const int qd = DIR == 0 ? qa : (DIR == 1 ? qb : qc);
  const int s = Dir<DIR>::s, b = q - qd * s;
  R[b] += Tb<T>::D(qd, 0) * f;
  if (qd != 1) R[b + s] += Tb<T>::D(qd, 1) * f;  // D[1][1] = 0
  R[b + 2 * s] += Tb<T>::D(qd, 2) * f;
}
// R += D_x^T Fx + D_y^T Fy + D_z^T Fz restricted to the three lines through (qa, qb, qc).
template <typename T>
__device__ __forceinline__ void add_grad_test(T* R, int qa, int qb, int qc, T fx, T fy, T fz) {
  add_dir_test<T, 0>(R, qa, qb, qc, fx);
  add_dir_test<T, 1>(R, qa, qb, qc, fy);
  add_dir_test<T, 2>(R, qa, qb, qc, fz);
}

// ------------------------------------------------------------------------ cell addressing
// Uniform lattice of a uniform Q2 map: cell (i, j, k) has node (a, b, c) at
// (2i + a) + sx (2j + b) + sy (2k + c) with sx = 2 nx + 1, sy = sx (2 ny + 1).
struct UniformGeom {
  int nx, ny, nz;
  int64_t sx, sy;      // lattice strides
  int64_t n_dofs;
  uint32_t dir_faces;  // Dirichlet face bits
  double h;            // cell edge
};

// Bricks of 8 x 4 x 4 cells per 128-thread block (x fastest within a warp row).
__device__ __forceinline__ bool brick_cell(const UniformGeom& g, int& i, int& j, int& k, int b = -1) {
  const int nbx = (g.nx + 7) >> 3, nby = (g.ny + 3) >> 2;
  if (b < 0) b = blockIdx.x;
  int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
  int t = threadIdx.x;
  i = bx * 8 + (t & 7);
  j = by * 4 + ((t >> 3) & 3);
  k = bz * 4 + (t >> 5);
  return i < g.nx && j < g.ny && k < g.nz;
}
inline int brick_blocks(int nx, int ny, int nz) { return ((nx + 7) / 8) * ((ny + 3) / 4) * ((nz + 3) / 4); }

// 27-bit mask of the cell's local nodes on Dirichlet faces.
__device__ __forceinline__ uint32_t dirichlet_mask(const UniformGeom& g, int i, int j, int k) {
  if (!g.dir_faces) return 0u;
  uint32_t mx = ((g.dir_faces & 1u) && i == 0 ? 1u : 0u) | ((g.dir_faces & 2u) && i == g.nx - 1 ? 4u : 0u);
  uint32_t my = ((g.dir_faces & 4u) && j == 0 ? 1u : 0u) | ((g.dir_faces & 8u) && j == g.ny - 1 ? 4u : 0u);
  uint32_t mz = ((g.dir_faces & 16u) && k == 0 ? 1u : 0u) | ((g.dir_faces & 32u) && k == g.nz - 1 ? 4u : 0u);
  uint32_t m = 0;
#pragma unroll
  for (int l = 0; l < 27; ++l) {
    const int a = l % 3, b = (l / 3) % 3, c = l / 9;
    if (((mx >> a) | (my >> b) | (mz >> c)) & 1u) m |= 1u << l;
  }
  return m;
}

// Vectors are stored in Store<T>::type (df64 values live in fp64 memory).
template <typename T>
__device__ __forceinline__ void gather_uniform(const typename Store<T>::type* __restrict__ src, int64_t base,
                                               int64_t sx, int64_t sy, uint32_t dmask, T* U) {
#pragma unroll
  for (int l = 0; l < 27; ++l) {
    const int a = l % 3, b = (l / 3) % 3, c = l / 9;
    T v = from_store<T>(__ldg(src + base + a + sx * b + sy * c));
    U[l] = ((dmask >> l) & 1u) ? T(0) : v;
  }
}
template <typename T>
__device__ __forceinline__ void scatter_uniform(typename Store<T>::type* __restrict__ dst, int64_t base, int64_t sx,
                                                int64_t sy, uint32_t dmask, const T* R) {
  // Recompute the 27 addresses here instead of keeping the gather's 27 64-bit addresses
  // alive across the whole cell computation (54 registers): the empty asm hides the
  // equality of base/strides from the compiler.
  asm volatile("" : "+l"(base), "+l"(sx), "+l"(sy));
  typename Store<T>::type* __restrict__ d = dst + base;
#pragma unroll
  for (int l = 0; l < 27; ++l) {
    const int a = l % 3, b = (l / 3) % 3, c = l / 9;
    if (!((dmask >> l) & 1u)) atomicAdd(d + a + sx * b + sy * c, to_store<T>(R[l]));
  }
}

template <typename T> __device__ __forceinline__ T shfl_down_t(T v, int d) {
  return __shfl_down_sync(0xffffffffu, v, d);
}
template <> __device__ __forceinline__ df64 shfl_down_t<df64>(df64 v, int d) {
  return df64(__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d));
}

// Scatter-add of a warp of the 8 x 4 x 4 brick (lanes: 8 cells along x times 4 along y).  Cells
// that are neighbours inside the warp share a face of 9 nodes: each lane first folds its x-low
// face into the x-high face of the lane to its left, then its y-low face into the lane below,
// both by register shuffles, so a node shared inside the warp is added to memory once; only
// faces between warps (z) and bricks need atomics on more than one lane (about 14 atomics per
// cell instead of 27).  Every lane of the warp must call this; inactive lanes pass zeros.
template <typename T>
__device__ __forceinline__ void scatter_uniform_warp(typename Store<T>::type* __restrict__ dst, int64_t base,
                                                     int64_t sx, int64_t sy, uint32_t dmask, T* R, bool active) {
  const int xl = threadIdx.x & 7, yl = (threadIdx.x >> 3) & 3;
#pragma unroll
  for (int bc = 0; bc < 9; ++bc) {
    const int o = 3 * (bc % 3) + 9 * (bc / 3);
    const T w = shfl_down_t<T>(R[o], 1);
    if (xl < 7) R[o + 2] += w;
  }
#pragma unroll
  for (int ac = 0; ac < 9; ++ac) {
    const int a = ac % 3, o = a + 9 * (ac / 3);
    const T w = shfl_down_t<T>((a == 0 && xl > 0) ? T(0) : R[o], 8);
    if (yl < 3) R[o + 6] += w;
  }
  if (!active) return;
  asm volatile("" : "+l"(base), "+l"(sx), "+l"(sy));
  typename Store<T>::type* __restrict__ d = dst + base;
#pragma unroll
  for (int l = 0; l < 27; ++l) {
    const int a = l % 3, b = (l / 3) % 3, c = l / 9;
    if ((a == 0 && xl > 0) || (b == 0 && yl > 0) || ((dmask >> l) & 1u)) continue;
    atomicAdd(d + a + sx * b + sy * c, to_store<T>(R[l]));
  }
}

// Octree map: SoA cell map [27][ncp], negative entries -(1 + r) point at constraint row r.
struct OctGeom {
  const int32_t* __restrict__ cmap;
  const uint8_t* __restrict__ level;
  const int32_t* __restrict__ order;
  const int32_t* __restrict__ rowptr;
  const int32_t* __restrict__ cols;
  const double* __restrict__ w64;
  const float* __restrict__ w32;
  const uint8_t* __restrict__ dflag;  // NULL if no Dirichlet DoFs
  int64_t ncp;                        // padded cell count (SoA stride)
  int64_t ncells;
  int64_t n_dofs;
  double h0;                          // edge of a level-0 cell
};

template <typename T> __device__ __forceinline__ const typename Store<T>::type* con_w(const OctGeom& g);
template <> __device__ __forceinline__ const double* con_w<double>(const OctGeom& g) { return g.w64; }
template <> __device__ __forceinline__ const float* con_w<float>(const OctGeom& g) { return g.w32; }
template <> __device__ __forceinline__ const double* con_w<df64>(const OctGeom& g) { return g.w64; }

template <typename T, bool MASK = true>
__device__ __forceinline__ void gather_oct(const OctGeom& g, const typename Store<T>::type* __restrict__ src,
                                           int64_t cell, T* U) {
  // All 27 index loads, then all 27 value loads with no branch in between (constrained slots
  // read entry 0 and are overwritten below), so a thread keeps 27 independent loads in flight.
  int32_t id[27];
#pragma unroll
  for (int l = 0; l < 27; ++l) id[l] = __ldg(g.cmap + l * g.ncp + cell);
#pragma unroll
  for (int l = 0; l < 27; ++l) U[l] = from_store<T>(__ldg(src + (id[l] >= 0 ? id[l] : 0)));
  bool constrained = false, dirichlet = MASK && g.dflag;
#pragma unroll
  for (int l = 0; l < 27; ++l) constrained |= id[l] < 0;
  if (dirichlet) {
#pragma unroll
    for (int l = 0; l < 27; ++l)
      if (id[l] >= 0 && __ldg(g.dflag + id[l])) U[l] = T(0);
  }
  if (constrained) {
#pragma unroll
    for (int l = 0; l < 27; ++l) {
      if (id[l] >= 0) continue;
      const int r = -1 - id[l];
      const auto* w = con_w<T>(g);
      T v = T(0);
      for (int e = __ldg(g.rowptr + r); e < __ldg(g.rowptr + r + 1); ++e) {
        int32_t m = __ldg(g.cols + e);
        T um = from_store<T>(__ldg(src + m));
        if (dirichlet && __ldg(g.dflag + m)) um = T(0);
        v += from_store<T>(__ldg(w + e)) * um;
      }
      U[l] = v;
    }
  }
}
template <typename T, bool MASK = true>
__device__ __forceinline__ void scatter_oct(const OctGeom& g, typename Store<T>::type* __restrict__ dst, int64_t cell,
                                            const T* R) {
  int32_t ids[27];
#pragma unroll
  for (int l = 0; l < 27; ++l) ids[l] = __ldg(g.cmap + l * g.ncp + cell);
  bool constrained = false;
#pragma unroll
  for (int l = 0; l < 27; ++l) {
    const int32_t id = ids[l];
    constrained |= id < 0;
    if (id >= 0 && !(MASK && g.dflag && __ldg(g.dflag + id))) atomicAdd(dst + id, to_store<T>(R[l]));
  }
  if (!constrained) return;
#pragma unroll
  for (int l = 0; l < 27; ++l) {
    const int32_t id = ids[l];
    if (id >= 0) {
      continue;
    } else {
      const int r = -1 - id;
      const auto* w = con_w<T>(g);
      const typename Store<T>::type rl = to_store<T>(R[l]);
      for (int e = __ldg(g.rowptr + r); e < __ldg(g.rowptr + r + 1); ++e) {
        int32_t m = __ldg(g.cols + e);
        if (!(MASK && g.dflag && __ldg(g.dflag + m))) atomicAdd(dst + m, __ldg(w + e) * rl);
      }
    }
  }
}

}  // namespace mf
