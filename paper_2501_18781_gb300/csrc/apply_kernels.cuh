// Matrix-free operator apply kernels: gather -> values/gradients at Gauss points -> pointwise
// physics -> integrate -> scatter-add (one thread per Q2 cell, registers only).  Included by one
// translation unit per arithmetic (apply_f64.cu, apply_f32.cu, apply_df64.cu) so that the three
// instantiations compile in parallel.
#pragma once
#include <algorithm>
#include <type_traits>

#include "scalar_local.cuh"

namespace mf {

MF_DEFINE_TABLE_UPLOAD

UniformGeom uniform_geom(const mf_dofmap* m);
OctGeom oct_geom(const mf_dofmap* m);

namespace {

struct CellLoc {
  int64_t cell;
  int64_t base;
  uint32_t dmask;
  double h;
};

// Work unit w: the w-th slot of blockDim.x cells of the (sorted) octree cell list, or the
// w-th 8 x 4 x 4 brick of a uniform mesh; the thread's cell within it.
template <bool OCT>
__device__ __forceinline__ bool locate(const UniformGeom& ug, const OctGeom& og, int64_t w, CellLoc& L) {
  if (OCT) {
    const int64_t t = w * blockDim.x + threadIdx.x;
    if (t >= og.ncells) return false;
    L.cell = __ldg(og.order + t);
    L.h = og.h0 / double(1 << __ldg(og.level + L.cell));
    L.base = 0;
    L.dmask = 0;
    return true;
  } else {
    int i, j, k;
    if (!brick_cell(ug, i, j, k, int(w))) return false;
    L.cell = i + int64_t(ug.nx) * (j + int64_t(ug.ny) * k);
    L.base = 2 * int64_t(i) + ug.sx * (2 * int64_t(j)) + ug.sy * (2 * int64_t(k));
    L.dmask = dirichlet_mask(ug, i, j, k);
    L.h = ug.h;
    return true;
  }
}

template <typename T, bool OCT, bool MASK = true>
__device__ __forceinline__ void gather(const UniformGeom& ug, const OctGeom& og, const CellLoc& L,
                                       const typename Store<T>::type* src, T* U) {
  if (OCT) gather_oct<T, MASK>(og, src, L.cell, U);
  else gather_uniform<T>(src, L.base, ug.sx, ug.sy, L.dmask, U);
}
template <typename T, bool OCT, bool MASK = true>
__device__ __forceinline__ void scatter(const UniformGeom& ug, const OctGeom& og, const CellLoc& L,
                                        typename Store<T>::type* dst, const T* R) {
  if (OCT) scatter_oct<T, MASK>(og, dst, L.cell, R);
  else scatter_uniform<T>(dst, L.base, ug.sx, ug.sy, L.dmask, R);
}

// Scalar operators.  KIND: K_HELM, K_HEAT, K_REINIT, K_MASS; MODE 0 = coefficients from the
// nodal field in the kernel, 1 = tabulated per Gauss point.
template <typename T, int KIND, int MODE, bool BETA, bool TR, bool OCT>
__device__ __forceinline__ void scalar_cell(const ScalarArgs<typename Store<T>::type>& A, const UniformGeom& ug,
                                            const OctGeom& og, CellLoc L, bool active) {
  // On uniform meshes all 32 lanes of a warp take part in the warp-level scatter: a lane
  // without a cell (active = false) stays and contributes zeros; a lane whose cell is in the
  // mesh but outside the objective box (compute = false) contributes zeros but still writes the
  // nodes it owns, which may hold its neighbours' folded contributions.
  if (KIND == K_MASS) L.dmask = 0u;  // the plain mass matrix has no Dirichlet rows
  const T h = T(OCT ? L.h : ug.h);
  // every term carries at least one power of h: R = h * (...), with
  // w h^3 m u = h (w (m h^2) u), w h k g = h (w k g), w h^2 beta.g = h (w h beta.g)
  const T mh2 = T(A.mass) * h * h;
  bool compute = active;
  if (KIND == K_MASS && A.use_box && active) {
    // centre of a uniform cell from its lattice base
    const int64_t kk = L.base / ug.sy, jj = (L.base % ug.sy) / ug.sx, ii = L.base % ug.sx;
    const double cx = A.lo[0] + (double(ii) * 0.5 + 0.5) * L.h, cy = A.lo[1] + (double(jj) * 0.5 + 0.5) * L.h,
                 cz = A.lo[2] + (double(kk) * 0.5 + 0.5) * L.h;
    if (!(fabs(cx) <= A.box_half && fabs(cy) <= A.box_half && cz >= A.box_zmin)) compute = false;
  }
  if constexpr (OCT) {
    if (!compute) return;
  }
  // scalar coefficient (or phi for in-kernel reinit) at the 27 Gauss points
  T C[27];
  if (compute)
  if constexpr (KIND == K_HELM || KIND == K_HEAT || KIND == K_REINIT) {
    if constexpr (MODE == 0) {
      gather<T, OCT, false>(ug, og, CellLoc{L.cell, L.base, 0u, L.h}, A.field, C);
      to_qpoints<T>(C);
      if constexpr (KIND == K_HELM) {
#pragma unroll
        for (int q = 0; q < 27; ++q) C[q] = A.a_g + (A.a_l - A.a_g) * heaviside<T>(C[q], A.heaviside, A.eps);
      } else if constexpr (KIND == K_HEAT) {
#pragma unroll
        for (int q = 0; q < 27; ++q) C[q] = A.k0 + A.k_slope * C[q];
      }
    } else if constexpr (KIND != K_REINIT) {
#pragma unroll
      for (int q = 0; q < 27; ++q) C[q] = from_store<T>(__ldg(A.qcoef + q * A.ncp + L.cell));
    }
  }
  for (int r = 0; r < A.nrhs; ++r) {
    T U[27], R[27];
    if (compute) {
      gather<T, OCT, KIND != K_MASS>(ug, og, L, A.src + r * A.ld, U);
      scalar_local<T, KIND, MODE, BETA, TR>(A, L.cell, h, mh2, C, U, R);
    } else {
#pragma unroll
      for (int q = 0; q < 27; ++q) R[q] = T(0);
    }
    if constexpr (OCT) scatter_oct<T, KIND != K_MASS>(og, A.dst + r * A.ld, L.cell, R);
    else scatter_uniform_warp<T>(A.dst + r * A.ld, L.base, ug.sx, ug.sy, L.dmask, R, active);
  }
}

// One launch sweeps all nwork work units; with fewer blocks than units (the persistent
// variant, grid = a few blocks per SM) each block strides over them.  All right-hand sides of
// a cell are applied while its coefficients sit in registers.  Two fp32 instances are held to five
// blocks of 128 per SM (96 registers): the octree reinitialisation (no spills; its indirect gathers are
// latency-bound, and 20 warps per SM instead of 16 measured 2.41 -> 2.32 ms for the 8-RHS base-32
// octree apply) and the uniform heat operator without convection (48 bytes of spills; 128^3 apply
// 0.168 -> 0.161 ms).  The other instances would spill more at that bound.
template <typename T, int KIND, int MODE, bool BETA, bool TR, bool OCT>
__global__ void __launch_bounds__(128, (sizeof(T) == 4 && ((OCT && KIND == K_REINIT) ||
                                                           (!OCT && KIND == K_HEAT && !BETA))) ? 5 : 1)
    k_scalar(ScalarArgs<typename Store<T>::type> A, UniformGeom ug, OctGeom og,
                                                int64_t nwork) {
  for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
    CellLoc L;
    const bool active = locate<OCT>(ug, og, w, L);
    if (OCT && !active) continue;
    scalar_cell<T, KIND, MODE, BETA, TR, OCT>(A, ug, og, L, active);
  }
}

// Oseen operator, Q2 velocity / Q1 pressure on a uniform mesh, coefficients tabulated.
// Pw[q][abc] = P[qa][a] P[qb][b] P[qc][c] (Q1 basis at the Gauss points).
template <typename T> __device__ __forceinline__ T q1w(int q, int n) { return Tb<T>::PW(q, n); }

template <typename T>
__global__ void __launch_bounds__(128, 1) k_oseen(OseenArgs<typename Store<T>::type> A, UniformGeom ug) {
  using St = typename Store<T>::type;
  int i, j, k;
  if (!brick_cell(ug, i, j, k)) return;
  const int64_t cell = i + int64_t(ug.nx) * (j + int64_t(ug.ny) * k);
  const int64_t nc = int64_t(ug.nx) * ug.ny * ug.nz;
  const int64_t base = 2 * int64_t(i) + ug.sx * (2 * int64_t(j)) + ug.sy * (2 * int64_t(k));
  const uint32_t dmask = dirichlet_mask(ug, i, j, k);
  const int64_t px = ug.nx + 1, pxy = px * (ug.ny + 1);
  const int64_t pbase = i + px * (j + (ug.ny + 1) * int64_t(k));
  // every term carries a factor h (applied once before the scatter): w h^3 sigma rho u =
  // h (w rho (sigma h^2) u), w h^2 rho beta.g = h (w rho (h beta.g)), w h mu g = h (w mu g)
  const T h = T(ug.h), sh2 = T(A.sigma) * h * h;
  const St* __restrict__ psrc = A.src + 3 * A.nu;

  T R0[27], R1[27], R2[27];
  {
    T Pn[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) Pn[n] = from_store<T>(__ldg(psrc + pbase + (n & 1) + px * ((n >> 1) & 1) + pxy * (n >> 2)));
#pragma unroll
    for (int q = 0; q < 27; ++q) { R0[q] = T(0); R1[q] = T(0); R2[q] = T(0); }
#pragma unroll
    for (int qc = 0; qc < 3; ++qc)
#pragma unroll
      for (int qb = 0; qb < 3; ++qb)
#pragma unroll
        for (int qa = 0; qa < 3; ++qa) {
          const int q = qa + 3 * qb + 9 * qc;
          T pq = T(0);
#pragma unroll
          for (int n = 0; n < 8; ++n) pq += q1w<T>(q, n) * Pn[n];
          const T s = Tb<T>::W3(q) * (-h * pq);   // -int p div v
          add_dir_test<T, 0>(R0, qa, qb, qc, s);
          add_dir_test<T, 1>(R1, qa, qb, qc, s);
          add_dir_test<T, 2>(R2, qa, qb, qc, s);
        }
  }
  T Rp[8];
#pragma unroll
  for (int n = 0; n < 8; ++n) Rp[n] = T(0);

#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    T U[27];
    gather_uniform<T>(A.src + d * A.nu, base, ug.sx, ug.sy, dmask, U);
    to_qpoints<T>(U);
#pragma unroll
    for (int qc = 0; qc < 3; ++qc)
#pragma unroll
      for (int qb = 0; qb < 3; ++qb)
#pragma unroll
        for (int qa = 0; qa < 3; ++qa) {
          const int q = qa + 3 * qb + 9 * qc;
          const T w = Tb<T>::W3(q);
          T gx, gy, gz;
          grad_at<T>(U, qa, qb, qc, gx, gy, gz);
          const T rho = from_store<T>(__ldg(A.rho + q * nc + cell));
          const T mu = from_store<T>(__ldg(A.mu + q * nc + cell));
          const T bx = from_store<T>(__ldg(A.beta + (0 * 27 + q) * nc + cell));
          const T by = from_store<T>(__ldg(A.beta + (1 * 27 + q) * nc + cell));
          const T bz = from_store<T>(__ldg(A.beta + (2 * 27 + q) * nc + cell));
          const T fv = w * (rho * (sh2 * U[q] + h * (bx * gx + by * gy + bz * gz)));
          const T c1 = w * mu;
          const T cx = c1 * gx, cy = c1 * gy, cz = c1 * gz;
          const T gd = d == 0 ? gx : (d == 1 ? gy : gz);
          // 2 mu eps(u):eps(v) = mu (grad u_d . grad v_d + d_c u_d d_d v_c), trial component d
          if (d == 0) {
            R0[q] += fv;
            add_grad_test<T>(R0, qa, qb, qc, cx, cy, cz);
            add_dir_test<T, 0>(R0, qa, qb, qc, cx);
            add_dir_test<T, 0>(R1, qa, qb, qc, cy);
            add_dir_test<T, 0>(R2, qa, qb, qc, cz);
          } else if (d == 1) {
            R1[q] += fv;
            add_grad_test<T>(R1, qa, qb, qc, cx, cy, cz);
            add_dir_test<T, 1>(R0, qa, qb, qc, cx);
            add_dir_test<T, 1>(R1, qa, qb, qc, cy);
            add_dir_test<T, 1>(R2, qa, qb, qc, cz);
          } else {
            R2[q] += fv;
            add_grad_test<T>(R2, qa, qb, qc, cx, cy, cz);
            add_dir_test<T, 2>(R0, qa, qb, qc, cx);
            add_dir_test<T, 2>(R1, qa, qb, qc, cy);
            add_dir_test<T, 2>(R2, qa, qb, qc, cz);
          }
          const T s = w * (-h * gd);  // -int q div u
#pragma unroll
          for (int n = 0; n < 8; ++n) Rp[n] += q1w<T>(q, n) * s;
        }
  }
#pragma unroll
  for (int q = 0; q < 27; ++q) { R0[q] *= h; R1[q] *= h; R2[q] *= h; }
  to_nodes<T>(R0);
  scatter_uniform<T>(A.dst, base, ug.sx, ug.sy, dmask, R0);
  to_nodes<T>(R1);
  scatter_uniform<T>(A.dst + A.nu, base, ug.sx, ug.sy, dmask, R1);
  to_nodes<T>(R2);
  scatter_uniform<T>(A.dst + 2 * A.nu, base, ug.sx, ug.sy, dmask, R2);
  St* pdst = A.dst + 3 * A.nu;
#pragma unroll
  for (int n = 0; n < 8; ++n)
    atomicAdd(pdst + pbase + (n & 1) + px * ((n >> 1) & 1) + pxy * (n >> 2), to_store<T>(h * Rp[n]));
}

// The same Oseen cell operator with the Gauss-point loop outside: all three velocity
// components sit in registers at once (81 values + 81 accumulators), so each Gauss point's
// rho, mu and beta are read once instead of once per component.  Fits the fp32 register file.
// EXT adds the melt-pool terms: the Darcy coefficient kd (a mass-like term kd u . v) and the
// trace correction -2 mu tr(eps(u)) n n of the viscous stress, both read per Gauss point.
template <typename T, bool EXT = false>
__global__ void __launch_bounds__(128) k_oseen_qouter(OseenArgs<typename Store<T>::type> A, UniformGeom ug) {
  using St = typename Store<T>::type;
  int i, j, k;
  if (!brick_cell(ug, i, j, k)) return;
  const int64_t cell = i + int64_t(ug.nx) * (j + int64_t(ug.ny) * k);
  const int64_t nc = int64_t(ug.nx) * ug.ny * ug.nz;
  const int64_t base = 2 * int64_t(i) + ug.sx * (2 * int64_t(j)) + ug.sy * (2 * int64_t(k));
  const uint32_t dmask = dirichlet_mask(ug, i, j, k);
  const int64_t px = ug.nx + 1, pxy = px * (ug.ny + 1);
  const int64_t pbase = i + px * (j + (ug.ny + 1) * int64_t(k));
  const T h = T(ug.h), mh2 = -(h * h);
  if constexpr (sizeof(T) == 4) {
    // L2 prefetch of the Gauss-point coefficient rows cm, cv and cb while the inputs load: a brick
    // row's 8 cells share one 32-byte sector per table row, so each lane fetches that sector for its
    // brick row and every 8th of the 135 rows
    const int64_t row_cell = cell - (threadIdx.x & 7);
#pragma unroll 1
    for (int r = threadIdx.x & 7; r < 135; r += 8) {
      const St* t = r < 27 ? A.cm + r * nc : (r < 54 ? A.cv + (r - 27) * nc : A.cb + (r - 54) * nc);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(t + row_cell));
    }
  }
  T U0[27], U1[27], U2[27];
  gather_uniform<T>(A.src, base, ug.sx, ug.sy, dmask, U0);
  gather_uniform<T>(A.src + A.nu, base, ug.sx, ug.sy, dmask, U1);
  gather_uniform<T>(A.src + 2 * A.nu, base, ug.sx, ug.sy, dmask, U2);
  to_qpoints<T>(U0);
  to_qpoints<T>(U1);
  to_qpoints<T>(U2);
  // nodal pressure times -h^2: the pressure test term -w h^3 p div v = (w psi . (-h^2 p)) g_ref(v)
  T Pn[8];
  const St* __restrict__ psrc = A.src + 3 * A.nu;
#pragma unroll
  for (int n = 0; n < 8; ++n)
    Pn[n] = mh2 * from_store<T>(__ldg(psrc + pbase + (n & 1) + px * ((n >> 1) & 1) + pxy * (n >> 2)));
  T R0[27], R1[27], R2[27], Rp[8];
#pragma unroll
  for (int q = 0; q < 27; ++q) { R0[q] = T(0); R1[q] = T(0); R2[q] = T(0); }
#pragma unroll
  for (int n = 0; n < 8; ++n) Rp[n] = T(0);
#pragma unroll
  for (int qc = 0; qc < 3; ++qc)
#pragma unroll
    for (int qb = 0; qb < 3; ++qb)
#pragma unroll
      for (int qa = 0; qa < 3; ++qa) {
        const int q = qa + 3 * qb + 9 * qc;
        // Gauss-point coefficients with weight and powers of h folded in (tabulated once per
        // operator): cm = w h^3 (sigma rho [+ Darcy]), cv = w h mu, (bx, by, bz) = w h^2 rho beta
        const T cm = from_store<T>(__ldg(A.cm + q * nc + cell));
        const T cv = from_store<T>(__ldg(A.cv + q * nc + cell));
        const T bx = from_store<T>(__ldg(A.cb + (0 * 27 + q) * nc + cell));
        const T by = from_store<T>(__ldg(A.cb + (1 * 27 + q) * nc + cell));
        const T bz = from_store<T>(__ldg(A.cb + (2 * 27 + q) * nc + cell));
        T pw = T(0);
#pragma unroll
        for (int n = 0; n < 8; ++n) pw += Tb<T>::PWW(q, n) * Pn[n];
        T g[3][3];  // g[d][e] = d u_d / d x_e (reference)
        grad_at<T>(U0, qa, qb, qc, g[0][0], g[0][1], g[0][2]);
        grad_at<T>(U1, qa, qb, qc, g[1][0], g[1][1], g[1][2]);
        grad_at<T>(U2, qa, qb, qc, g[2][0], g[2][1], g[2][2]);
        // value test: sigma rho u_d + rho beta . grad u_d, accumulated by multiply-adds only
        R0[q] = fma(bz, g[0][2], fma(by, g[0][1], fma(bx, g[0][0], fma(cm, U0[q], R0[q]))));
        R1[q] = fma(bz, g[1][2], fma(by, g[1][1], fma(bx, g[1][0], fma(cm, U1[q], R1[q]))));
        R2[q] = fma(bz, g[2][2], fma(by, g[2][1], fma(bx, g[2][0], fma(cm, U2[q], R2[q]))));
        // gradient test: mu (grad u + grad u^T) - p I
        const T cv2 = cv + cv;
        T s00 = fma(cv2, g[0][0], pw), s11 = fma(cv2, g[1][1], pw), s22 = fma(cv2, g[2][2], pw);
        T s01 = cv * (g[0][1] + g[1][0]), s02 = cv * (g[0][2] + g[2][0]), s12 = cv * (g[1][2] + g[2][1]);
        const T div = g[0][0] + g[1][1] + g[2][2];
        if constexpr (EXT) {
          // trace correction: -2 mu (div u) n n (the Darcy term sits in cm)
          const T nx = from_store<T>(__ldg(A.nrm + q * nc + cell));
          const T ny = from_store<T>(__ldg(A.nrm + (27 + q) * nc + cell));
          const T nz = from_store<T>(__ldg(A.nrm + (54 + q) * nc + cell));
          const T t = -(cv2 * div);
          const T tx = t * nx, ty = t * ny, tz = t * nz;
          s00 += tx * nx;
          s11 += ty * ny;
          s22 += tz * nz;
          s01 += tx * ny;
          s02 += tx * nz;
          s12 += ty * nz;
        }
        add_grad_test<T>(R0, qa, qb, qc, s00, s01, s02);
        add_grad_test<T>(R1, qa, qb, qc, s01, s11, s12);
        add_grad_test<T>(R2, qa, qb, qc, s02, s12, s22);
        // continuity test: -q div u (the factor -h^2 is applied at the scatter)
#pragma unroll
        for (int n = 0; n < 8; ++n) Rp[n] += Tb<T>::PWW(q, n) * div;
      }
  to_nodes<T>(R0);
  scatter_uniform<T>(A.dst, base, ug.sx, ug.sy, dmask, R0);
  to_nodes<T>(R1);
  scatter_uniform<T>(A.dst + A.nu, base, ug.sx, ug.sy, dmask, R1);
  to_nodes<T>(R2);
  scatter_uniform<T>(A.dst + 2 * A.nu, base, ug.sx, ug.sy, dmask, R2);
  St* pdst = A.dst + 3 * A.nu;
#pragma unroll
  for (int n = 0; n < 8; ++n)
    atomicAdd(pdst + pbase + (n & 1) + px * ((n >> 1) & 1) + pxy * (n >> 2), to_store<T>(mh2 * Rp[n]));
}

// The two coupling blocks of the Oseen operator alone, for the Schur complement B D^-1 B^T of
// the block preconditioner.  Same quadrature and scaling as k_oseen_qouter's pressure terms:
//   (B^T p)_{v} = -int p div v   (velocity rows; Dirichlet rows receive nothing)
//   (B u)_{q}  = -int q div u    (pressure rows; Dirichlet velocity values read as 0)
// dst must be zero on entry (atomic scatter).
template <typename T>
__global__ void __launch_bounds__(128) k_oseen_bt(const typename Store<T>::type* __restrict__ p,
                                                  typename Store<T>::type* __restrict__ dst_u, int64_t nu,
                                                  UniformGeom ug) {
  int i, j, k;
  if (!brick_cell(ug, i, j, k)) return;
  const int64_t base = 2 * int64_t(i) + ug.sx * (2 * int64_t(j)) + ug.sy * (2 * int64_t(k));
  const uint32_t dmask = dirichlet_mask(ug, i, j, k);
  const int64_t px = ug.nx + 1, pxy = px * (ug.ny + 1);
  const int64_t pbase = i + px * (j + (ug.ny + 1) * int64_t(k));
  const T h = T(ug.h);
  T Pn[8];
#pragma unroll
  for (int n = 0; n < 8; ++n) Pn[n] = from_store<T>(__ldg(p + pbase + (n & 1) + px * ((n >> 1) & 1) + pxy * (n >> 2)));
  T R0[27], R1[27], R2[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) { R0[q] = T(0); R1[q] = T(0); R2[q] = T(0); }
#pragma unroll
  for (int qc = 0; qc < 3; ++qc)
#pragma unroll
    for (int qb = 0; qb < 3; ++qb)
#pragma unroll
      for (int qa = 0; qa < 3; ++qa) {
        const int q = qa + 3 * qb + 9 * qc;
        T pq = T(0);
#pragma unroll
        for (int n = 0; n < 8; ++n) pq += q1w<T>(q, n) * Pn[n];
        const T pw = Tb<T>::W3(q) * (-h * pq);
        add_dir_test<T, 0>(R0, qa, qb, qc, pw);
        add_dir_test<T, 1>(R1, qa, qb, qc, pw);
        add_dir_test<T, 2>(R2, qa, qb, qc, pw);
      }
#pragma unroll
  for (int q = 0; q < 27; ++q) { R0[q] *= h; R1[q] *= h; R2[q] *= h; }
  to_nodes<T>(R0);
  scatter_uniform<T>(dst_u, base, ug.sx, ug.sy, dmask, R0);
  to_nodes<T>(R1);
  scatter_uniform<T>(dst_u + nu, base, ug.sx, ug.sy, dmask, R1);
  to_nodes<T>(R2);
  scatter_uniform<T>(dst_u + 2 * nu, base, ug.sx, ug.sy, dmask, R2);
}

template <typename T>
__global__ void __launch_bounds__(128) k_oseen_div(const typename Store<T>::type* __restrict__ u, int64_t nu,
                                                   typename Store<T>::type* __restrict__ dst_p, UniformGeom ug) {
  int i, j, k;
  if (!brick_cell(ug, i, j, k)) return;
  const int64_t base = 2 * int64_t(i) + ug.sx * (2 * int64_t(j)) + ug.sy * (2 * int64_t(k));
  const uint32_t dmask = dirichlet_mask(ug, i, j, k);
  const int64_t px = ug.nx + 1, pxy = px * (ug.ny + 1);
  const int64_t pbase = i + px * (j + (ug.ny + 1) * int64_t(k));
  const T h = T(ug.h);
  T U0[27], U1[27], U2[27];
  gather_uniform<T>(u, base, ug.sx, ug.sy, dmask, U0);
  gather_uniform<T>(u + nu, base, ug.sx, ug.sy, dmask, U1);
  gather_uniform<T>(u + 2 * nu, base, ug.sx, ug.sy, dmask, U2);
  to_qpoints<T>(U0);
  to_qpoints<T>(U1);
  to_qpoints<T>(U2);
  T Rp[8];
#pragma unroll
  for (int n = 0; n < 8; ++n) Rp[n] = T(0);
#pragma unroll
  for (int qc = 0; qc < 3; ++qc)
#pragma unroll
    for (int qb = 0; qb < 3; ++qb)
#pragma unroll
      for (int qa = 0; qa < 3; ++qa) {
        const int q = qa + 3 * qb + 9 * qc;
        T gx0, gy0, gz0, gx1, gy1, gz1, gx2, gy2, gz2;
        grad_at<T>(U0, qa, qb, qc, gx0, gy0, gz0);
        grad_at<T>(U1, qa, qb, qc, gx1, gy1, gz1);
        grad_at<T>(U2, qa, qb, qc, gx2, gy2, gz2);
        const T s = Tb<T>::W3(q) * (-h * (gx0 + gy1 + gz2));
#pragma unroll
        for (int n = 0; n < 8; ++n) Rp[n] += q1w<T>(q, n) * s;
      }
#pragma unroll
  for (int n = 0; n < 8; ++n)
    atomicAdd(dst_p + pbase + (n & 1) + px * ((n >> 1) & 1) + pxy * (n >> 2), to_store<T>(h * Rp[n]));
}

}  // namespace

template <typename T, int KIND, int MODE, bool BETA, bool TR>
static inline mf_status launch_one(mf_ctx* ctx, const mf_dofmap* m, const ScalarArgs<typename Store<T>::type>& a) {
  UniformGeom ug = m->uniform ? uniform_geom(m) : UniformGeom{};
  OctGeom og = oct_geom(m);
  // octree cell slots may be 64 or 128 wide; uniform bricks are 128 cells
  const int threads = m->uniform ? 128 : (a.block == 64 ? 64 : 128);
  const int64_t nwork = m->uniform ? brick_blocks(ug.nx, ug.ny, ug.nz) : (m->n_cells + threads - 1) / threads;
  int64_t grid = nwork;
  if (a.persistent_blocks > 0) grid = std::min<int64_t>(nwork, int64_t(a.persistent_blocks) * ctx->sm_count);
  if (grid < 1) return MF_OK;
  if (m->uniform)
    k_scalar<T, KIND, MODE, BETA, TR, false><<<unsigned(grid), threads, 0, ctx->stream>>>(a, ug, og, nwork);
  else
    k_scalar<T, KIND, MODE, BETA, TR, true><<<unsigned(grid), threads, 0, ctx->stream>>>(a, ug, og, nwork);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

// in-kernel coefficients exist for fp64 and fp32; double-float kernels read tabulated ones
template <typename T, int KIND, bool BETA, bool TR>
static inline mf_status launch_mode(mf_ctx* ctx, const mf_dofmap* m, int mode, const ScalarArgs<typename Store<T>::type>& a) {
  if constexpr (!std::is_same<T, df64>::value) {
    if (mode == 0) return launch_one<T, KIND, 0, BETA, TR>(ctx, m, a);
  }
  return launch_one<T, KIND, 1, BETA, TR>(ctx, m, a);
}

template <typename T>
static inline mf_status dispatch_scalar(mf_ctx* ctx, const mf_dofmap* m, int kind, int mode, bool beta, bool tr,
                                 const ScalarArgs<typename Store<T>::type>& a) {
  MF_CUDA_TRY(upload_tables_here());
  switch (kind) {
    case K_HELM:
      return launch_mode<T, K_HELM, false, false>(ctx, m, mode, a);
    case K_HEAT:
      if (!beta) return launch_mode<T, K_HEAT, false, false>(ctx, m, mode, a);
      if (!tr) return launch_mode<T, K_HEAT, true, false>(ctx, m, mode, a);
      return launch_mode<T, K_HEAT, true, true>(ctx, m, mode, a);
    case K_REINIT:
      return launch_mode<T, K_REINIT, false, false>(ctx, m, mode, a);
    case K_MASS:
      return launch_one<T, K_MASS, 1, false, false>(ctx, m, a);
  }
  return fail(MF_EINVAL, "unknown scalar operator kind");
}

}  // namespace mf
