// Local (one cell) action of the scalar operators in collocation form, shared by the apply
// and the dense element-matrix path of the diagonal.
#pragma once

#include "ops.h"

namespace mf {

// Smoothed Heaviside of the interpolated level set (Section 2.3).
template <typename T> __device__ __forceinline__ T heaviside(T phi, int kind, T eps) {
  if (kind == 0) {  // tanh-regularised reading: H = clamp((1 + phi)/2)
    T H = T(0.5) * (T(1) + phi);
    return H < T(0) ? T(0) : (H > T(1) ? T(1) : H);
  }
  // eq. (heaviside) with d = 2 eps atanh(phi)
  const T lim = T(1) - (sizeof(T) == 8 ? T(2.220446049250313e-16) : T(1.1920929e-7));
  T p = phi > lim ? lim : (phi < -lim ? -lim : phi);
  T d = T(2) * eps * atanh(p);
  if (d <= T(-3) * eps) return T(0);
  if (d >= T(3) * eps) return T(1);
  const T pi = T(3.141592653589793);
  return T(0.5) + d / (T(6) * eps) + sin(pi * d / (T(3) * eps)) / (T(2) * pi);
}

// U: nodal values of the cell (overwritten); R: the cell's contribution, at the nodes.
// C: scalar coefficient at the Gauss points (in-kernel phi for MODE 0 reinit).
template <typename T, int KIND, int MODE, bool BETA, bool TR>
__device__ __forceinline__ void scalar_local(const ScalarArgs<typename Store<T>::type>& A, int64_t cell, T h, T mh2,
                                             const T* C, T* U, T* R) {
  const T eps = T(A.eps);
  to_qpoints<T>(U);
#pragma unroll
  for (int q = 0; q < 27; ++q) R[q] = T(0);
#pragma unroll
  for (int qc = 0; qc < 3; ++qc)
#pragma unroll
    for (int qb = 0; qb < 3; ++qb)
#pragma unroll
      for (int qa = 0; qa < 3; ++qa) {
        const int q = qa + 3 * qb + 9 * qc;
        const T w = Tb<T>::W3(q);
        const T u = U[q];
        T fv;
        if constexpr (KIND == K_HEAT) {  // rho_cp / dt per Gauss point when the heat capacity varies
          fv = A.qmass ? w * ((from_store<T>(__ldg(A.qmass + q * A.ncp + cell)) * (h * h)) * u) : w * (mh2 * u);
        } else {
          fv = w * (mh2 * u);
        }
        if constexpr (KIND == K_MASS) {
          R[q] += fv;
          continue;
        }
        T gx, gy, gz;
        grad_at<T>(U, qa, qb, qc, gx, gy, gz);
        T Fx, Fy, Fz;
        if constexpr (KIND == K_REINIT) {
          T nx, ny, nz;
          if constexpr (MODE == 0) {
            grad_at<T>(C, qa, qb, qc, nx, ny, nz);
            T nn = sqrt(nx * nx + ny * ny + nz * nz);
            T inv = nn < T(1e-12) ? T(0) : T(1) / nn;
            nx *= inv; ny *= inv; nz *= inv;
          } else {
            nx = from_store<T>(__ldg(A.qvec + (0 * 27 + q) * A.ncp + cell));
            ny = from_store<T>(__ldg(A.qvec + (1 * 27 + q) * A.ncp + cell));
            nz = from_store<T>(__ldg(A.qvec + (2 * 27 + q) * A.ncp + cell));
          }
          const T s = w * (eps * (nx * gx + ny * gy + nz * gz));
          Fx = s * nx; Fy = s * ny; Fz = s * nz;
        } else {
          const T c = w * C[q];
          Fx = c * gx; Fy = c * gy; Fz = c * gz;
        }
        if constexpr (BETA) {
          const T bx = from_store<T>(__ldg(A.qvec + (0 * 27 + q) * A.ncp + cell));
          const T by = from_store<T>(__ldg(A.qvec + (1 * 27 + q) * A.ncp + cell));
          const T bz = from_store<T>(__ldg(A.qvec + (2 * 27 + q) * A.ncp + cell));
          if constexpr (!TR) {
            fv += w * (h * (bx * gx + by * gy + bz * gz));
          } else {
            const T s = w * (h * u);
            Fx += s * bx; Fy += s * by; Fz += s * bz;
          }
        }
        R[q] += fv;
        add_grad_test<T>(R, qa, qb, qc, Fx, Fy, Fz);
      }
  to_nodes<T>(R);
#pragma unroll
  for (int q = 0; q < 27; ++q) R[q] *= h;
}

}  // namespace mf
