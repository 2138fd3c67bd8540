// Set-up kernels of the operators: Gauss-point coefficient tables (always evaluated in
// fp64), matrix-free diagonals and block-Jacobi blocks, the laser top-face load of
// eq. (laser_gauss) and the conductivity gradient of the heat-step adjoint.
#include <cmath>

#include "scalar_local.cuh"

namespace mf {

MF_DEFINE_TABLE_UPLOAD

UniformGeom uniform_geom(const mf_dofmap* m);
OctGeom oct_geom(const mf_dofmap* m);

namespace {

// cell index t of the map's natural order -> location
struct Loc {
  int64_t cell;
  int64_t base;
  uint32_t dmask;
  double h;
  int i, j, k;
};

template <bool OCT>
__device__ __forceinline__ bool natural_cell(const UniformGeom& ug, const OctGeom& og, int64_t t, Loc& L) {
  if (OCT) {
    if (t >= og.ncells) return false;
    L.cell = t;
    L.h = og.h0 / double(1 << __ldg(og.level + t));
    L.base = 0;
    L.dmask = 0;
    return true;
  }
  const int64_t nc = int64_t(ug.nx) * ug.ny * ug.nz;
  if (t >= nc) return false;
  L.i = int(t % ug.nx);
  L.j = int((t / ug.nx) % ug.ny);
  L.k = int(t / (int64_t(ug.nx) * ug.ny));
  L.cell = t;
  L.base = 2 * int64_t(L.i) + ug.sx * (2 * int64_t(L.j)) + ug.sy * (2 * int64_t(L.k));
  L.dmask = dirichlet_mask(ug, L.i, L.j, L.k);
  L.h = ug.h;
  return true;
}

template <bool OCT, bool MASK>
__device__ __forceinline__ void gather64(const UniformGeom& ug, const OctGeom& og, const Loc& L, const double* src,
                                         double* U) {
  if (OCT) gather_oct<double, MASK>(og, src, L.cell, U);
  else gather_uniform<double>(src, L.base, ug.sx, ug.sy, MASK ? L.dmask : 0u, U);
}

// ---------------------------------------------------------------- Gauss-point tables
template <bool OCT>
__global__ void k_scalar_qtables(UniformGeom ug, OctGeom og, int kind, const double* field, const double* kq_user,
                                 const double* beta, int64_t nd, double k0, double kslope, double a_l, double a_g,
                                 int hv, double eps, double rhocp, int64_t ncp, double* qc64, float* qc32,
                                 double* qv64, float* qv32, const double* rhocp_q, const double* beta_q, double dt,
                                 double* qm64, float* qm32) {
  Loc L;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (!natural_cell<OCT>(ug, og, t, L)) return;
  double C[27];
  if (kind == K_HEAT && kq_user) {
    for (int q = 0; q < 27; ++q) C[q] = kq_user[L.cell * 27 + q];
  } else if (field) {
    gather64<OCT, false>(ug, og, L, field, C);
    to_qpoints<double>(C);
  }
  if (kind == K_HELM) {
    for (int q = 0; q < 27; ++q) {
      double a = a_g + (a_l - a_g) * heaviside<double>(C[q], hv, eps);
      qc64[q * ncp + L.cell] = a;
      qc32[q * ncp + L.cell] = float(a);
    }
  } else if (kind == K_HEAT) {
    for (int q = 0; q < 27; ++q) {
      double k = kq_user ? C[q] : k0 + kslope * C[q];
      qc64[q * ncp + L.cell] = k;
      qc32[q * ncp + L.cell] = float(k);
    }
    if (rhocp_q) {
      for (int q = 0; q < 27; ++q) {
        const double m = rhocp_q[L.cell * 27 + q] / dt;
        qm64[q * ncp + L.cell] = m;
        qm32[q * ncp + L.cell] = float(m);
      }
    }
    if (beta || beta_q) {
      for (int d = 0; d < 3; ++d) {
        double B[27];
        if (beta_q) {
          for (int q = 0; q < 27; ++q) B[q] = beta_q[(L.cell * 27 + q) * 3 + d];
        } else {
          gather64<OCT, false>(ug, og, L, beta + d * nd, B);
          to_qpoints<double>(B);
        }
        for (int q = 0; q < 27; ++q) {
          const double v = (rhocp_q ? rhocp_q[L.cell * 27 + q] : rhocp) * B[q];
          qv64[(d * 27 + q) * ncp + L.cell] = v;
          qv32[(d * 27 + q) * ncp + L.cell] = float(v);
        }
      }
    }
  } else if (kind == K_REINIT) {
#pragma unroll
    for (int qc = 0; qc < 3; ++qc)
#pragma unroll
      for (int qb = 0; qb < 3; ++qb)
#pragma unroll
        for (int qa = 0; qa < 3; ++qa) {
          const int q = qa + 3 * qb + 9 * qc;
          double nx, ny, nz;
          grad_at<double>(C, qa, qb, qc, nx, ny, nz);
          double nn = sqrt(nx * nx + ny * ny + nz * nz);
          double inv = nn < 1e-12 ? 0.0 : 1.0 / nn;
          double n3[3] = {nx * inv, ny * inv, nz * inv};
          for (int d = 0; d < 3; ++d) {
            qv64[(d * 27 + q) * ncp + L.cell] = n3[d];
            qv32[(d * 27 + q) * ncp + L.cell] = float(n3[d]);
          }
        }
  }
}

__global__ void k_oseen_qtables(UniformGeom ug, const double* phi, const double* beta, double rho_l, double rho_g,
                                double mu_l, double mu_g, int hv, double eps, double* r64, float* r32, double* m64,
                                float* m32, double* b64, float* b32) {
  Loc L;
  OctGeom og{};
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (!natural_cell<false>(ug, og, t, L)) return;
  const int64_t nc = int64_t(ug.nx) * ug.ny * ug.nz;
  double C[27];
  gather64<false, false>(ug, og, L, phi, C);
  to_qpoints<double>(C);
  for (int q = 0; q < 27; ++q) {
    double H = heaviside<double>(C[q], hv, eps);
    double rho = 1.0 / (H / rho_l + (1.0 - H) / rho_g);  // eq. (rhoEff)
    double mu = H * mu_l + (1.0 - H) * mu_g;              // eq. (muEff)
    r64[q * nc + L.cell] = rho;
    r32[q * nc + L.cell] = float(rho);
    m64[q * nc + L.cell] = mu;
    m32[q * nc + L.cell] = float(mu);
  }
  for (int d = 0; d < 3; ++d) {
    gather64<false, false>(ug, og, L, beta + d * ug.n_dofs, C);
    to_qpoints<double>(C);
    for (int q = 0; q < 27; ++q) {
      b64[(d * 27 + q) * nc + L.cell] = C[q];
      b32[(d * 27 + q) * nc + L.cell] = float(C[q]);
    }
  }
}

// Melt-pool extensions of the Oseen tables, evaluated in fp64 at the Gauss points from the nodal
// phi and T: three-phase rho and mu (eqs. solid_liquid_gas_density, solid_liquid_gas_property with
// H_s of eq. heaviside_sl), the Darcy coefficient H_phi C f_s^2 / ((1 - f_s)^3 + b) of eq.
// (darcy_damping_force) and the unit normal grad phi_h / |grad phi_h| of the trace correction.
__global__ void k_oseen_ext_tables(UniformGeom ug, const double* phi, const double* T, int hv, double eps, int flags,
                                   double rho_l, double rho_g, double rho_s, double mu_l, double mu_g, double mu_s,
                                   double t_sol, double t_liq, double dc, double db, double* r64, float* r32,
                                   double* m64, float* m32, double* kd64, float* kd32, double* n64, float* n32) {
  Loc L;
  OctGeom og{};
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (!natural_cell<false>(ug, og, t, L)) return;
  const int64_t nc = int64_t(ug.nx) * ug.ny * ug.nz;
  const bool need_t = (flags & (MF_OSEEN_THREE_PHASE | MF_OSEEN_DARCY)) != 0;
  double P[27], TT[27];
  gather64<false, false>(ug, og, L, phi, P);
  to_qpoints<double>(P);
  if (need_t) {
    gather64<false, false>(ug, og, L, T, TT);
    to_qpoints<double>(TT);
  }
  for (int qc = 0; qc < 3; ++qc)
    for (int qb = 0; qb < 3; ++qb)
      for (int qa = 0; qa < 3; ++qa) {
        const int q = qa + 3 * qb + 9 * qc;
        const int64_t o = q * nc + L.cell;
        const double H = heaviside<double>(P[q], hv, eps);
        double fs = 0.0;
        if (need_t) {
          fs = (t_liq - TT[q]) / (t_liq - t_sol);
          fs = fs < 0.0 ? 0.0 : (fs > 1.0 ? 1.0 : fs);
        }
        if (flags & MF_OSEEN_THREE_PHASE) {
          const double Hs = 3.0 * fs * fs - 2.0 * fs * fs * fs;
          const double rho_sl = Hs * rho_s + (1.0 - Hs) * rho_l;
          const double rho = 1.0 / (H / rho_sl + (1.0 - H) / rho_g);
          const double mu = H * (Hs * mu_s + (1.0 - Hs) * mu_l) + (1.0 - H) * mu_g;
          r64[o] = rho;
          r32[o] = float(rho);
          m64[o] = mu;
          m32[o] = float(mu);
        }
        const double kd = (flags & MF_OSEEN_DARCY) ? H * dc * fs * fs / ((1.0 - fs) * (1.0 - fs) * (1.0 - fs) + db) : 0.0;
        kd64[o] = kd;
        kd32[o] = float(kd);
        double nx = 0.0, ny = 0.0, nz = 0.0;
        if (flags & MF_OSEEN_TRACE_CORRECTION) {
          double gx, gy, gz;
          grad_at<double>(P, qa, qb, qc, gx, gy, gz);  // reference gradient = h grad phi_h
          const double g = sqrt(gx * gx + gy * gy + gz * gz);
          if (!(g < 1e-12)) {
            nx = gx / g;
            ny = gy / g;
            nz = gz / g;
          }
        }
        n64[o] = nx;
        n64[27 * nc + o] = ny;
        n64[54 * nc + o] = nz;
        n32[o] = float(nx);
        n32[27 * nc + o] = float(ny);
        n32[54 * nc + o] = float(nz);
      }
}

// cm = w h^3 (sigma rho + kd), cv = w h mu and cb_d = w h^2 rho beta_d per (Gauss point, cell), in
// fp64 and fp32
__global__ void k_oseen_fold(int64_t nc, double h, double sigma, const double* rho, const double* mu,
                             const double* kd, const double* beta, double* cm64, float* cm32, double* cb64,
                             float* cb32, double* cv64, float* cv32) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= 27 * nc) return;
  const int q = int(t / nc);
  const double w = cW364[q];
  const double m = w * h * h * h * (sigma * rho[t] + (kd ? kd[t] : 0.0));
  const double c = w * h * h * rho[t];
  const double v = w * h * mu[t];
  cm64[t] = m;
  cm32[t] = float(m);
  for (int d = 0; d < 3; ++d) {
    const double b = c * beta[d * 27 * nc + t];
    cb64[d * 27 * nc + t] = b;
    cb32[d * 27 * nc + t] = float(b);
  }
  cv64[t] = v;
  cv32[t] = float(v);
}

// ---------------------------------------------------------------- diagonals
// out[l] += sum_q c[q] X[qa][a] Y[qb][b] Z[qc][c] with 1D tables X, Y, Z (3x3, [q][a]).
template <typename T>
__device__ __forceinline__ void separable_add(const T* c, const T* X, const T* Y, const T* Z, T* out) {
  T t[27];
#pragma unroll
  for (int i = 0; i < 27; ++i) t[i] = c[i];
  // x: t[a, qb, qc] = sum_qa X[qa][a] t[qa, qb, qc]
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    T u0 = t[3 * j], u1 = t[3 * j + 1], u2 = t[3 * j + 2];
    t[3 * j] = X[0] * u0 + X[3] * u1 + X[6] * u2;
    t[3 * j + 1] = X[1] * u0 + X[4] * u1 + X[7] * u2;
    t[3 * j + 2] = X[2] * u0 + X[5] * u1 + X[8] * u2;
  }
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    const int b = (j % 3) + 9 * (j / 3);
    T u0 = t[b], u1 = t[b + 3], u2 = t[b + 6];
    t[b] = Y[0] * u0 + Y[3] * u1 + Y[6] * u2;
    t[b + 3] = Y[1] * u0 + Y[4] * u1 + Y[7] * u2;
    t[b + 6] = Y[2] * u0 + Y[5] * u1 + Y[8] * u2;
  }
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    T u0 = t[j], u1 = t[j + 9], u2 = t[j + 18];
    out[j] += Z[0] * u0 + Z[3] * u1 + Z[6] * u2;
    out[j + 9] += Z[1] * u0 + Z[4] * u1 + Z[7] * u2;
    out[j + 18] += Z[2] * u0 + Z[5] * u1 + Z[8] * u2;
  }
}

// Diagonal of the element matrix, summed into diag, for cells without constrained nodes:
// A_e[l,l] = sum_q w h^3 m N_l^2 + w h (gN_l)^T K (gN_l) + w h^2 N_l c . gN_l
// with N_l = S_a S_b S_c and reference derivatives S' in one factor.
template <bool OCT>
__global__ void k_scalar_diag(ScalarArgs<double> A, int kind, bool beta, UniformGeom ug, OctGeom og, int64_t ncount,
                              double* diag) {
  Loc L;
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= ncount) return;
  if (OCT) t = __ldg(og.order + t);
  if (!natural_cell<OCT>(ug, og, t, L)) return;
  const double h = L.h;
  double out[27], c[27];
  for (int i = 0; i < 27; ++i) out[i] = 0.0;
  // mass
  for (int q = 0; q < 27; ++q) c[q] = cW364[q] * h * h * h * (A.qmass ? A.qmass[q * A.ncp + L.cell] : A.mass);
  separable_add(c, cSS64, cSS64, cSS64, out);
  if (kind == K_HELM || kind == K_HEAT) {
    for (int q = 0; q < 27; ++q) c[q] = cW364[q] * h * A.qcoef[q * A.ncp + L.cell];
    separable_add(c, cSpSp64, cSS64, cSS64, out);
    separable_add(c, cSS64, cSpSp64, cSS64, out);
    separable_add(c, cSS64, cSS64, cSpSp64, out);
  } else if (kind == K_REINIT) {
    // K = eps n n^T: terms (d, e) with S' in factors d and e
    for (int d = 0; d < 3; ++d)
      for (int e = d; e < 3; ++e) {
        for (int q = 0; q < 27; ++q) {
          double nd = A.qvec[(d * 27 + q) * A.ncp + L.cell], ne = A.qvec[(e * 27 + q) * A.ncp + L.cell];
          c[q] = cW364[q] * h * A.eps * nd * ne * (d == e ? 1.0 : 2.0);
        }
        const double* F[3] = {cSS64, cSS64, cSS64};
        if (d == e) F[d] = cSpSp64;
        else { F[d] = cSSp64; F[e] = cSSp64; }
        separable_add(c, F[0], F[1], F[2], out);
      }
  }
  if (beta) {
    for (int d = 0; d < 3; ++d) {
      for (int q = 0; q < 27; ++q) c[q] = cW364[q] * h * h * A.qvec[(d * 27 + q) * A.ncp + L.cell];
      const double* F[3] = {cSS64, cSS64, cSS64};
      F[d] = cSSp64;
      separable_add(c, F[0], F[1], F[2], out);
    }
  }
  if (OCT) {
    for (int l = 0; l < 27; ++l) {
      int32_t id = __ldg(og.cmap + l * og.ncp + L.cell);
      if (!(og.dflag && og.dflag[id])) atomicAdd(diag + id, out[l]);
    }
  } else {
    for (int l = 0; l < 27; ++l) {
      if ((L.dmask >> l) & 1u) continue;
      const int a = l % 3, b = (l / 3) % 3, cc = l / 9;
      atomicAdd(diag + L.base + a + ug.sx * b + ug.sy * cc, out[l]);
    }
  }
}

// Cells with constrained nodes: dense element matrix from unit vectors, then
// diag_j += sum_{l,l'} C[l][j] A_e[l][l'] C[l'][j] over the free DoFs j the cell touches.
template <int KIND, bool BETA>
__global__ void k_scalar_diag_constrained(ScalarArgs<double> A, OctGeom og, int64_t first, int64_t count,
                                          double* diag) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t cell = __ldg(og.order + first + t);
  const double h = og.h0 / double(1 << og.level[cell]);
  const double mh2 = A.mass * h * h;
  double C[27];
  if (KIND != K_REINIT)
    for (int q = 0; q < 27; ++q) C[q] = A.qcoef[q * A.ncp + cell];
  double Ae[27][27];
  for (int l = 0; l < 27; ++l) {
    double U[27], R[27];
    for (int i = 0; i < 27; ++i) U[i] = i == l ? 1.0 : 0.0;
    scalar_local<double, KIND, 1, BETA, false>(A, cell, h, mh2, C, U, R);
    for (int i = 0; i < 27; ++i) Ae[i][l] = R[i];
  }
  for (int l = 0; l < 27; ++l) {
    int32_t id = og.cmap[l * og.ncp + cell];
    int eb = 0, ee = 1;
    if (id < 0) { eb = og.rowptr[-1 - id]; ee = og.rowptr[-id]; }
    for (int e = eb; e < ee; ++e) {
      const int32_t j = id >= 0 ? id : og.cols[e];
      const double wj = id >= 0 ? 1.0 : og.w64[e];
      if (og.dflag && og.dflag[j]) continue;
      double acc = 0.0;
      for (int l2 = 0; l2 < 27; ++l2) {
        int32_t id2 = og.cmap[l2 * og.ncp + cell];
        if (id2 >= 0) {
          if (id2 == j) acc += Ae[l][l2];
        } else {
          for (int e2 = og.rowptr[-1 - id2]; e2 < og.rowptr[-id2]; ++e2)
            if (og.cols[e2] == j) acc += Ae[l][l2] * og.w64[e2];
        }
      }
      atomicAdd(diag + j, wj * acc);
    }
  }
}

__global__ void k_set_dirichlet(double* v, const int32_t* list, int64_t n, double val, int stride) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) v[int64_t(list[t]) * stride] = val;
}

// Oseen block-Jacobi: 3x3 nodal velocity blocks of A_uu and the pressure scaling.
__global__ void k_oseen_blocks(OseenArgs<double> A, UniformGeom ug, double* blk, double* pm, double* pk) {
  Loc L;
  OctGeom og{};
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (!natural_cell<false>(ug, og, t, L)) return;
  const int64_t nc = int64_t(ug.nx) * ug.ny * ug.nz;
  const double h = L.h;
  double s[27], c[27];
  for (int i = 0; i < 27; ++i) s[i] = 0.0;
  // scalar part: sigma rho mass + rho convection + mu |grad|^2
  // mass-like part: sigma rho (+ the Darcy coefficient of the melt-pool extension)
  for (int q = 0; q < 27; ++q)
    c[q] = cW364[q] * h * h * h * (A.sigma * A.rho[q * nc + L.cell] + (A.ext ? A.kd[q * nc + L.cell] : 0.0));
  separable_add(c, cSS64, cSS64, cSS64, s);
  for (int d = 0; d < 3; ++d) {
    for (int q = 0; q < 27; ++q) c[q] = cW364[q] * h * h * A.rho[q * nc + L.cell] * A.beta[(d * 27 + q) * nc + L.cell];
    const double* F[3] = {cSS64, cSS64, cSS64};
    F[d] = cSSp64;
    separable_add(c, F[0], F[1], F[2], s);
  }
  for (int q = 0; q < 27; ++q) c[q] = cW364[q] * h * A.mu[q * nc + L.cell];
  double X[6][27];
  for (int i = 0; i < 6; ++i)
    for (int l = 0; l < 27; ++l) X[i][l] = 0.0;
  separable_add(c, cSpSp64, cSS64, cSS64, X[0]);  // xx
  separable_add(c, cSS64, cSpSp64, cSS64, X[1]);  // yy
  separable_add(c, cSS64, cSS64, cSpSp64, X[2]);  // zz
  separable_add(c, cSSp64, cSSp64, cSS64, X[3]);  // xy
  separable_add(c, cSSp64, cSS64, cSSp64, X[4]);  // xz
  separable_add(c, cSS64, cSSp64, cSSp64, X[5]);  // yz
  for (int l = 0; l < 27; ++l) {
    if ((L.dmask >> l) & 1u) continue;
    const int a = l % 3, b = (l / 3) % 3, cc = l / 9;
    const int64_t id = L.base + a + ug.sx * b + ug.sy * cc;
    const double lap = X[0][l] + X[1][l] + X[2][l];
    // B[c][d] = delta_cd (s + mu |grad N|^2) + mu d_d N d_c N
    double B[9] = {s[l] + lap + X[0][l], X[3][l], X[4][l],
                   X[3][l], s[l] + lap + X[1][l], X[5][l],
                   X[4][l], X[5][l], s[l] + lap + X[2][l]};
    if (A.ext) {
      // trace correction -2 mu (div u) n n (n = 0 where it is switched off): with u = N e_e,
      // B[d][e] += sum_q -2 w h mu n_d (n . grad N) d_e N, not symmetric in (d, e)
      for (int q = 0; q < 27; ++q) {
        const int qa = q % 3, qb = (q / 3) % 3, qc = q / 9;
        const double n0 = A.nrm[q * nc + L.cell], n1 = A.nrm[(27 + q) * nc + L.cell];
        const double n2 = A.nrm[(54 + q) * nc + L.cell];
        if (n0 == 0.0 && n1 == 0.0 && n2 == 0.0) continue;
        const double g0 = cSp64[3 * qa + a] * cS64[3 * qb + b] * cS64[3 * qc + cc];
        const double g1 = cS64[3 * qa + a] * cSp64[3 * qb + b] * cS64[3 * qc + cc];
        const double g2 = cS64[3 * qa + a] * cS64[3 * qb + b] * cSp64[3 * qc + cc];
        const double t = -2.0 * cW364[q] * h * A.mu[q * nc + L.cell] * (n0 * g0 + n1 * g1 + n2 * g2);
        const double tn[3] = {t * n0, t * n1, t * n2};
        for (int d = 0; d < 3; ++d) {
          B[3 * d] += tn[d] * g0;
          B[3 * d + 1] += tn[d] * g1;
          B[3 * d + 2] += tn[d] * g2;
        }
      }
    }
    for (int e = 0; e < 9; ++e) atomicAdd(blk + id * 9 + e, B[e]);
  }
  // pressure: sum_q w h^3 psi_i^2 / mu and sum_q w h |grad psi_i|^2 / (sigma rho)
  const int64_t px = ug.nx + 1, pxy = px * (ug.ny + 1);
  const int64_t pbase = L.i + px * (L.j + (ug.ny + 1) * int64_t(L.k));
  for (int n = 0; n < 8; ++n) {
    const int a = n & 1, b = (n >> 1) & 1, cc = n >> 2;
    double m = 0.0, kk = 0.0;
    for (int q = 0; q < 27; ++q) {
      const int qa = q % 3, qb = (q / 3) % 3, qc = q / 9;
      const double pa = cP64[2 * qa + a], pb = cP64[2 * qb + b], pc = cP64[2 * qc + cc];
      const double psi = pa * pb * pc;
      const double g2 = pb * pb * pc * pc + pa * pa * pc * pc + pa * pa * pb * pb;  // |psi'|^2 with P' = -+1
      m += cW364[q] * h * h * h * psi * psi / A.mu[q * nc + L.cell];
      kk += cW364[q] * h * g2 / (A.sigma * A.rho[q * nc + L.cell] + (A.ext ? A.kd[q * nc + L.cell] : 0.0));
    }
    const int64_t id = pbase + a + px * b + pxy * cc;
    atomicAdd(pm + id, m);
    atomicAdd(pk + id, kk);
  }
}

__global__ void k_invert_blocks(double* blk, const uint8_t* dir, int64_t n) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* B = blk + 9 * i;
  if (dir && dir[i]) {
    for (int e = 0; e < 9; ++e) B[e] = (e % 4 == 0) ? 1.0 : 0.0;
    return;
  }
  double a = B[0], b = B[1], c = B[2], d = B[3], e = B[4], f = B[5], g = B[6], hh = B[7], k = B[8];
  double A0 = e * k - f * hh, A1 = -(d * k - f * g), A2 = d * hh - e * g;
  double det = a * A0 + b * A1 + c * A2;
  double inv = 1.0 / det;
  B[0] = A0 * inv; B[1] = -(b * k - c * hh) * inv; B[2] = (b * f - c * e) * inv;
  B[3] = A1 * inv; B[4] = (a * k - c * g) * inv; B[5] = -(a * f - c * d) * inv;
  B[6] = A2 * inv; B[7] = -(a * hh - b * g) * inv; B[8] = (a * e - b * d) * inv;
}

template <typename T> __global__ void k_pressure_scaling(const T* pm, const T* pk, T* pinv, int64_t n) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // Schur complement diagonal ~ (1/pm + 1/pk)^-1; store its inverse
  pinv[i] = T(1) / pm[i] + T(1) / pk[i];
}

// The same blocks and pressure scaling in fp32, for the block-triangular preconditioner (which
// applies them in fp32): built from the folded fp32 Gauss-point tables cm = w h^3 (sigma rho +
// Darcy), cb_d = w h^2 rho beta_d and cv = w h mu.  One thread per cell; its 27 x 9 block entries
// accumulate in the thread's own shared-memory column (entry (e, l) at [(9 l + e) kBlk32][thread])
// and leave with one atomic each into the entry-major output blk[e nu + node].
constexpr int kBlk32 = 32;
__global__ void __launch_bounds__(kBlk32) k_oseen_blocks32(OseenArgs<float> A, UniformGeom ug, float* blk, float* pm,
                                                           float* pk) {
  __shared__ float sB[243 * kBlk32];
  Loc L;
  OctGeom og{};
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (!natural_cell<false>(ug, og, t, L)) return;
  const int64_t nc = int64_t(ug.nx) * ug.ny * ug.nz, cell = L.cell;
  float* B = sB + threadIdx.x;
  auto at = [&](int e, int l) -> float& { return B[(9 * l + e) * kBlk32]; };
  float c[27], s[27];
  // scalar part sigma rho mass (+ Darcy) + rho convection, on the three diagonal entries
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    c[q] = A.cm[q * nc + cell];
    s[q] = 0.f;
  }
  separable_add<float>(c, cSS32, cSS32, cSS32, s);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int q = 0; q < 27; ++q) c[q] = A.cb[(d * 27 + q) * nc + cell];
    separable_add<float>(c, d == 0 ? cSSp32 : cSS32, d == 1 ? cSSp32 : cSS32, d == 2 ? cSSp32 : cSS32, s);
  }
#pragma unroll
  for (int l = 0; l < 27; ++l)
#pragma unroll
    for (int e = 0; e < 9; ++e) at(e, l) = (e % 4 == 0) ? s[l] : 0.f;
  // viscous part: B[d][e] = delta_de mu |grad N|^2 + mu d_e N d_d N
#pragma unroll
  for (int q = 0; q < 27; ++q) c[q] = A.cv[q * nc + cell];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int l = 0; l < 27; ++l) s[l] = 0.f;
    separable_add<float>(c, d == 0 ? cSpSp32 : cSS32, d == 1 ? cSpSp32 : cSS32, d == 2 ? cSpSp32 : cSS32, s);
#pragma unroll
    for (int l = 0; l < 27; ++l) {
      at(0, l) += d == 0 ? 2.f * s[l] : s[l];
      at(4, l) += d == 1 ? 2.f * s[l] : s[l];
      at(8, l) += d == 2 ? 2.f * s[l] : s[l];
    }
  }
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const int d = p == 2 ? 1 : 0, e = p == 0 ? 1 : 2;  // (0,1), (0,2), (1,2)
#pragma unroll
    for (int l = 0; l < 27; ++l) s[l] = 0.f;
    separable_add<float>(c, (d == 0) ? cSSp32 : cSS32, (d == 1 || e == 1) ? cSSp32 : cSS32,
                         (e == 2) ? cSSp32 : cSS32, s);
#pragma unroll
    for (int l = 0; l < 27; ++l) {
      at(3 * d + e, l) += s[l];
      at(3 * e + d, l) += s[l];
    }
  }
  if (A.ext) {
    // trace correction: B[d][e] += sum_q -2 cv n_d (n . grad N) d_e N (nonsymmetric)
    float n0[27], n1[27], n2[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      n0[q] = A.nrm[q * nc + cell];
      n1[q] = A.nrm[(27 + q) * nc + cell];
      n2[q] = A.nrm[(54 + q) * nc + cell];
      c[q] *= -2.f;
    }
    for (int l = 0; l < 27; ++l) {
      const int a = l % 3, b = (l / 3) % 3, cc = l / 9;
      float Sa[3], Pa[3], Sb[3], Pb[3], Sc[3], Pc[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        Sa[k] = cS32[3 * k + a];
        Pa[k] = cSp32[3 * k + a];
        Sb[k] = cS32[3 * k + b];
        Pb[k] = cSp32[3 * k + b];
        Sc[k] = cS32[3 * k + cc];
        Pc[k] = cSp32[3 * k + cc];
      }
      float acc[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) acc[e] = 0.f;
#pragma unroll
      for (int q = 0; q < 27; ++q) {
        const int qa = q % 3, qb = (q / 3) % 3, qc = q / 9;
        const float g0 = Pa[qa] * Sb[qb] * Sc[qc], g1 = Sa[qa] * Pb[qb] * Sc[qc], g2 = Sa[qa] * Sb[qb] * Pc[qc];
        const float tq = c[q] * (n0[q] * g0 + n1[q] * g1 + n2[q] * g2);
        const float tn[3] = {tq * n0[q], tq * n1[q], tq * n2[q]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          acc[3 * d] += tn[d] * g0;
          acc[3 * d + 1] += tn[d] * g1;
          acc[3 * d + 2] += tn[d] * g2;
        }
      }
#pragma unroll
      for (int e = 0; e < 9; ++e) at(e, l) += acc[e];
    }
  }
  const int64_t nu = A.nu;
  for (int l = 0; l < 27; ++l) {
    if ((L.dmask >> l) & 1u) continue;
    const int a = l % 3, b = (l / 3) % 3, cc = l / 9;
    const int64_t id = L.base + a + ug.sx * b + ug.sy * cc;
#pragma unroll
    for (int e = 0; e < 9; ++e) atomicAdd(blk + e * nu + id, at(e, l));
  }
  // pressure: sum_q psi_i^2 w h^3 / mu and sum_q |grad psi_i|^2 w h / (sigma rho + Darcy), with
  // w h^3 / mu = (w h^2)^2 / cv and w h / (sigma rho + Darcy) = (w h^2)^2 / cm
  const float h = float(L.h);
  float r1[27], r2[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const float whh = cW332[q] * h * h;
    r1[q] = whh * (whh / A.cv[q * nc + cell]);
    r2[q] = whh * (whh / A.cm[q * nc + cell]);
  }
  const int64_t px = ug.nx + 1, pxy = px * (ug.ny + 1);
  const int64_t pbase = L.i + px * (L.j + (ug.ny + 1) * int64_t(L.k));
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const int a = n & 1, b = (n >> 1) & 1, cc = n >> 2;
    float m = 0.f, kk = 0.f;
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      const int qa = q % 3, qb = (q / 3) % 3, qc = q / 9;
      const float pa = cP32[2 * qa + a], pb = cP32[2 * qb + b], pc = cP32[2 * qc + cc];
      const float psi = pa * pb * pc;
      m += psi * psi * r1[q];
      kk += (pb * pb * pc * pc + pa * pa * pc * pc + pa * pa * pb * pb) * r2[q];
    }
    const int64_t id = pbase + a + px * b + pxy * cc;
    atomicAdd(pm + id, m);
    atomicAdd(pk + id, kk);
  }
}

// inverse of each entry-major fp32 3 x 3 block in place
__global__ void k_invert_blocks_soa32(float* blk, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float a = blk[i], b = blk[n + i], c = blk[2 * n + i], d = blk[3 * n + i], e = blk[4 * n + i];
  const float f = blk[5 * n + i], g = blk[6 * n + i], hh = blk[7 * n + i], k = blk[8 * n + i];
  const float A0 = e * k - f * hh, A1 = -(d * k - f * g), A2 = d * hh - e * g;
  const float inv = 1.f / (a * A0 + b * A1 + c * A2);
  blk[i] = A0 * inv;
  blk[n + i] = -(b * k - c * hh) * inv;
  blk[2 * n + i] = (b * f - c * e) * inv;
  blk[3 * n + i] = A1 * inv;
  blk[4 * n + i] = (a * k - c * g) * inv;
  blk[5 * n + i] = -(a * f - c * d) * inv;
  blk[6 * n + i] = A2 * inv;
  blk[7 * n + i] = -(a * hh - b * g) * inv;
  blk[8 * n + i] = (a * e - b * d) * inv;
}

// identity blocks at the listed (Dirichlet) nodes, entry-major
__global__ void k_identity_blocks_soa32(float* blk, const int32_t* list, int64_t nl, int64_t n) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= nl) return;
  const int64_t i = list[t];
#pragma unroll
  for (int e = 0; e < 9; ++e) blk[e * n + i] = (e % 4 == 0) ? 1.f : 0.f;
}

// ---------------------------------------------------------------- laser load
__global__ void k_laser(UniformGeom ug, double lox, double loy, double P, double r, double x0, double y0, double chi,
                        double* f, double* dF) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(ug.nx) * ug.ny) return;
  const int i = int(t % ug.nx), j = int(t / ug.nx), k = ug.nz - 1;
  const double h = ug.h;
  const double ox = lox + i * h, oy = loy + j * h;
  double fe[5][9];
  for (int p = 0; p < 5; ++p)
    for (int n = 0; n < 9; ++n) fe[p][n] = 0.0;
  const double pi = 3.141592653589793;
  for (int qb = 0; qb < 3; ++qb)
    for (int qa = 0; qa < 3; ++qa) {
      const double x = ox + h * cG64[qa], y = oy + h * cG64[qb];
      const double r2 = (x - x0) * (x - x0) + (y - y0) * (y - y0);
      const double q = 2.0 * chi * P / (pi * r * r) * exp(-2.0 * r2 / (r * r));
      const double dq[5] = {q, q / P, q * (-2.0 / r + 4.0 * r2 / (r * r * r)), 4.0 * q * (x - x0) / (r * r),
                            4.0 * q * (y - y0) / (r * r)};
      const double w = cW64[qa] * cW64[qb] * h * h;
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
          const double N = cS64[3 * qa + a] * cS64[3 * qb + b];
          for (int p = 0; p < 5; ++p) fe[p][a + 3 * b] += w * dq[p] * N;
        }
    }
  const uint32_t dmask = dirichlet_mask(ug, i, j, k);
  const int64_t base = 2 * int64_t(i) + ug.sx * (2 * int64_t(j)) + ug.sy * (2 * int64_t(k) + 2);
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) {
      if ((dmask >> (a + 3 * b + 18)) & 1u) continue;
      const int64_t id = base + a + ug.sx * b;
      atomicAdd(f + id, fe[0][a + 3 * b]);
      if (dF)
        for (int p = 1; p < 5; ++p) atomicAdd(dF + (p - 1) * ug.n_dofs + id, fe[p][a + 3 * b]);
    }
}

// dJ/dk_q = -lambda^T (dA/dk_q) theta = -w_q h grad_ref(lambda) . grad_ref(theta)
__global__ void k_grad_kq(UniformGeom ug, const double* lam, const double* th, double* out) {
  Loc L;
  OctGeom og{};
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (!natural_cell<false>(ug, og, t, L)) return;
  double U[27], V[27];
  gather_uniform<double>(lam, L.base, ug.sx, ug.sy, 0u, U);
  gather_uniform<double>(th, L.base, ug.sx, ug.sy, 0u, V);
  to_qpoints<double>(U);
  to_qpoints<double>(V);
#pragma unroll
  for (int qc = 0; qc < 3; ++qc)
#pragma unroll
    for (int qb = 0; qb < 3; ++qb)
#pragma unroll
      for (int qa = 0; qa < 3; ++qa) {
        const int q = qa + 3 * qb + 9 * qc;
        double ax, ay, az, bx, by, bz;
        grad_at<double>(U, qa, qb, qc, ax, ay, az);
        grad_at<double>(V, qa, qb, qc, bx, by, bz);
        out[L.cell * 27 + q] = -cW364[q] * L.h * (ax * bx + ay * by + az * bz);
      }
}

inline int blocks(int64_t n, int b) { return int((n + b - 1) / b); }

}  // namespace

mf_status launch_scalar_qtables(mf_ctx* ctx, const mf_dofmap* m, int kind, const double* field, const double* kq_user,
                                const double* beta, double k0, double k_slope, double a_l, double a_g, int hv,
                                double eps, double rhocp, double* qc64, float* qc32, double* qv64, float* qv32,
                                const double* rhocp_q, const double* beta_q, double dt, double* qm64, float* qm32) {
  MF_CUDA_TRY(upload_tables_here());
  UniformGeom ug = m->uniform ? uniform_geom(m) : UniformGeom{};
  OctGeom og = oct_geom(m);
  const int64_t ncp = m->n_cells;
  if (m->uniform)
    k_scalar_qtables<false><<<blocks(m->n_cells, 128), 128, 0, ctx->stream>>>(
        ug, og, kind, field, kq_user, beta, m->n_dofs, k0, k_slope, a_l, a_g, hv, eps, rhocp, ncp, qc64, qc32, qv64, qv32,
        rhocp_q, beta_q, dt, qm64, qm32);
  else
    k_scalar_qtables<true><<<blocks(m->n_cells, 128), 128, 0, ctx->stream>>>(
        ug, og, kind, field, kq_user, beta, m->n_dofs, k0, k_slope, a_l, a_g, hv, eps, rhocp, ncp, qc64, qc32, qv64, qv32,
        rhocp_q, beta_q, dt, qm64, qm32);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

mf_status launch_oseen_qtables(mf_ctx* ctx, const mf_dofmap* mu, const double* phi, const double* beta, double rho_l,
                               double rho_g, double mu_l, double mu_g, int hv, double eps, double* r64, float* r32,
                               double* m64, float* m32, double* b64, float* b32) {
  MF_CUDA_TRY(upload_tables_here());
  UniformGeom ug = uniform_geom(mu);
  k_oseen_qtables<<<blocks(mu->n_cells, 128), 128, 0, ctx->stream>>>(ug, phi, beta, rho_l, rho_g, mu_l, mu_g, hv, eps,
                                                                      r64, r32, m64, m32, b64, b32);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

mf_status launch_oseen_fold(mf_ctx* ctx, const mf_dofmap* mu, double sigma, const double* rho, const double* muq,
                            const double* kd, const double* beta, double* cm64, float* cm32, double* cb64,
                            float* cb32, double* cv64, float* cv32) {
  MF_CUDA_TRY(upload_tables_here());
  const int64_t nc = mu->n_cells;
  k_oseen_fold<<<blocks(27 * nc, 256), 256, 0, ctx->stream>>>(nc, mu->mesh->h0, sigma, rho, muq, kd, beta, cm64, cm32,
                                                              cb64, cb32, cv64, cv32);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

mf_status launch_oseen_ext_tables(mf_ctx* ctx, const mf_dofmap* mu, const mf_op_params& p, const double* phi,
                                  const double* T, double* rho64, float* rho32, double* muq64, float* muq32,
                                  double* kd64, float* kd32, double* nrm64, float* nrm32) {
  MF_CUDA_TRY(upload_tables_here());
  UniformGeom ug = uniform_geom(mu);
  k_oseen_ext_tables<<<blocks(mu->n_cells, 128), 128, 0, ctx->stream>>>(
      ug, phi, T, p.heaviside, p.eps, p.oseen_flags, p.rho_l, p.rho_g, p.rho_s, p.mu_l, p.mu_g, p.mu_s, p.t_solidus,
      p.t_liquidus, p.darcy_c, p.darcy_b, rho64, rho32, muq64, muq32, kd64, kd32, nrm64, nrm32);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

mf_status launch_scalar_diag(mf_ctx* ctx, const mf_dofmap* m, int kind, bool beta, const ScalarArgs<double>& a,
                             double* diag) {
  MF_CUDA_TRY(upload_tables_here());
  MF_CUDA_TRY(cudaMemsetAsync(diag, 0, sizeof(double) * m->n_dofs, ctx->stream));
  UniformGeom ug = m->uniform ? uniform_geom(m) : UniformGeom{};
  OctGeom og = oct_geom(m);
  const int64_t nfree = m->uniform ? m->n_cells : m->n_unconstrained;
  if (m->uniform)
    k_scalar_diag<false><<<blocks(nfree, 128), 128, 0, ctx->stream>>>(a, kind, beta, ug, og, nfree, diag);
  else if (nfree > 0)
    k_scalar_diag<true><<<blocks(nfree, 128), 128, 0, ctx->stream>>>(a, kind, beta, ug, og, nfree, diag);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  if (!m->uniform && m->n_constrained_cells > 0) {
    const int64_t nc = m->n_constrained_cells;
    if (beta) return fail(MF_EUNSUPPORTED, "convection on hanging-node meshes");
    switch (kind) {
      case K_HELM: k_scalar_diag_constrained<K_HELM, false><<<blocks(nc, 32), 32, 0, ctx->stream>>>(a, og, nfree, nc, diag); break;
      case K_HEAT: k_scalar_diag_constrained<K_HEAT, false><<<blocks(nc, 32), 32, 0, ctx->stream>>>(a, og, nfree, nc, diag); break;
      case K_REINIT: k_scalar_diag_constrained<K_REINIT, false><<<blocks(nc, 32), 32, 0, ctx->stream>>>(a, og, nfree, nc, diag); break;
      default: return fail(MF_EINVAL, "diagonal of this operator kind");
    }
    ctx->launches++;
    MF_CUDA_TRY(cudaGetLastError());
  }
  const int64_t nd = int64_t(m->dirichlet_list.size());
  if (nd) {
    k_set_dirichlet<<<blocks(nd, 256), 256, 0, ctx->stream>>>(diag, m->d_dir_list.as<int32_t>(), nd, 1.0, 1);
    ctx->launches++;
    MF_CUDA_TRY(cudaGetLastError());
  }
  return MF_OK;
}

mf_status launch_oseen_blockdiag(mf_ctx* ctx, const mf_dofmap* mu, const mf_dofmap* mp, const OseenArgs<double>& a,
                                 double* blk, double* pdiag) {
  MF_CUDA_TRY(upload_tables_here());
  UniformGeom ug = uniform_geom(mu);
  const int64_t nu = mu->n_dofs, np = mp->n_dofs;
  DevBuf tmp;
  MF_TRY(tmp.alloc(sizeof(double) * 2 * np));
  double* pm = tmp.as<double>();
  double* pk = pm + np;
  MF_CUDA_TRY(cudaMemsetAsync(blk, 0, sizeof(double) * 9 * nu, ctx->stream));
  MF_CUDA_TRY(cudaMemsetAsync(pm, 0, sizeof(double) * 2 * np, ctx->stream));
  k_oseen_blocks<<<blocks(mu->n_cells, 64), 64, 0, ctx->stream>>>(a, ug, blk, pm, pk);
  DevBuf dflag;
  if (!mu->dirichlet_list.empty()) MF_TRY(dflag.upload(mu->dirichlet, ctx->stream));
  k_invert_blocks<<<blocks(nu, 256), 256, 0, ctx->stream>>>(blk, dflag.as<uint8_t>(), nu);
  k_pressure_scaling<double><<<blocks(np, 256), 256, 0, ctx->stream>>>(pm, pk, pdiag, np);
  ctx->launches += 3;
  MF_CUDA_TRY(cudaGetLastError());
  MF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return MF_OK;
}

mf_status launch_oseen_blockdiag32(mf_ctx* ctx, const mf_dofmap* mu, const mf_dofmap* mp, const OseenArgs<float>& a,
                                   float* blk, float* pinv) {
  MF_CUDA_TRY(upload_tables_here());
  if (!mu->uniform) return fail(MF_EUNSUPPORTED, "Oseen blocks: uniform meshes");
  UniformGeom ug = uniform_geom(mu);
  const int64_t nu = mu->n_dofs, np = mp->n_dofs;
  DevBuf tmp;
  MF_TRY(tmp.alloc(sizeof(float) * 2 * np));
  float* pm = tmp.as<float>();
  float* pk = pm + np;
  MF_CUDA_TRY(cudaMemsetAsync(blk, 0, sizeof(float) * 9 * nu, ctx->stream));
  MF_CUDA_TRY(cudaMemsetAsync(pm, 0, sizeof(float) * 2 * np, ctx->stream));
  k_oseen_blocks32<<<blocks(mu->n_cells, kBlk32), kBlk32, 0, ctx->stream>>>(a, ug, blk, pm, pk);
  k_invert_blocks_soa32<<<blocks(nu, 256), 256, 0, ctx->stream>>>(blk, nu);
  const int64_t nd = int64_t(mu->dirichlet_list.size());
  if (nd) k_identity_blocks_soa32<<<blocks(nd, 256), 256, 0, ctx->stream>>>(blk, mu->d_dir_list.as<int32_t>(), nd, nu);
  k_pressure_scaling<float><<<blocks(np, 256), 256, 0, ctx->stream>>>(pm, pk, pinv, np);
  ctx->launches += nd ? 4 : 3;
  MF_CUDA_TRY(cudaGetLastError());
  MF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));  // before the scratch is freed
  return MF_OK;
}

mf_status launch_laser(mf_ctx* ctx, const mf_dofmap* m, const double lz[5], double* f, double* dF) {
  MF_CUDA_TRY(upload_tables_here());
  if (!m->uniform) return fail(MF_EUNSUPPORTED, "laser load on octree maps");
  UniformGeom ug = uniform_geom(m);
  MF_CUDA_TRY(cudaMemsetAsync(f, 0, sizeof(double) * m->n_dofs, ctx->stream));
  if (dF) MF_CUDA_TRY(cudaMemsetAsync(dF, 0, sizeof(double) * 4 * m->n_dofs, ctx->stream));
  k_laser<<<blocks(int64_t(ug.nx) * ug.ny, 128), 128, 0, ctx->stream>>>(ug, m->mesh->lo[0], m->mesh->lo[1], lz[0], lz[1],
                                                                         lz[2], lz[3], lz[4], f, dF);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

mf_status launch_grad_kq(mf_ctx* ctx, const mf_dofmap* m, const double* lam, const double* theta, double* out) {
  MF_CUDA_TRY(upload_tables_here());
  if (!m->uniform) return fail(MF_EUNSUPPORTED, "k_q gradient on octree maps");
  UniformGeom ug = uniform_geom(m);
  k_grad_kq<<<blocks(m->n_cells, 128), 128, 0, ctx->stream>>>(ug, lam, theta, out);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

}  // namespace mf
