// Double-float apply of the scalar Q2 operators on uniform meshes: Helmholtz and the implicit heat
// step without convection (Section 2.3 coefficients, Appendix B matrix-free evaluation), with the
// conductivity (or a(phi)) tabulated per Gauss point and a constant value coefficient.
//
// Vectors stay fp64 in HBM; in the kernel every value is a pair of floats hi + lo (48-bit
// significand) and every operation is an error-free fp32 transformation on the fp32 pipes, which
// GB300 runs at 64 times its fp64 rate (Dekker's product through the FMA residual, Knuth's two-sum;
// Joldes, Muller and Popescu, ACM TOMS 2017, bound these "double-word" algorithms).  Pairs are
// carried unnormalised through each contraction (|lo| a few ulp(hi) at most) and renormalised at its
// end; the error of a sum stays below a few 2^-47 (|a| + |b|), so results agree with the fp64 apply
// to a few 1e-14 of |A||u| componentwise.  Doubles enter and leave the kernel by bit manipulation
// (GB300 converts between fp64 and fp32 only at its fp64 rate), scaled by one power of two per warp so
// that the warp's largest input lies in [1, 2): any fp64 magnitude is kept to 47 bits relative to that
// largest input of the warp's 8 x 4 cells; inputs more than 2^126 below it count as zero.
//
// One thread per cell in 8 x 4 x 4 bricks (the warp-level scatter of the fp64 kernels).  The cell's
// 27 values at the Gauss points are parked in the thread's own column of shared memory, and the
// test side is accumulated one z-plane at a time, so no more than 27 value pairs are live in
// registers (96 registers, five blocks of 128 threads per SM) and enough warps stay resident to cover
// the dependent chains of the double-float arithmetic.  No thread reads another thread's column:
// no barrier is needed.
#include "df_pairs.cuh"

namespace mf {

MF_DEFINE_TABLE_UPLOAD

UniformGeom uniform_geom(const mf_dofmap* m);

namespace {

struct DfArgs {
  const double* src;
  double* dst;
  int nrhs;         // right-hand sides, one per blockIdx.y
  int64_t ld;       // distance between right-hand sides
  const float* ch;  // [27][ncells] high parts of w_q h c_q (c: conductivity or a(phi) at Gauss point q)
  const float* cl;  // [27][ncells] low parts
  int64_t ncells;
  float wmh[27], wml[27];  // w_q m h^3 (m: value coefficient), high and low parts
};

__device__ __forceinline__ dd shfl_down_dd(dd v, int d) {
  return {__shfl_down_sync(0xffffffffu, v.h, d), __shfl_down_sync(0xffffffffu, v.l, d)};
}

// Scatter-add of a warp of the 8 x 4 x 4 brick: the faces shared by x and y neighbours inside the
// warp are folded by shuffles on the pairs (all lanes share one scale), then every node is added to
// memory once per warp as the double hi 2^bias + lo 2^bias.  Every lane calls this; inactive lanes
// pass zeros.
__device__ __forceinline__ void scatter_dd_warp(double* __restrict__ dst, int64_t base, int64_t sx, int64_t sy,
                                                uint32_t dmask, dd* R, bool active, int bias) {
  const int xl = threadIdx.x & 7, yl = (threadIdx.x >> 3) & 3;
#pragma unroll
  for (int bc = 0; bc < 9; ++bc) {
    const int o = 3 * (bc % 3) + 9 * (bc / 3);
    const dd w = shfl_down_dd(R[o], 1);
    if (xl < 7) R[o + 2] = dd_add(R[o + 2], w);
  }
#pragma unroll
  for (int ac = 0; ac < 9; ++ac) {
    const int a = ac % 3, o = a + 9 * (ac / 3);
    const dd w = shfl_down_dd((a == 0 && xl > 0) ? dd{0.f, 0.f} : R[o], 8);
    if (yl < 3) R[o + 6] = dd_add(R[o + 6], w);
  }
  if (!active) return;
  asm volatile("" : "+l"(base), "+l"(sx), "+l"(sy));
  double* __restrict__ d = dst + base;
#pragma unroll
  for (int l = 0; l < 27; ++l) {
    const int a = l % 3, b = (l / 3) % 3, c = l / 9;
    if ((a == 0 && xl > 0) || (b == 0 && yl > 0) || ((dmask >> l) & 1u)) continue;
    atomicAdd(d + a + sx * b + sy * c, f2d_bits(R[l].h, bias) + f2d_bits(R[l].l, bias));
  }
}

constexpr int kThreads = 128;

// The test side R = w m h^3 u + h D^T (w c grad u) is split by direction.  First the z fluxes
// F_z = (w h c) d_z u at all 27 points (one register pair each); then plane by plane (z = const) the
// plane's 9 outputs: value term, the z part sum_{q'} D[q'][qc] F_z(q'), and the x and y parts from
// the plane's own values, followed by the plane-local x and y transposed sweeps.  Only 9
// accumulators are live at a time; the swept plane is parked in the shared-memory slots of the
// plane's Gauss-point values (no longer needed), and the z sweep runs on all 27 at the end.
__global__ void __launch_bounds__(kThreads, 5) k_scalar_df_uniform(DfArgs A, UniformGeom ug) {
  __shared__ float sh[27][kThreads], sl[27][kThreads];
  int i, j, k;
  const bool active = brick_cell(ug, i, j, k);
  const int t = threadIdx.x;
  const int64_t cell = active ? i + int64_t(ug.nx) * (j + int64_t(ug.ny) * k) : 0;
  const int64_t base = active ? 2 * int64_t(i) + ug.sx * (2 * int64_t(j)) + ug.sy * (2 * int64_t(k)) : 0;
  const uint32_t dmask = active ? dirichlet_mask(ug, i, j, k) : 0u;
  int bias = 0;
  {
    // gather (Dirichlet nodes read as 0) and interpolate to the Gauss points; right-hand side
    // blockIdx.y
    dd U[27];
    const double* __restrict__ s = A.src + int64_t(blockIdx.y) * A.ld + base;
    double X[27];
    int emax = 0;
#pragma unroll
    for (int l = 0; l < 27; ++l) {
      const int a = l % 3, b = (l / 3) % 3, c = l / 9;
      const double v = active ? __ldg(s + a + ug.sx * b + ug.sy * c) : 0.0;
      X[l] = ((dmask >> l) & 1u) ? 0.0 : v;
      emax = max(emax, (__double2hiint(X[l]) >> 20) & 0x7FF);
    }
    // one power-of-two scale per warp (its 8 x 4 cells share faces folded below): the largest
    // input maps to [1, 2)
    emax = int(__reduce_max_sync(0xffffffffu, unsigned(emax)));
    bias = emax ? emax - 1023 : 0;
#pragma unroll
    for (int l = 0; l < 27; ++l) U[l] = d2dd_bits(X[l], bias);
    dsweep<0>(U);
    dsweep<1>(U);
    dsweep<2>(U);
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      sh[q][t] = U[q].h;
      sl[q][t] = U[q].l;
    }
  }
  auto Uq = [&](int q) { return dd{sh[q][t], sl[q][t]}; };
  auto coef = [&](int q) {
    return active ? dd{__ldg(A.ch + q * A.ncells + cell), __ldg(A.cl + q * A.ncells + cell)} : dd{0.f, 0.f};
  };
  dd FZ[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const int qc = q / 9, bz = q - 9 * qc;
    FZ[q] = dd_norm(dd_mul(coef(q), ddline(qc, Uq(bz), Uq(bz + 9), Uq(bz + 18))));
  }
#pragma unroll
  for (int qc = 0; qc < 3; ++qc) {
    dd R[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      const int q = p + 9 * qc;
      dd acc = dd_mul(dd{A.wmh[q], A.wml[q]}, Uq(q));
#pragma unroll
      for (int c2 = 0; c2 < 3; ++c2)
        if (c2 != 1 || qc != 1) acc = dd_fma(acc, cD(c2, qc), FZ[p + 9 * c2]);
      R[p] = acc;
    }
#pragma unroll
    for (int qb = 0; qb < 3; ++qb)
#pragma unroll
      for (int qa = 0; qa < 3; ++qa) {
        const int p = qa + 3 * qb, q = p + 9 * qc;
        const int bx = q - qa, by = q - 3 * qb;
        const dd gx = ddline(qa, Uq(bx), Uq(bx + 1), Uq(bx + 2));
        const dd gy = ddline(qb, Uq(by), Uq(by + 3), Uq(by + 6));
        const dd cq = coef(q);
        const dd fx = dd_mul(cq, gx), fy = dd_mul(cq, gy);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          if (qa != 1 || m != 1) R[p - qa + m] = dd_fma(R[p - qa + m], cD(qa, m), fx);
          if (qb != 1 || m != 1) R[p - 3 * qb + 3 * m] = dd_fma(R[p - 3 * qb + 3 * m], cD(qb, m), fy);
        }
      }
#pragma unroll
    for (int p = 0; p < 9; ++p) R[p] = dd_norm(R[p]);
#pragma unroll
    for (int b = 0; b < 3; ++b) {   // x, transposed
      const dd u0 = R[3 * b], u1 = R[3 * b + 1], u2 = R[3 * b + 2];
      R[3 * b] = dd_norm(dd_add(dd_mul(cS(0, 0), u0), dd_mul(cS(2, 0), u2)));
      R[3 * b + 1] = dd_norm(dd_add(dd_add(dd_mul(cS(0, 1), u0), u1), dd_mul(cS(2, 1), u2)));
      R[3 * b + 2] = dd_norm(dd_add(dd_mul(cS(0, 2), u0), dd_mul(cS(2, 2), u2)));
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {   // y, transposed
      const dd u0 = R[a], u1 = R[a + 3], u2 = R[a + 6];
      R[a] = dd_norm(dd_add(dd_mul(cS(0, 0), u0), dd_mul(cS(2, 0), u2)));
      R[a + 3] = dd_norm(dd_add(dd_add(dd_mul(cS(0, 1), u0), u1), dd_mul(cS(2, 1), u2)));
      R[a + 6] = dd_norm(dd_add(dd_mul(cS(0, 2), u0), dd_mul(cS(2, 2), u2)));
    }
    // the plane's values at the Gauss points are no longer needed: park the partial result there
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      sh[p + 9 * qc][t] = R[p].h;
      sl[p + 9 * qc][t] = R[p].l;
    }
  }
  dd R[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) R[q] = Uq(q);
  dsweep_t<2>(R);
#pragma unroll
  for (int q = 0; q < 27; ++q)
    if (!active) R[q] = dd{0.f, 0.f};
  scatter_dd_warp(A.dst + int64_t(blockIdx.y) * A.ld, base, ug.sx, ug.sy, dmask, R, active, bias);
}

// The heat operator with convection, rho_cp (beta . grad u) v, and its transpose, in the same plane
// structure.  cb_d = w_q h^2 rho_cp beta_d at the Gauss points (float pairs, [d][q][cell]).  Transpose:
// the term adds cb_d u to the gradient-test fluxes (F_z in the z-flux pass, F_x and F_y in the plane
// loop).  Forward: it is a value-test term, cb . grad u: its x and y parts are added where the plane
// loop forms grad u, its z part is formed with the z fluxes and parked in a second shared-memory
// column (dynamic shared memory, four blocks per SM).
struct DfConvArgs {
  const double* src;
  double* dst;
  int nrhs;
  int64_t ld;
  const float* ch;  // [27][ncells] w_q h c_q
  const float* cl;
  const float* bh;  // [3][27][ncells] w_q h^2 rho_cp beta_d
  const float* bl;
  int64_t ncells;
  float wmh[27], wml[27];
  const float* mh;  // QM: [27][ncells] w_q h^3 m_q per Gauss point (m_q = rho_cp,q / dt) instead of wmh
  const float* ml;
};

template <bool TR, bool QM>
__global__ void __launch_bounds__(kThreads, TR ? 5 : 4) k_scalar_df_uniform_conv(DfConvArgs A, UniformGeom ug) {
  extern __shared__ float conv_smem[];
  float(*sh)[kThreads] = reinterpret_cast<float(*)[kThreads]>(conv_smem);
  float(*sl)[kThreads] = reinterpret_cast<float(*)[kThreads]>(conv_smem + 27 * kThreads);
  float(*zh)[kThreads] = reinterpret_cast<float(*)[kThreads]>(conv_smem + 54 * kThreads);
  float(*zl)[kThreads] = reinterpret_cast<float(*)[kThreads]>(conv_smem + 81 * kThreads);
  int i, j, k;
  const bool active = brick_cell(ug, i, j, k);
  const int t = threadIdx.x;
  const int64_t cell = active ? i + int64_t(ug.nx) * (j + int64_t(ug.ny) * k) : 0;
  const int64_t base = active ? 2 * int64_t(i) + ug.sx * (2 * int64_t(j)) + ug.sy * (2 * int64_t(k)) : 0;
  const uint32_t dmask = active ? dirichlet_mask(ug, i, j, k) : 0u;
  int bias = 0;
  {
    dd U[27];
    const double* __restrict__ s = A.src + int64_t(blockIdx.y) * A.ld + base;
    double X[27];
    int emax = 0;
#pragma unroll
    for (int l = 0; l < 27; ++l) {
      const int a = l % 3, b = (l / 3) % 3, c = l / 9;
      const double v = active ? __ldg(s + a + ug.sx * b + ug.sy * c) : 0.0;
      X[l] = ((dmask >> l) & 1u) ? 0.0 : v;
      emax = max(emax, (__double2hiint(X[l]) >> 20) & 0x7FF);
    }
    emax = int(__reduce_max_sync(0xffffffffu, unsigned(emax)));
    bias = emax ? emax - 1023 : 0;
#pragma unroll
    for (int l = 0; l < 27; ++l) U[l] = d2dd_bits(X[l], bias);
    dsweep<0>(U);
    dsweep<1>(U);
    dsweep<2>(U);
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      sh[q][t] = U[q].h;
      sl[q][t] = U[q].l;
    }
  }
  auto Uq = [&](int q) { return dd{sh[q][t], sl[q][t]}; };
  auto coef = [&](int q) {
    return active ? dd{__ldg(A.ch + q * A.ncells + cell), __ldg(A.cl + q * A.ncells + cell)} : dd{0.f, 0.f};
  };
  auto bet = [&](int d, int q) {
    const int64_t o = (d * 27 + q) * A.ncells + cell;
    return active ? dd{__ldg(A.bh + o), __ldg(A.bl + o)} : dd{0.f, 0.f};
  };
  dd FZ[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const int qc = q / 9, bz = q - 9 * qc;
    const dd gz = ddline(qc, Uq(bz), Uq(bz + 9), Uq(bz + 18));
    dd f = dd_mul(coef(q), gz);
    if (TR) {
      f = dd_fma(f, bet(2, q), Uq(q));
    } else {
      const dd cz = dd_norm(dd_mul(bet(2, q), gz));
      zh[q][t] = cz.h;
      zl[q][t] = cz.l;
    }
    FZ[q] = dd_norm(f);
  }
#pragma unroll
  for (int qc = 0; qc < 3; ++qc) {
    dd R[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      const int q = p + 9 * qc;
      const dd wm = !QM ? dd{A.wmh[q], A.wml[q]}
                        : active ? dd{__ldg(A.mh + q * A.ncells + cell), __ldg(A.ml + q * A.ncells + cell)}
                                 : dd{0.f, 0.f};
      dd acc = dd_mul(wm, Uq(q));
      if (!TR) acc = dd_add(acc, dd{zh[q][t], zl[q][t]});
#pragma unroll
      for (int c2 = 0; c2 < 3; ++c2)
        if (c2 != 1 || qc != 1) acc = dd_fma(acc, cD(c2, qc), FZ[p + 9 * c2]);
      R[p] = acc;
    }
#pragma unroll
    for (int qb = 0; qb < 3; ++qb)
#pragma unroll
      for (int qa = 0; qa < 3; ++qa) {
        const int p = qa + 3 * qb, q = p + 9 * qc;
        const int bx = q - qa, by = q - 3 * qb;
        const dd gx = ddline(qa, Uq(bx), Uq(bx + 1), Uq(bx + 2));
        const dd gy = ddline(qb, Uq(by), Uq(by + 3), Uq(by + 6));
        const dd cq = coef(q);
        dd fx = dd_mul(cq, gx), fy = dd_mul(cq, gy);
        if (TR) {
          const dd u = Uq(q);
          fx = dd_fma(fx, bet(0, q), u);
          fy = dd_fma(fy, bet(1, q), u);
        } else {
          R[p] = dd_fma(dd_fma(R[p], bet(0, q), gx), bet(1, q), gy);
        }
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          if (qa != 1 || m != 1) R[p - qa + m] = dd_fma(R[p - qa + m], cD(qa, m), fx);
          if (qb != 1 || m != 1) R[p - 3 * qb + 3 * m] = dd_fma(R[p - 3 * qb + 3 * m], cD(qb, m), fy);
        }
      }
#pragma unroll
    for (int p = 0; p < 9; ++p) R[p] = dd_norm(R[p]);
#pragma unroll
    for (int b = 0; b < 3; ++b) {   // x, transposed
      const dd u0 = R[3 * b], u1 = R[3 * b + 1], u2 = R[3 * b + 2];
      R[3 * b] = dd_norm(dd_add(dd_mul(cS(0, 0), u0), dd_mul(cS(2, 0), u2)));
      R[3 * b + 1] = dd_norm(dd_add(dd_add(dd_mul(cS(0, 1), u0), u1), dd_mul(cS(2, 1), u2)));
      R[3 * b + 2] = dd_norm(dd_add(dd_mul(cS(0, 2), u0), dd_mul(cS(2, 2), u2)));
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {   // y, transposed
      const dd u0 = R[a], u1 = R[a + 3], u2 = R[a + 6];
      R[a] = dd_norm(dd_add(dd_mul(cS(0, 0), u0), dd_mul(cS(2, 0), u2)));
      R[a + 3] = dd_norm(dd_add(dd_add(dd_mul(cS(0, 1), u0), u1), dd_mul(cS(2, 1), u2)));
      R[a + 6] = dd_norm(dd_add(dd_mul(cS(0, 2), u0), dd_mul(cS(2, 2), u2)));
    }
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      sh[p + 9 * qc][t] = R[p].h;
      sl[p + 9 * qc][t] = R[p].l;
    }
  }
  dd R[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) R[q] = Uq(q);
  dsweep_t<2>(R);
#pragma unroll
  for (int q = 0; q < 27; ++q)
    if (!active) R[q] = dd{0.f, 0.f};
  scatter_dd_warp(A.dst + int64_t(blockIdx.y) * A.ld, base, ug.sx, ug.sy, dmask, R, active, bias);
}

// ---------------------------------------------------------------------------------------------
// Double-float Oseen apply (Q2 velocity / Q1 pressure, uniform mesh, folded Gauss-point coefficients
// cm = w h^3 sigma rho, cv = w h mu, cb = w h^2 rho beta as float pairs).  A block of three warps
// owns an 8 x 4 x 1 brick of 32 cells; warp c evaluates the test functions of velocity component c
// for the brick's cells, reading the other components' Gauss-point values (for the symmetric part of
// the stress) from shared memory.  Velocity and pressure inputs are scaled by their own powers of two
// (the block's largest velocity / pressure input in [1, 2)); the coefficients are rescaled by exact
// powers of two so that every velocity test term is accumulated in the larger of the two scales.

struct DfOseenArgs {
  const double* src;
  double* dst;
  int64_t nu;                  // velocity DoFs per component (pressure block starts at 3 nu)
  const float *cmh, *cml;      // [27][ncells]
  const float *cvh, *cvl;      // [27][ncells]
  const float *cbh, *cbl;      // [3][27][ncells]
  int64_t ncells;
  float pwh[27][8], pwl[27][8];  // -h^2 w_q psi_n(x_q): pressure / continuity coupling
  float wph[3][2], wpl[3][2];    // 1D w_g psi_a(g) (Q1 hat a at Gauss point g)
  float mh2h, mh2l;              // -h^2
  const float *nrh, *nrl;        // melt-pool trace correction: interface normal per Gauss point, [3][27][ncells]
};

__device__ __forceinline__ dd dd_scale(dd a, float s) { return {a.h * s, a.l * s}; }   // s a power of two
__device__ __forceinline__ float pow2f(int e) {  // 2^e for e in [-126, 127]; 0 below
  return e < -126 ? 0.f : __uint_as_float(unsigned(min(e, 127) + 127) << 23);
}

// EXT: the melt-pool trace correction -2 mu (div u) n (x) n : grad v adds t n_C n_d to the flux of
// component C in direction d, t = -2 cv div u (the Darcy term sits in cm)
template <bool EXT>
__device__ __forceinline__ void oseen_df_component(const int C, const DfOseenArgs& A, const UniformGeom& ug,
                                                   float (*sh)[27][32],
                                                   float (*sl)[27][32], float (*ph)[32], float (*pl)[32],
                                                   float (*ah)[32], float (*al)[32], int lane, bool active,
                                                   int64_t cell, int64_t base, uint32_t dmask, float su, int bias_out,
                                                   int bias_u, double* pdst, int64_t pbase, int64_t px, int64_t pxy) {
  auto V = [&](int e, int q) { return dd{sh[e][q][lane], sl[e][q][lane]}; };
  auto load = [&](const float* hh, const float* ll, int64_t off) {
    return active ? dd_scale(dd{__ldg(hh + off), __ldg(ll + off)}, su) : dd{0.f, 0.f};
  };
  const int64_t nc = A.ncells;
  // derivative of component e along direction d at Gauss point (qa, qb, qc)
  auto deriv = [&](int e, int d, int qa, int qb, int qc) {
    const int q = qa + 3 * qb + 9 * qc;
    if (d == 0) return ddline(qa, V(e, q - qa), V(e, q - qa + 1), V(e, q - qa + 2));
    if (d == 1) return ddline(qb, V(e, q - 3 * qb), V(e, q - 3 * qb + 3), V(e, q - 3 * qb + 6));
    return ddline(qc, V(e, q - 9 * qc), V(e, q - 9 * qc + 9), V(e, q - 9 * qc + 18));
  };
  // derivative of component e along direction C (a run-time direction, the same for the whole warp)
  auto derivC = [&](int e, int qa, int qb, int qc) {
    const int q = qa + 3 * qb + 9 * qc;
    const int qd = C == 0 ? qa : (C == 1 ? qb : qc), st = C == 0 ? 1 : (C == 1 ? 3 : 9);
    const int b0 = q - qd * st;
    return ddline(qd, V(e, b0), V(e, b0 + st), V(e, b0 + 2 * st));
  };
  // interface normal component d at Gauss point q (unscaled: a unit vector)
  auto nrm = [&](int d, int q) {
    const int64_t o = (d * 27 + q) * nc + cell;
    return active ? dd{__ldg(A.nrh + o), __ldg(A.nrl + o)} : dd{0.f, 0.f};
  };
  // t n_C = -2 cv (div u) n_C at Gauss point (qa, qb, qc)
  auto trace_tn = [&](dd cv, int qa, int qb, int qc) {
    const int q = qa + 3 * qb + 9 * qc;
    const dd div = dd_add(dd_add(deriv(0, 0, qa, qb, qc), deriv(1, 1, qa, qb, qc)), deriv(2, 2, qa, qb, qc));
    const dd m2cv = dd{-2.f * cv.h, -2.f * cv.l};
    return dd_mul(dd_mul(m2cv, dd_norm(div)), nrm(C, q));
  };
  // test flux of component C in direction d: cv (d_d u_C + d_C u_d), plus the pressure on the diagonal
  auto flux = [&](int d, dd cv, dd gd, int qa, int qb, int qc) {
    const int q = qa + 3 * qb + 9 * qc;
    if (d == C) return dd_add(dd_mul(dd_add(cv, cv), gd), dd{ph[q][lane], pl[q][lane]});
    return dd_mul(cv, dd_add(gd, derivC(d, qa, qb, qc)));
  };
  // z part of the test side, column by column, into this thread's accumulator column:
  // Z(qa, qb, qc) = sum_{qc'} D[qc'][qc] F_z(qa, qb, qc')
#pragma unroll 1
  for (int p = 0; p < 9; ++p) {
    const int qa = p % 3, qb = p / 3;
    dd fz[3];
#pragma unroll
    for (int qc = 0; qc < 3; ++qc) {
      const dd cv = load(A.cvh, A.cvl, (p + 9 * qc) * nc + cell);
      dd f = flux(2, cv, deriv(C, 2, qa, qb, qc), qa, qb, qc);
      if (EXT) f = dd_fma(f, trace_tn(cv, qa, qb, qc), nrm(2, p + 9 * qc));
      fz[qc] = dd_norm(f);
    }
#pragma unroll
    for (int qc = 0; qc < 3; ++qc) {
      dd acc = dd{0.f, 0.f};
#pragma unroll
      for (int c2 = 0; c2 < 3; ++c2)
        if (c2 != 1 || qc != 1) acc = dd_fma(acc, cD(c2, qc), fz[c2]);
      ah[p + 9 * qc][lane] = acc.h;
      al[p + 9 * qc][lane] = acc.l;
    }
  }
  // plane by plane: value terms and the x and y parts, then the transposed x and y sweeps
#pragma unroll 1
  for (int qc = 0; qc < 3; ++qc) {
    dd P[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) P[p] = dd{ah[p + 9 * qc][lane], al[p + 9 * qc][lane]};
#pragma unroll
    for (int qb = 0; qb < 3; ++qb)
#pragma unroll
      for (int qa = 0; qa < 3; ++qa) {
        const int p = qa + 3 * qb, q = p + 9 * qc;
        const dd cm = load(A.cmh, A.cml, q * nc + cell), cv = load(A.cvh, A.cvl, q * nc + cell);
        const dd gx = deriv(C, 0, qa, qb, qc), gy = deriv(C, 1, qa, qb, qc), gz = deriv(C, 2, qa, qb, qc);
        // sigma rho u_C + rho beta . grad u_C
        dd v = dd_mul(cm, V(C, q));
        v = dd_fma(v, load(A.cbh, A.cbl, (0 * 27 + q) * nc + cell), gx);
        v = dd_fma(v, load(A.cbh, A.cbl, (1 * 27 + q) * nc + cell), gy);
        v = dd_fma(v, load(A.cbh, A.cbl, (2 * 27 + q) * nc + cell), gz);
        P[p] = dd_add(P[p], v);
        dd fx = flux(0, cv, gx, qa, qb, qc), fy = flux(1, cv, gy, qa, qb, qc);
        if (EXT) {
          const dd tn = trace_tn(cv, qa, qb, qc);
          fx = dd_fma(fx, tn, nrm(0, q));
          fy = dd_fma(fy, tn, nrm(1, q));
        }
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          if (qa != 1 || m != 1) P[p - qa + m] = dd_fma(P[p - qa + m], cD(qa, m), fx);
          if (qb != 1 || m != 1) P[p - 3 * qb + 3 * m] = dd_fma(P[p - 3 * qb + 3 * m], cD(qb, m), fy);
        }
      }
#pragma unroll
    for (int p = 0; p < 9; ++p) P[p] = dd_norm(P[p]);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const dd u0 = P[3 * b], u1 = P[3 * b + 1], u2 = P[3 * b + 2];
      P[3 * b] = dd_norm(dd_add(dd_mul(cS(0, 0), u0), dd_mul(cS(2, 0), u2)));
      P[3 * b + 1] = dd_norm(dd_add(dd_add(dd_mul(cS(0, 1), u0), u1), dd_mul(cS(2, 1), u2)));
      P[3 * b + 2] = dd_norm(dd_add(dd_mul(cS(0, 2), u0), dd_mul(cS(2, 2), u2)));
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const dd u0 = P[a], u1 = P[a + 3], u2 = P[a + 6];
      P[a] = dd_norm(dd_add(dd_mul(cS(0, 0), u0), dd_mul(cS(2, 0), u2)));
      P[a + 3] = dd_norm(dd_add(dd_add(dd_mul(cS(0, 1), u0), u1), dd_mul(cS(2, 1), u2)));
      P[a + 6] = dd_norm(dd_add(dd_mul(cS(0, 2), u0), dd_mul(cS(2, 2), u2)));
    }
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      ah[p + 9 * qc][lane] = P[p].h;
      al[p + 9 * qc][lane] = P[p].l;
    }
  }
  {
    dd R[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) R[q] = active ? dd{ah[q][lane], al[q][lane]} : dd{0.f, 0.f};
    dsweep_t<2>(R);
    scatter_dd_warp(A.dst + C * A.nu, base, ug.sx, ug.sy, dmask, R, active, bias_out);
  }
  // continuity: -int psi_n d_C u_C, this component's share (velocity scale), added by this warp; the
  // Q1 test functions are tensor products, so the sum over the 27 points factorises into three 1D
  // contractions with w_g psi_a(g) (the factor -h^2 applied at the end)
  dd Rp[8];
#pragma unroll
  for (int n = 0; n < 8; ++n) Rp[n] = dd{0.f, 0.f};
  auto wp = [&](int g, int a) { return dd{A.wph[g][a], A.wpl[g][a]}; };
#pragma unroll 1
  for (int qc = 0; qc < 3; ++qc) {
    dd G[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) G[p] = derivC(C, p % 3, p / 3, qc);
    dd T[2][2];
#pragma unroll
    for (int na = 0; na < 2; ++na) {
      dd T1[3];
#pragma unroll
      for (int qb = 0; qb < 3; ++qb)
        T1[qb] = dd_norm(dd_add(dd_add(dd_mul(wp(0, na), G[3 * qb]), dd_mul(wp(1, na), G[3 * qb + 1])),
                                dd_mul(wp(2, na), G[3 * qb + 2])));
#pragma unroll
      for (int nb = 0; nb < 2; ++nb)
        T[na][nb] = dd_norm(dd_add(dd_add(dd_mul(wp(0, nb), T1[0]), dd_mul(wp(1, nb), T1[1])), dd_mul(wp(2, nb), T1[2])));
    }
#pragma unroll
    for (int n = 0; n < 8; ++n) Rp[n] = dd_fma(Rp[n], wp(qc, n >> 2), T[n & 1][(n >> 1) & 1]);
  }
  if (active) {
    const dd mh2{A.mh2h, A.mh2l};
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const dd r = dd_mul(mh2, dd_norm(Rp[n]));
      atomicAdd(pdst + pbase + (n & 1) + px * ((n >> 1) & 1) + pxy * (n >> 2),
                f2d_bits(r.h, bias_u) + f2d_bits(r.l, bias_u));
    }
  }
}

template <bool EXT>
__global__ void __launch_bounds__(96, 4) k_oseen_df_uniform(DfOseenArgs A, UniformGeom ug) {
  __shared__ float sh[3][27][32], sl[3][27][32];   // velocity values at the Gauss points
  __shared__ float ph[27][32], pl[27][32];         // pressure term at the Gauss points (output scale)
  __shared__ float ah[3][27][32], al[3][27][32];   // each component's test-side accumulators
  __shared__ int sE[3];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nbx = (ug.nx + 7) >> 3, nby = (ug.ny + 3) >> 2;
  const int b = blockIdx.x;
  const int i = (b % nbx) * 8 + (lane & 7), j = ((b / nbx) % nby) * 4 + (lane >> 3), k = b / (nbx * nby);
  const bool active = i < ug.nx && j < ug.ny;
  const int64_t cell = active ? i + int64_t(ug.nx) * (j + int64_t(ug.ny) * k) : 0;
  const int64_t base = active ? 2 * int64_t(i) + ug.sx * (2 * int64_t(j)) + ug.sy * (2 * int64_t(k)) : 0;
  const uint32_t dmask = active ? dirichlet_mask(ug, i, j, k) : 0u;
  const int64_t px = ug.nx + 1, pxy = px * (ug.ny + 1);
  const int64_t pbase = active ? i + px * (j + (ug.ny + 1) * int64_t(k)) : 0;
  // L2 prefetch of the coefficient tables cv (read in the z pass), cm and cb (read in the plane loop)
  // while the inputs load and the sweeps run: a brick row's 8 cells share one 32-byte sector per
  // table row, so each lane fetches that sector for its brick row and every 24th of the 270 table
  // rows (high and low parts: cv 54, cm 54, cb 162).  Fetching the normal table of the melt-pool
  // terms as well measured slower (1.57 against 1.54 ms at 64^3).
  if (j < ug.ny) {
    const int64_t row_cell = int64_t(i - (lane & 7)) + int64_t(ug.nx) * (j + int64_t(ug.ny) * k);
#pragma unroll 1
    for (int r = w * 8 + (lane & 7); r < 270; r += 24) {
      const float* t;
      int rr;
      if (r < 54) { rr = r; t = (rr & 1) ? A.cvl : A.cvh; }
      else if (r < 108) { rr = r - 54; t = (rr & 1) ? A.cml : A.cmh; }
      else { rr = r - 108; t = (rr & 1) ? A.cbl : A.cbh; }
      asm volatile("prefetch.global.L2 [%0];" ::"l"(t + int64_t(rr >> 1) * A.ncells + row_cell));
    }
  }
  // raw inputs: this warp's velocity component and the cell's 8 pressures
  double X[27], Pn[8];
  int eu = 0, ep = 0;
#pragma unroll
  for (int l = 0; l < 27; ++l) {
    const int a = l % 3, bb = (l / 3) % 3, c = l / 9;
    const double v = active ? __ldg(A.src + w * A.nu + base + a + ug.sx * bb + ug.sy * c) : 0.0;
    X[l] = ((dmask >> l) & 1u) ? 0.0 : v;
    eu = max(eu, (__double2hiint(X[l]) >> 20) & 0x7FF);
  }
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    Pn[n] = active ? __ldg(A.src + 3 * A.nu + pbase + (n & 1) + px * ((n >> 1) & 1) + pxy * (n >> 2)) : 0.0;
    ep = max(ep, (__double2hiint(Pn[n]) >> 20) & 0x7FF);
  }
  eu = int(__reduce_max_sync(0xffffffffu, unsigned(eu)));
  ep = int(__reduce_max_sync(0xffffffffu, unsigned(ep)));   // the same cells in every warp
  if (lane == 0) sE[w] = eu;
  __syncthreads();
  eu = max(sE[0], max(sE[1], sE[2]));
  const int bias_u = eu ? eu - 1023 : 0, bias_p = ep ? ep - 1023 : 0;
  const int bias_out = max(bias_u, bias_p);
  const float su = pow2f(bias_u - bias_out);   // velocity terms into the output scale
  {
    dd U[27];
#pragma unroll
    for (int l = 0; l < 27; ++l) U[l] = d2dd_bits(X[l], bias_u);
    dsweep<0>(U);
    dsweep<1>(U);
    dsweep<2>(U);
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      sh[w][q][lane] = U[q].h;
      sl[w][q][lane] = U[q].l;
    }
    // pressure term -h^2 w_q sum_n psi_n(x_q) p_n at the warp's plane of Gauss points
    dd P[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) P[n] = d2dd_bits(Pn[n], bias_p);
    const float sp = pow2f(bias_p - bias_out);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      const int q = p + 9 * w;
      dd acc = dd{0.f, 0.f};
#pragma unroll
      for (int n = 0; n < 8; ++n) acc = dd_fma(acc, dd{A.pwh[q][n], A.pwl[q][n]}, P[n]);
      acc = dd_scale(dd_norm(acc), sp);
      ph[q][lane] = acc.h;
      pl[q][lane] = acc.l;
    }
  }
  __syncthreads();
  // one code path for the three warps (component w at run time): the three instruction streams of a
  // compile-time component kept warps waiting on instruction fetch
  oseen_df_component<EXT>(w, A, ug, sh, sl, ph, pl, ah[w], al[w], lane, active, cell, base, dmask, su, bias_out,
                          bias_u, A.dst + 3 * A.nu, pbase, px, pxy);
}

__global__ void k_split_plain(const double* __restrict__ c, int64_t n, float* h, float* l) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float hi = __double2float_rn(c[t]);
  h[t] = hi;
  l[t] = __double2float_rn(c[t] - double(hi));
}

// w_q s c_q of a Gauss-point coefficient table (s = h for the conductivity, h^3 for the value
// coefficient), split into high and low float parts
__global__ void k_split_coef(const double* __restrict__ c, int64_t ncells, double h, float* ch, float* cl) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= 27 * ncells) return;
  const int q = int(t / ncells);
  const double v = c[t] * cW364[q] * h;
  const float hi = __double2float_rn(v);
  ch[t] = hi;
  cl[t] = __double2float_rn(v - double(hi));
}

// [3][27][ncells] rho_cp beta_d -> w_q h^2 rho_cp beta_d as float pairs
__global__ void k_split_vec(const double* __restrict__ b, int64_t ncells, double h2, float* bh, float* bl) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= 81 * ncells) return;
  const int q = int((t / ncells) % 27);
  const double v = b[t] * cW364[q] * h2;
  const float hi = __double2float_rn(v);
  bh[t] = hi;
  bl[t] = __double2float_rn(v - double(hi));
}

}  // namespace

mf_status launch_df_vec_split(mf_ctx* ctx, const mf_dofmap* m, const double* qvec64, float* bh, float* bl) {
  MF_CUDA_TRY(upload_tables_here());
  const int64_t n = 81 * m->n_cells;
  const double h = m->mesh->h0;
  k_split_vec<<<int((n + 255) / 256), 256, 0, ctx->stream>>>(qvec64, m->n_cells, h * h, bh, bl);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

mf_status launch_scalar_df_uniform_conv(mf_ctx* ctx, const mf_dofmap* m, const double* src, double* dst, int nrhs,
                                        int64_t ld, const float* ch, const float* cl, const float* bh, const float* bl,
                                        double mass, bool transpose, const float* mh, const float* ml) {
  MF_CUDA_TRY(upload_tables_here());
  static bool attrs = false;
  if (!attrs) {
    MF_CUDA_TRY(cudaFuncSetAttribute(k_scalar_df_uniform_conv<false, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, int(108 * kThreads * sizeof(float))));
    MF_CUDA_TRY(cudaFuncSetAttribute(k_scalar_df_uniform_conv<false, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, int(108 * kThreads * sizeof(float))));
    attrs = true;
  }
  if ((mh == nullptr) != (ml == nullptr)) return fail(MF_EINVAL, "per-Gauss-point mass: both parts or neither");
  const Tables tb = make_tables();
  DfConvArgs a{};
  a.src = src;
  a.dst = dst;
  a.nrhs = nrhs;
  a.ld = ld;
  a.ch = ch;
  a.cl = cl;
  a.bh = bh;
  a.bl = bl;
  a.ncells = m->n_cells;
  a.mh = mh;
  a.ml = ml;
  const double h = m->mesh->h0;
  for (int q = 0; q < 27; ++q) {
    const double v = tb.W3[q] * mass * h * h * h;
    a.wmh[q] = float(v);
    a.wml[q] = float(v - double(a.wmh[q]));
  }
  const UniformGeom ug = uniform_geom(m);
  const dim3 grid(brick_blocks(ug.nx, ug.ny, ug.nz), nrhs);
  const size_t sm_tr = 54 * kThreads * sizeof(float), sm_fw = 108 * kThreads * sizeof(float);
  if (transpose && mh)
    k_scalar_df_uniform_conv<true, true><<<grid, kThreads, sm_tr, ctx->stream>>>(a, ug);
  else if (transpose)
    k_scalar_df_uniform_conv<true, false><<<grid, kThreads, sm_tr, ctx->stream>>>(a, ug);
  else if (mh)
    k_scalar_df_uniform_conv<false, true><<<grid, kThreads, sm_fw, ctx->stream>>>(a, ug);
  else
    k_scalar_df_uniform_conv<false, false><<<grid, kThreads, sm_fw, ctx->stream>>>(a, ug);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

mf_status launch_df_mass_split(mf_ctx* ctx, const mf_dofmap* m, const double* qmass64, float* mh, float* ml) {
  MF_CUDA_TRY(upload_tables_here());
  const int64_t n = 27 * m->n_cells;
  const double h = m->mesh->h0;
  k_split_coef<<<int((n + 255) / 256), 256, 0, ctx->stream>>>(qmass64, m->n_cells, h * h * h, mh, ml);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

mf_status launch_df_coef_split(mf_ctx* ctx, const mf_dofmap* m, const double* qcoef64, float* ch, float* cl) {
  MF_CUDA_TRY(upload_tables_here());
  const int64_t n = 27 * m->n_cells;
  k_split_coef<<<int((n + 255) / 256), 256, 0, ctx->stream>>>(qcoef64, m->n_cells, m->mesh->h0, ch, cl);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

mf_status launch_scalar_df_uniform(mf_ctx* ctx, const mf_dofmap* m, const double* src, double* dst, int nrhs,
                                   int64_t ld, const float* ch, const float* cl, double mass) {
  MF_CUDA_TRY(upload_tables_here());
  const Tables tb = make_tables();
  DfArgs a{};
  a.src = src;
  a.dst = dst;
  a.nrhs = nrhs;
  a.ld = ld;
  a.ch = ch;
  a.cl = cl;
  a.ncells = m->n_cells;
  const double h = m->mesh->h0;
  for (int q = 0; q < 27; ++q) {
    const double v = tb.W3[q] * mass * h * h * h;
    a.wmh[q] = float(v);
    a.wml[q] = float(v - double(a.wmh[q]));
  }
  const UniformGeom ug = uniform_geom(m);
  k_scalar_df_uniform<<<dim3(brick_blocks(ug.nx, ug.ny, ug.nz), nrhs), kThreads, 0, ctx->stream>>>(a, ug);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

mf_status launch_split_pairs(mf_ctx* ctx, const double* c, int64_t n, float* h, float* l) {
  k_split_plain<<<int((n + 255) / 256), 256, 0, ctx->stream>>>(c, n, h, l);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

mf_status launch_oseen_df_uniform(mf_ctx* ctx, const mf_dofmap* mu, const double* src, double* dst, const float* cm,
                                  const float* cv, const float* cb, const float* nr) {
  MF_CUDA_TRY(upload_tables_here());
  const Tables tb = make_tables();
  DfOseenArgs a{};
  a.src = src;
  a.dst = dst;
  a.nu = mu->n_dofs;
  a.ncells = mu->n_cells;
  const int64_t nc = mu->n_cells;
  a.cmh = cm;
  a.cml = cm + 27 * nc;
  a.cvh = cv;
  a.cvl = cv + 27 * nc;
  a.cbh = cb;
  a.cbl = cb + 81 * nc;
  const double h = mu->mesh->h0;
  for (int q = 0; q < 27; ++q)
    for (int n = 0; n < 8; ++n) {
      const double v = -(h * h) * tb.PWW[8 * q + n];
      a.pwh[q][n] = float(v);
      a.pwl[q][n] = float(v - double(a.pwh[q][n]));
    }
  for (int g = 0; g < 3; ++g)
    for (int q1 = 0; q1 < 2; ++q1) {
      const double v = tb.W[g] * tb.P[2 * g + q1];
      a.wph[g][q1] = float(v);
      a.wpl[g][q1] = float(v - double(a.wph[g][q1]));
    }
  a.mh2h = float(-(h * h));
  a.mh2l = float(-(h * h) - double(a.mh2h));
  const UniformGeom ug = uniform_geom(mu);
  const int nb = ((ug.nx + 7) / 8) * ((ug.ny + 3) / 4) * ug.nz;
  if (nr) {
    a.nrh = nr;
    a.nrl = nr + 81 * nc;
    k_oseen_df_uniform<true><<<nb, 96, 0, ctx->stream>>>(a, ug);
  } else {
    k_oseen_df_uniform<false><<<nb, 96, 0, ctx->stream>>>(a, ug);
  }
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

}  // namespace mf
