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
#include "ops.h"

namespace mf {

MF_DEFINE_TABLE_UPLOAD

UniformGeom uniform_geom(const mf_dofmap* m);

namespace {

struct dd {
  float h, l;
};

// double -> pair of floats for x 2^-bias, by bits (no fp64 instruction: GB300 converts between fp64
// and fp32 at its fp64 rate): hi = the top 24 significand bits (truncated), lo = the remaining 29
// bits rounded once (the high 23 and low 6 bits made floats exactly through the 2^23 offset, joined by
// one FMA), so hi + lo = x 2^-bias to 2^-47 relative.  Magnitudes below 2^-126 after scaling give 0.
__device__ __forceinline__ dd d2dd_bits(double x, int bias) {
  const unsigned hi32 = unsigned(__double2hiint(x)), lo32 = unsigned(__double2loint(x));
  const unsigned E0 = (hi32 >> 20) & 0x7FFu, sign = hi32 & 0x80000000u;
  const int E = int(E0) - bias;
  if (E0 == 0u || E < 897 || E > 1150) return {0.f, 0.f};
  const unsigned Ef = unsigned(E - 896);
  const float h = __uint_as_float(sign | (Ef << 23) | ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29));
  const unsigned m = lo32 & 0x1FFFFFFFu;
  const float mh = __fsub_rn(__uint_as_float(0x4B000000u | (m >> 6)), 8388608.0f);
  const float ml = __fsub_rn(__uint_as_float(0x4B000000u | (m & 63u)), 8388608.0f);
  const float mf = __fmaf_rn(mh, 64.0f, ml);
  const float l = __fmul_rn(__fmul_rn(mf, 0x1p-52f), __uint_as_float(Ef << 23));
  return {h, __uint_as_float(__float_as_uint(l) | sign)};
}
// f 2^bias as a double, by bits (exact for normal floats; zero and subnormals give 0)
__device__ __forceinline__ double f2d_bits(float f, int bias) {
  const unsigned b = __float_as_uint(f), e = (b >> 23) & 0xFFu;
  const unsigned hi = e ? (b & 0x80000000u) | (unsigned(int(e) + 896 + bias) << 20) | ((b >> 3) & 0xFFFFFu) : 0u;
  return __hiloint2double(int(hi), e ? int(b << 29) : 0);
}
// two-sum of the high parts (exact), low parts added in fp32
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return {s, __fadd_rn(e, __fadd_rn(a.l, b.l))};
}
// exact fp32 product of the high parts (FMA residual) plus the two cross terms
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return {p, e};
}
__device__ __forceinline__ dd dd_norm(dd a) {
  const float s = __fadd_rn(a.h, a.l);
  return {s, __fsub_rn(a.l, __fsub_rn(s, a.h))};
}
__device__ __forceinline__ dd dd_fma(dd acc, dd a, dd b) { return dd_add(acc, dd_mul(a, b)); }

__device__ __forceinline__ dd cS(int q, int a) { return {cSh[3 * q + a], cSl[3 * q + a]}; }
__device__ __forceinline__ dd cD(int q, int p) { return {cDh[3 * q + p], cDl[3 * q + p]}; }

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

// nodes -> Gauss points along DIR, in place (the middle Gauss point is the middle node)
template <int DIR> __device__ __forceinline__ void dsweep(dd* U) {
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    const int b = line_base<DIR>(j), s = Dir<DIR>::s;
    const dd u0 = U[b], u1 = U[b + s], u2 = U[b + 2 * s];
    U[b] = dd_norm(dd_add(dd_add(dd_mul(cS(0, 0), u0), dd_mul(cS(0, 1), u1)), dd_mul(cS(0, 2), u2)));
    U[b + 2 * s] = dd_norm(dd_add(dd_add(dd_mul(cS(2, 0), u0), dd_mul(cS(2, 1), u1)), dd_mul(cS(2, 2), u2)));
  }
}
// Gauss points -> nodes along DIR (transposed), in place
template <int DIR> __device__ __forceinline__ void dsweep_t(dd* U) {
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    const int b = line_base<DIR>(j), s = Dir<DIR>::s;
    const dd u0 = U[b], u1 = U[b + s], u2 = U[b + 2 * s];
    U[b] = dd_norm(dd_add(dd_mul(cS(0, 0), u0), dd_mul(cS(2, 0), u2)));
    U[b + s] = dd_norm(dd_add(dd_add(dd_mul(cS(0, 1), u0), u1), dd_mul(cS(2, 1), u2)));
    U[b + 2 * s] = dd_norm(dd_add(dd_mul(cS(0, 2), u0), dd_mul(cS(2, 2), u2)));
  }
}
// collocation derivative at point qd of a line (D[1][1] = 0)
__device__ __forceinline__ dd ddline(int qd, dd u0, dd u1, dd u2) {
  if (qd == 1) return dd_add(dd_mul(cD(1, 0), u0), dd_mul(cD(1, 2), u2));
  return dd_add(dd_add(dd_mul(cD(qd, 0), u0), dd_mul(cD(qd, 1), u1)), dd_mul(cD(qd, 2), u2));
}

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

// w_q h c_q of the Gauss-point coefficient table, split into high and low float parts
__global__ void k_split_coef(const double* __restrict__ c, int64_t ncells, double h, float* ch, float* cl) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= 27 * ncells) return;
  const int q = int(t / ncells);
  const double v = c[t] * cW364[q] * h;
  const float hi = __double2float_rn(v);
  ch[t] = hi;
  cl[t] = __double2float_rn(v - double(hi));
}

}  // namespace

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

}  // namespace mf
