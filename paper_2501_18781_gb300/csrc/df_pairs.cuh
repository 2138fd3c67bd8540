// Double-float ("dd") arithmetic on the fp32 pipes and the Q2 sum-factorisation sweeps in it, shared
// by the double-float kernels (uniform and octree meshes).  A value is an unnormalised pair of floats
// hi + lo (48-bit significand): Dekker's product through the FMA residual, Knuth's two-sum for the
// high parts (Joldes, Muller and Popescu, ACM TOMS 2017, bound these "double-word" algorithms).
// Doubles enter and leave by bit manipulation, scaled by a power of two chosen by the caller.
#pragma once

#include "ops.h"

namespace mf {
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

}  // namespace
}  // namespace mf
