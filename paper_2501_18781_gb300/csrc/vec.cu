// Vector kernels of the Krylov solvers.  All reductions accumulate in fp64 over a fixed
// grid of kRedBlocks blocks, then the last block to finish sums the partials in a fixed order,
// so every dot product is deterministic.
#include <algorithm>
#include <mutex>
#include <string>
#include <type_traits>

#include <cuda_fp16.h>

#include "reduce.cuh"

namespace mf {

namespace {

__global__ void __launch_bounds__(kRedThreads) k_finish(const double* part, int g, double* out, int mode, double* S) {
  finish_row(part, g, blockIdx.x, Finish{out, mode, S, nullptr});
}

// Per-block partial sums of x.y (and x2.y2).  Each thread keeps four independent
// accumulators over elements one grid stride apart, so four loads per vector are in flight
// per thread (enough bytes in flight to approach HBM bandwidth with one block per warp slot);
// the partition and the summation order are fixed, so results are reproducible bit for bit.
template <typename TX, typename TY>
__global__ void __launch_bounds__(kRedThreads) k_dot2_partial(const TX* x, const TY* y, const TX* x2, const TY* y2,
                                                             int64_t n, int64_t ld, double* part, Finish fin) {
  const int r = blockIdx.y;
  x += r * ld; y += r * ld;
  if (x2) { x2 += r * ld; y2 += r * ld; }
  const int64_t st = int64_t(gridDim.x) * blockDim.x;
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if constexpr (std::is_same<TX, float>::value && std::is_same<TY, float>::value) {
    Dot2f a0, a1, a2, a3, b0, b1, b2, b3;
    for (; i + 3 * st < n; i += 4 * st) {
      const float p0 = x[i], p1 = x[i + st], p2 = x[i + 2 * st], p3 = x[i + 3 * st];
      const float q0 = y[i], q1 = y[i + st], q2 = y[i + 2 * st], q3 = y[i + 3 * st];
      a0.add(p0, q0); a1.add(p1, q1); a2.add(p2, q2); a3.add(p3, q3);
      if (x2) {
        b0.add(x2[i], y2[i]); b1.add(x2[i + st], y2[i + st]);
        b2.add(x2[i + 2 * st], y2[i + 2 * st]); b3.add(x2[i + 3 * st], y2[i + 3 * st]);
      }
    }
    for (; i < n; i += st) {
      a0.add(x[i], y[i]);
      if (x2) b0.add(x2[i], y2[i]);
    }
    const double s = block_sum((a0.value() + a1.value()) + (a2.value() + a3.value()));
    const double s2 = x2 ? block_sum((b0.value() + b1.value()) + (b2.value() + b3.value())) : 0.0;
    if (threadIdx.x == 0) {
      part[int64_t(r) * 2 * gridDim.x + blockIdx.x] = s;
      part[int64_t(r) * 2 * gridDim.x + gridDim.x + blockIdx.x] = s2;
    }
    finish_if_last(part, fin);
    return;
  }
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;
  if (x2) {
    for (; i + 3 * st < n; i += 4 * st) {
      const double p0 = double(x[i]), p1 = double(x[i + st]), p2 = double(x[i + 2 * st]), p3 = double(x[i + 3 * st]);
      const double q0 = double(y[i]), q1 = double(y[i + st]), q2 = double(y[i + 2 * st]), q3 = double(y[i + 3 * st]);
      const double u0 = double(x2[i]), u1 = double(x2[i + st]), u2 = double(x2[i + 2 * st]), u3 = double(x2[i + 3 * st]);
      const double v0 = double(y2[i]), v1 = double(y2[i + st]), v2 = double(y2[i + 2 * st]), v3 = double(y2[i + 3 * st]);
      a0 += p0 * q0; a1 += p1 * q1; a2 += p2 * q2; a3 += p3 * q3;
      b0 += u0 * v0; b1 += u1 * v1; b2 += u2 * v2; b3 += u3 * v3;
    }
    for (; i < n; i += st) {
      a0 += double(x[i]) * double(y[i]);
      b0 += double(x2[i]) * double(y2[i]);
    }
  } else {
    for (; i + 3 * st < n; i += 4 * st) {
      const double p0 = double(x[i]), p1 = double(x[i + st]), p2 = double(x[i + 2 * st]), p3 = double(x[i + 3 * st]);
      const double q0 = double(y[i]), q1 = double(y[i + st]), q2 = double(y[i + 2 * st]), q3 = double(y[i + 3 * st]);
      a0 += p0 * q0; a1 += p1 * q1; a2 += p2 * q2; a3 += p3 * q3;
    }
    for (; i < n; i += st) a0 += double(x[i]) * double(y[i]);
  }
  double s = block_sum((a0 + a1) + (a2 + a3));
  double s2 = x2 ? block_sum((b0 + b1) + (b2 + b3)) : 0.0;
  if (threadIdx.x == 0) {
    part[int64_t(r) * 2 * gridDim.x + blockIdx.x] = s;
    part[int64_t(r) * 2 * gridDim.x + gridDim.x + blockIdx.x] = s2;
  }
  finish_if_last(part, fin);
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_cg_xr(int64_t n, int64_t ld, T* x, T* r, const T* p, const T* Ap,
                                                       const T* dinv, T* z, int zmode, const double* S, double* part,
                                                       Finish fin, bool skip_inactive) {
  const int rh = blockIdx.y;
  if (skip_inactive && S[rh * S_NSCAL + S_ACTIVE] == 0.0) return;  // this system has stopped
  const double alpha = S[rh * S_NSCAL + S_ALPHA];
  const int64_t o = rh * ld;
  double rr = 0.0, rz = 0.0;
  if constexpr (std::is_same<T, float>::value) {
    Dot2f crr, crz;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
      const float xi = x[o + i] + float(alpha) * p[o + i];
      const float ri = r[o + i] - float(alpha) * Ap[o + i];
      x[o + i] = xi;
      r[o + i] = ri;
      crr.add(ri, ri);
      if (zmode == 1) {
        const float zi = dinv[i] * ri;
        z[o + i] = zi;
        crz.add(ri, zi);
      } else if (zmode == 0) {
        crz.add(ri, ri);
      }
    }
    rr = crr.value();
    rz = crz.value();
  } else {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
      T xi = x[o + i] + T(alpha) * p[o + i];
      T ri = r[o + i] - T(alpha) * Ap[o + i];
      x[o + i] = xi;
      r[o + i] = ri;
      rr += double(ri) * double(ri);
      if (zmode == 1) {
        T zi = dinv[i] * ri;
        z[o + i] = zi;
        rz += double(ri) * double(zi);
      } else if (zmode == 0) {
        rz += double(ri) * double(ri);
      }
    }
  }
  rr = block_sum(rr);
  rz = block_sum(rz);
  if (threadIdx.x == 0) {
    part[int64_t(rh) * 2 * gridDim.x + blockIdx.x] = rr;
    part[int64_t(rh) * 2 * gridDim.x + gridDim.x + blockIdx.x] = rz;
  }
  finish_if_last(part, fin);
}

// y = S p for a 125-point stencil on an (nx + 1) x (ny + 1) x (nz + 1) grid (the scaled fp16
// tiled layout of stencil_at; entries toward nodes outside the grid are 0, and their loads are
// clamped into it).  All sixteen 16-byte words of a row are loaded before the first is used.  DOT: also p.y, reduced like cg_alpha (Finish mode 1), so one launch
// is a CG step's operator application and its alpha.  Fixed grid of at most kRedBlocks blocks.
template <bool DOT>
__global__ void __launch_bounds__(kRedThreads) k_stencil125(const __half* __restrict__ S,
                                                            const float* __restrict__ scale,
                                                            const float* __restrict__ p, float* __restrict__ y,
                                                            int nx, int ny, int nz, double* part, Finish fin) {
  if (DOT && fin.S[S_ACTIVE] == 0.0) return;  // the CG this step belongs to has stopped
  const int px = nx + 1, pxy = px * (ny + 1), np = pxy * (nz + 1);
  Dot2f acc;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    const int ix = i % px, iy = (i / px) % (ny + 1), iz = i / pxy;
    int ox[5], oy[5], oz[5];
#pragma unroll
    for (int d = 0; d < 5; ++d) {
      ox[d] = min(max(ix + d - 2, 0), nx);
      oy[d] = px * min(max(iy + d - 2, 0), ny);
      oz[d] = pxy * min(max(iz + d - 2, 0), nz);
    }
    const uint4* Si = reinterpret_cast<const uint4*>(S + stencil_at(0, i));
    uint4 w[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) w[k] = __ldcs(Si + 32 * k);
    float sz[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};  // one running sum per z plane
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const uint32_t pair[4] = {w[k].x, w[k].y, w[k].z, w[k].w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        __half2 h2;
        memcpy(&h2, &pair[j], 4);
        const float2 c = __half22float2(h2);
        const float cv[2] = {c.x, c.y};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int o = 8 * k + 2 * j + e;
          if (o < 125) {
            const int dx = o % 5, dy = (o / 5) % 5, dz = o / 25;
            sz[dz] = fmaf(cv[e], __ldg(p + (ox[dx] + oy[dy] + oz[dz])), sz[dz]);
          }
        }
      }
    }
    const float s = scale[i] * (((sz[0] + sz[1]) + (sz[2] + sz[3])) + sz[4]);
    y[i] = s;
    if (DOT) acc.add(p[i], s);
  }
  if constexpr (DOT) {
    const double t = block_sum(acc.value());
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    finish_if_last(part, fin);
  }
}

// pinv[i] = 1 / (row i's centre entry, o = 62) where that is positive; other entries unchanged
__global__ void k_stencil_diag_inverse(const __half* __restrict__ S, const float* __restrict__ scale, int64_t n,
                                       float* pinv) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float d = scale[i] * __half2float(S[stencil_at(62, i)]);
  if (d > 0.0f) pinv[i] = 1.0f / d;
}

template <typename T>
__global__ void k_cg_p(int64_t n, int64_t ld, const T* z, T* p, const double* S, bool skip_inactive) {
  const int rh = blockIdx.y;
  if (skip_inactive && S[rh * S_NSCAL + S_ACTIVE] == 0.0) return;
  const T beta = T(S[rh * S_NSCAL + S_BETA]);
  const int64_t o = rh * ld;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[o + i] = z[o + i] + beta * p[o + i];
}

template <typename TX, typename TY>
__global__ void k_axpby(int64_t n, double a, const TX* x, double b, TY* y) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = TY(a * double(x[i]) + (b == 0.0 ? 0.0 : b * double(y[i])));
}

template <typename T> __global__ void k_pmul(int64_t n, const T* d, const T* r, T* z) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    z[i] = d ? d[i] * r[i] : r[i];
}

template <typename T, typename TB>
__global__ void k_block_jacobi(int64_t nu, int64_t np, const TB* blk, const double* pinv, const T* r, T* z) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nu + np; i += int64_t(gridDim.x) * blockDim.x) {
    if (i < nu) {
      const TB* B = blk + 9 * i;
      const TB r0 = TB(r[i]), r1 = TB(r[nu + i]), r2 = TB(r[2 * nu + i]);
      z[i] = T(B[0] * r0 + B[1] * r1 + B[2] * r2);
      z[nu + i] = T(B[3] * r0 + B[4] * r1 + B[5] * r2);
      z[2 * nu + i] = T(B[6] * r0 + B[7] * r1 + B[8] * r2);
    } else {
      int64_t j = i - nu;
      z[3 * nu + j] = T(pinv[j] * double(r[3 * nu + j]));
    }
  }
}

// fp32 block inverses stored entry-major (entry e of node i at e * nu + i), so that each of a
// warp's nine loads is one coalesced run
__global__ void k_block_jacobi_soa32(int64_t nu, const float* __restrict__ blk, const float* __restrict__ r,
                                     float* __restrict__ z) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nu; i += int64_t(gridDim.x) * blockDim.x) {
    const float r0 = r[i], r1 = r[nu + i], r2 = r[2 * nu + i];
    z[i] = blk[i] * r0 + blk[nu + i] * r1 + blk[2 * nu + i] * r2;
    z[nu + i] = blk[3 * nu + i] * r0 + blk[4 * nu + i] * r1 + blk[5 * nu + i] * r2;
    z[2 * nu + i] = blk[6 * nu + i] * r0 + blk[7 * nu + i] * r1 + blk[8 * nu + i] * r2;
  }
}
// dst = s[0] src (velocity blocks; dst may be src) and z = B^-1 dst per node, in one pass
__global__ void k_block_jacobi_scaled32(int64_t nu, const float* __restrict__ blk, const double* s, const float* src,
                                        float* dst, float* __restrict__ z) {
  const float a = float(s[0]);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nu; i += int64_t(gridDim.x) * blockDim.x) {
    const float r0 = a * src[i], r1 = a * src[nu + i], r2 = a * src[2 * nu + i];
    dst[i] = r0;
    dst[nu + i] = r1;
    dst[2 * nu + i] = r2;
    z[i] = blk[i] * r0 + blk[nu + i] * r1 + blk[2 * nu + i] * r2;
    z[nu + i] = blk[3 * nu + i] * r0 + blk[4 * nu + i] * r1 + blk[5 * nu + i] * r2;
    z[2 * nu + i] = blk[6 * nu + i] * r0 + blk[7 * nu + i] * r1 + blk[8 * nu + i] * r2;
  }
}
template <typename TS, typename TD> __global__ void k_convert(int64_t n, const TS* s, TD* d) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    d[i] = TD(s[i]);
}

template <typename T>
__global__ void k_cheb_init(int64_t n, int64_t ld, const T* r, const T* dinv, T inv_theta, T* d) {
  const int64_t o = blockIdx.y * ld;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    d[o + i] = inv_theta * dinv[i] * r[o + i];
}

// One element of the Chebyshev step (the recurrence is spelled out where cheb_step is declared).
template <typename T, bool FIRST, bool LAST>
__device__ __forceinline__ void cheb_elem(T& zo, T zi_in, T ri_in, T adi, T& di_io, T dv, T c1, T c2, T& ro) {
  const T di = di_io;
  const T zi = FIRST ? di : zi_in + di;
  const T ri = ri_in - adi;
  const T dn = c1 * di + c2 * dv * ri;
  if (LAST) {
    zo = zi + dn;
  } else {
    zo = zi;
    ro = ri;
    di_io = dn;
  }
}

template <typename T, int W> struct alignas(sizeof(T) * W) ChebWord {
  T c[W];
};

// W = 1: one element per step of a thread; W > 1: 16-byte words of W elements (every vector starts
// on a 16-byte boundary and so does each right-hand side ld elements further on), the last n % W
// elements one by one.
template <typename T, bool FIRST, bool LAST, int W>
__global__ void k_cheb_step(int64_t n, int64_t ld, T* z, const T* res_in, T* res, const T* Ad, T* d, const T* dinv,
                            T c1, T c2) {
  using V = ChebWord<T, W>;
  const int64_t o = blockIdx.y * ld, stride = int64_t(gridDim.x) * blockDim.x;
  const int64_t t0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x, nw = n / W;
  for (int64_t w = t0; w < nw; w += stride) {
    V dv = reinterpret_cast<const V*>(d + o)[w];
    const V rv = reinterpret_cast<const V*>(res_in + o)[w];
    const V av = reinterpret_cast<const V*>(Ad + o)[w];
    const V iv = reinterpret_cast<const V*>(dinv)[w];
    V zv;
    if (!FIRST) zv = reinterpret_cast<const V*>(z + o)[w];
    V zo, ro;
#pragma unroll
    for (int c = 0; c < W; ++c)
      cheb_elem<T, FIRST, LAST>(zo.c[c], FIRST ? T(0) : zv.c[c], rv.c[c], av.c[c], dv.c[c], iv.c[c], c1, c2, ro.c[c]);
    reinterpret_cast<V*>(z + o)[w] = zo;
    if (!LAST) {
      reinterpret_cast<V*>(res + o)[w] = ro;
      reinterpret_cast<V*>(d + o)[w] = dv;
    }
  }
  for (int64_t i = nw * W + t0; i < n; i += stride) {
    T di = d[o + i], zo, ro;
    cheb_elem<T, FIRST, LAST>(zo, FIRST ? T(0) : z[o + i], res_in[o + i], Ad[o + i], di, dinv[i], c1, c2, ro);
    z[o + i] = zo;
    if (!LAST) {
      res[o + i] = ro;
      d[o + i] = di;
    }
  }
}

// CGS2 pieces of the GMRES solvers.  V holds k basis vectors ld apart.  Where V and w start on
// 16-byte boundaries and ld * sizeof(T) is a multiple of 16 (the solvers pad their bases so),
// every thread moves 16-byte words (four floats or two doubles), so each step of a thread has
// KG + 1 independent 16-byte loads in flight; otherwise the same code runs on single elements.
template <typename T, int W> struct alignas(sizeof(T) * W) Word {
  T c[W];
};

template <typename T> struct DotAcc;
template <> struct DotAcc<float> : Dot2f {};
template <> struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};

// part[(j0 + g) * gridDim.x + block] = the block's share of V_g . w for g < KG (V already offset
// to vector j0): one sweep over w for KG vectors.
template <typename T, int KG, int W>
__device__ __forceinline__ void multidot_group(const T* V, int64_t ld, const T* w, int64_t n, double* part, int j0) {
  using Wd = Word<T, W>;
  DotAcc<T> acc[KG];
  const int64_t t0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x, st = int64_t(gridDim.x) * blockDim.x;
  const int64_t nw = n / W, ldw = ld / W;
  const Wd* Vw = reinterpret_cast<const Wd*>(V);
  const Wd* ww = reinterpret_cast<const Wd*>(w);
  for (int64_t i = t0; i < nw; i += st) {
    const Wd y = ww[i];
    Wd x[KG];
#pragma unroll
    for (int g = 0; g < KG; ++g) x[g] = Vw[g * ldw + i];
#pragma unroll
    for (int g = 0; g < KG; ++g)
#pragma unroll
      for (int c = 0; c < W; ++c) acc[g].add(x[g].c[c], y.c[c]);
  }
  if (W > 1)  // the last n mod W elements
    for (int64_t i = nw * W + t0; i < n; i += st) {
      const T y = w[i];
#pragma unroll
      for (int g = 0; g < KG; ++g) acc[g].add(V[g * ld + i], y);
    }
#pragma unroll
  for (int g = 0; g < KG; ++g) {
    const double sg = block_sum(acc[g].value());
    if (threadIdx.x == 0) part[int64_t(j0 + g) * gridDim.x + blockIdx.x] = sg;
  }
}

// h_j partials of V_j . w for j < k: groups of eight vectors, then one group of the rest
template <typename T, int W>
__global__ void __launch_bounds__(kRedThreads, 4) k_multidot(const T* V, int64_t ld, int k, const T* w, int64_t n,
                                                             double* part) {
  int j0 = 0;
  for (; j0 + 8 <= k; j0 += 8) multidot_group<T, 8, W>(V + j0 * ld, ld, w, n, part, j0);
  const T* Vr = V + j0 * ld;
  switch (k - j0) {
    case 1: multidot_group<T, 1, W>(Vr, ld, w, n, part, j0); break;
    case 2: multidot_group<T, 2, W>(Vr, ld, w, n, part, j0); break;
    case 3: multidot_group<T, 3, W>(Vr, ld, w, n, part, j0); break;
    case 4: multidot_group<T, 4, W>(Vr, ld, w, n, part, j0); break;
    case 5: multidot_group<T, 5, W>(Vr, ld, w, n, part, j0); break;
    case 6: multidot_group<T, 6, W>(Vr, ld, w, n, part, j0); break;
    case 7: multidot_group<T, 7, W>(Vr, ld, w, n, part, j0); break;
    default: break;
  }
}
// The first pass's update and the second pass's products of classical Gram-Schmidt in one sweep,
// for KG <= 8 vectors: w <- w + sign V h (T arithmetic, as k_multiaxpy), then part[g] = the
// block's share of V_g . w (as k_multidot, same grid and per-thread order, so the results equal
// the two separate launches bit for bit).
template <typename T, int KG, int W>
__global__ void __launch_bounds__(kRedThreads, 4) k_axpy_multidot(const T* V, int64_t ld, const double* h, double sign,
                                                                  T* w, int64_t n, double* part) {
  using Wd = Word<T, W>;
  __shared__ T hs[KG];
  if (threadIdx.x < KG) hs[threadIdx.x] = T(sign * h[threadIdx.x]);
  __syncthreads();
  DotAcc<T> acc[KG];
  const int64_t t0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x, st = int64_t(gridDim.x) * blockDim.x;
  const int64_t nw = n / W, ldw = ld / W;
  const Wd* Vw = reinterpret_cast<const Wd*>(V);
  Wd* ww = reinterpret_cast<Wd*>(w);
  for (int64_t i = t0; i < nw; i += st) {
    Wd y = ww[i];
    Wd x[KG];
#pragma unroll
    for (int g = 0; g < KG; ++g) x[g] = Vw[g * ldw + i];
#pragma unroll
    for (int g = 0; g < KG; ++g)
#pragma unroll
      for (int c = 0; c < W; ++c) y.c[c] = fma(hs[g], x[g].c[c], y.c[c]);
    ww[i] = y;
#pragma unroll
    for (int g = 0; g < KG; ++g)
#pragma unroll
      for (int c = 0; c < W; ++c) acc[g].add(x[g].c[c], y.c[c]);
  }
  if (W > 1)
    for (int64_t i = nw * W + t0; i < n; i += st) {
      T y = w[i];
#pragma unroll
      for (int g = 0; g < KG; ++g) y = fma(hs[g], V[g * ld + i], y);
      w[i] = y;
#pragma unroll
      for (int g = 0; g < KG; ++g) acc[g].add(V[g * ld + i], y);
    }
#pragma unroll
  for (int g = 0; g < KG; ++g) {
    const double sg = block_sum(acc[g].value());
    if (threadIdx.x == 0) part[int64_t(g) * gridDim.x + blockIdx.x] = sg;
  }
}

__global__ void __launch_bounds__(kRedThreads) k_multidot_finish(const double* part, int g, double* h) {
  double s = 0.0;
  for (int i = threadIdx.x; i < g; i += blockDim.x) s += part[blockIdx.x * g + i];
  s = block_sum(s);
  if (threadIdx.x == 0) h[blockIdx.x] = s;
}

// w += sign V h over k <= 64 vectors, h staged in shared memory (in T: fp32 data takes fp32
// FMAs, since the fp64 pipe would bound this HBM-bound update); eight independent word loads
// per step of the j loop.  NORM: also |w|^2 of the result, reduced into fin.out (Finish mode 0)
// by the last block, which saves the separate norm pass of Gram-Schmidt.
template <typename T, int W, bool NORM>
__global__ void __launch_bounds__(256) k_multiaxpy(const T* V, int64_t ld, int k, const double* h, double sign, T* w,
                                                   int64_t n, double* part, Finish fin) {
  using Wd = Word<T, W>;
  __shared__ T hs[64];
  for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = T(sign * h[j]);
  __syncthreads();
  const int64_t t0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x, st = int64_t(gridDim.x) * blockDim.x;
  const int64_t nw = n / W, ldw = ld / W;
  const Wd* Vw = reinterpret_cast<const Wd*>(V);
  Wd* ww = reinterpret_cast<Wd*>(w);
  DotAcc<T> nrm;
  for (int64_t i = t0; i < nw; i += st) {
    Wd acc = ww[i];
    int j = 0;
    for (; j + 8 <= k; j += 8) {
      Wd x[8];
#pragma unroll
      for (int g = 0; g < 8; ++g) x[g] = Vw[(j + g) * ldw + i];
#pragma unroll
      for (int g = 0; g < 8; ++g)
#pragma unroll
        for (int c = 0; c < W; ++c) acc.c[c] = fma(hs[j + g], x[g].c[c], acc.c[c]);
    }
    for (; j < k; ++j) {
      const Wd x = Vw[j * ldw + i];
#pragma unroll
      for (int c = 0; c < W; ++c) acc.c[c] = fma(hs[j], x.c[c], acc.c[c]);
    }
    ww[i] = acc;
    if (NORM)
#pragma unroll
      for (int c = 0; c < W; ++c) nrm.add(acc.c[c], acc.c[c]);
  }
  if (W > 1)
    for (int64_t i = nw * W + t0; i < n; i += st) {
      T acc = w[i];
      for (int j = 0; j < k; ++j) acc = fma(hs[j], V[j * ld + i], acc);
      w[i] = acc;
      if (NORM) nrm.add(acc, acc);
    }
  if constexpr (NORM) {
    const double s = block_sum(nrm.value());
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    finish_if_last(part, fin);
  }
}

__global__ void k_splitmix(uint64_t seed, double* v, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    uint64_t z = seed + uint64_t(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    v[i] = double(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  }
}

__global__ void k_set_list(double* v, const int32_t* list, int64_t n, double val) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) v[list[t]] = val;
}
template <typename T> __global__ void k_zero_list(T* v, const int32_t* list, int64_t n) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) v[list[t]] = T(0);
}

inline int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return int(g < 4 * 152 * 4 ? (g < 1 ? 1 : g) : 4 * 152 * 4);
}

// The reduction scratch is allocated with the context (kScratchDoubles) and never grown, so
// that solver iterations can be captured in CUDA graphs.
// one arrival counter per right-hand side for the reductions that sum their own partials
unsigned* counters(mf_ctx* ctx) { return ctx->counters.as<unsigned>(); }

mf_status scratch(mf_ctx* ctx, size_t doubles, double** p) {
  if (ctx->scratch.bytes < doubles * sizeof(double))
    return fail(MF_EINVAL, "reduction scratch too small for this many right-hand sides");
  *p = ctx->scratch.as<double>();
  return MF_OK;
}

}  // namespace

#define LAUNCH_CHECK() \
  do { ctx->launches++; MF_CUDA_TRY(cudaGetLastError()); } while (0)

template <typename TX, typename TY> mf_status dot(mf_ctx* ctx, const TX* x, const TY* y, int64_t n, double* out) {
  double* part;
  MF_TRY(scratch(ctx, 2 * kRedBlocks, &part));
  k_dot2_partial<TX, TY><<<dim3(kRedBlocks, 1), kRedThreads, 0, ctx->stream>>>(x, y, nullptr, nullptr, n, 0, part,
                                                                                Finish{out, 0, nullptr, counters(ctx)});
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status dot<double, double>(mf_ctx*, const double*, const double*, int64_t, double*);
template mf_status dot<float, float>(mf_ctx*, const float*, const float*, int64_t, double*);

template <typename T>
mf_status dot_batched(mf_ctx* ctx, const T* x, const T* y, int64_t n, int64_t ld, int nvec, double* out) {
  double* part;
  MF_TRY(scratch(ctx, 2 * kRedBlocks * size_t(nvec), &part));
  k_dot2_partial<T, T><<<dim3(kRedBlocks, nvec), kRedThreads, 0, ctx->stream>>>(x, y, nullptr, nullptr, n, ld, part,
                                                                                 Finish{out, 0, nullptr, counters(ctx)});
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status dot_batched<double>(mf_ctx*, const double*, const double*, int64_t, int64_t, int, double*);
template mf_status dot_batched<float>(mf_ctx*, const float*, const float*, int64_t, int64_t, int, double*);

mf_status norm2_sq(mf_ctx* ctx, const double* x, int64_t n, double* out) { return dot<double, double>(ctx, x, x, n, out); }

template <typename TX, typename TY> mf_status axpby(mf_ctx* ctx, int64_t n, double a, const TX* x, double b, TY* y) {
  k_axpby<TX, TY><<<grid_for(n), 256, 0, ctx->stream>>>(n, a, x, b, y);
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status axpby<double, double>(mf_ctx*, int64_t, double, const double*, double, double*);
template mf_status axpby<float, double>(mf_ctx*, int64_t, double, const float*, double, double*);
template mf_status axpby<double, float>(mf_ctx*, int64_t, double, const double*, double, float*);
template mf_status axpby<float, float>(mf_ctx*, int64_t, double, const float*, double, float*);

template <typename T> mf_status pointwise_mul(mf_ctx* ctx, int64_t n, const T* d, const T* r, T* z) {
  k_pmul<T><<<grid_for(n), 256, 0, ctx->stream>>>(n, d, r, z);
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status pointwise_mul<double>(mf_ctx*, int64_t, const double*, const double*, double*);
template mf_status pointwise_mul<float>(mf_ctx*, int64_t, const float*, const float*, float*);

template <typename T>
mf_status block_jacobi(mf_ctx* ctx, int64_t nu, int64_t np, const double* blk, const double* pinv, const T* r, T* z) {
  k_block_jacobi<T, double><<<grid_for(nu + np), 256, 0, ctx->stream>>>(nu, np, blk, pinv, r, z);
  LAUNCH_CHECK();
  return MF_OK;
}
mf_status block_jacobi_u32_scaled(mf_ctx* ctx, int64_t nu, const float* blk, const double* s, const float* src,
                                  float* dst, float* z) {
  k_block_jacobi_scaled32<<<grid_for(nu), 256, 0, ctx->stream>>>(nu, blk, s, src, dst, z);
  LAUNCH_CHECK();
  return MF_OK;
}
mf_status block_jacobi_u32(mf_ctx* ctx, int64_t nu, const float* blk, const float* r, float* z) {
  k_block_jacobi_soa32<<<grid_for(nu), 256, 0, ctx->stream>>>(nu, blk, r, z);
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status block_jacobi<double>(mf_ctx*, int64_t, int64_t, const double*, const double*, const double*, double*);
template mf_status block_jacobi<float>(mf_ctx*, int64_t, int64_t, const double*, const double*, const float*, float*);

template <typename TS, typename TD> mf_status convert(mf_ctx* ctx, int64_t n, const TS* s, TD* d) {
  k_convert<TS, TD><<<grid_for(n), 256, 0, ctx->stream>>>(n, s, d);
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status convert<double, float>(mf_ctx*, int64_t, const double*, float*);
template mf_status convert<float, double>(mf_ctx*, int64_t, const float*, double*);

template <typename T> mf_status cg_alpha(mf_ctx* ctx, const T* p, const T* Ap, int64_t n, int64_t ld, int nrhs, double* S) {
  double* part;
  MF_TRY(scratch(ctx, 2 * kRedBlocks * size_t(nrhs), &part));
  k_dot2_partial<T, T><<<dim3(kRedBlocks, nrhs), kRedThreads, 0, ctx->stream>>>(p, Ap, nullptr, nullptr, n, ld, part,
                                                                                 Finish{nullptr, 1, S, counters(ctx)});
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status cg_alpha<double>(mf_ctx*, const double*, const double*, int64_t, int64_t, int, double*);
template mf_status cg_alpha<float>(mf_ctx*, const float*, const float*, int64_t, int64_t, int, double*);

template <typename T>
mf_status cg_update_xr(mf_ctx* ctx, int64_t n, int64_t ld, int nrhs, T* x, T* r, const T* p, const T* Ap,
                       const T* dinv, T* z, int zmode, double* S, bool skip_inactive) {
  double* part;
  MF_TRY(scratch(ctx, 2 * kRedBlocks * size_t(nrhs), &part));
  k_cg_xr<T><<<dim3(kRedBlocks, nrhs), kRedThreads, 0, ctx->stream>>>(
      n, ld, x, r, p, Ap, dinv, z, zmode, S, part, Finish{nullptr, zmode == 2 ? 5 : 2, S, counters(ctx)},
      skip_inactive);
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status cg_update_xr<double>(mf_ctx*, int64_t, int64_t, int, double*, double*, const double*, const double*,
                                        const double*, double*, int, double*, bool);
template mf_status cg_update_xr<float>(mf_ctx*, int64_t, int64_t, int, float*, float*, const float*, const float*,
                                       const float*, float*, int, double*, bool);

template <typename T> mf_status cg_rz(mf_ctx* ctx, const T* r, const T* z, int64_t n, int64_t ld, int nrhs, double* S) {
  double* part;
  MF_TRY(scratch(ctx, 2 * kRedBlocks * size_t(nrhs), &part));
  k_dot2_partial<T, T><<<dim3(kRedBlocks, nrhs), kRedThreads, 0, ctx->stream>>>(r, z, nullptr, nullptr, n, ld, part,
                                                                                 Finish{nullptr, 3, S, counters(ctx)});
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status cg_rz<double>(mf_ctx*, const double*, const double*, int64_t, int64_t, int, double*);
template mf_status cg_rz<float>(mf_ctx*, const float*, const float*, int64_t, int64_t, int, double*);

template <typename T>
mf_status cg_init_scalars(mf_ctx* ctx, const T* r, const T* z, int64_t n, int64_t ld, int nrhs, double* S) {
  double* part;
  MF_TRY(scratch(ctx, 2 * kRedBlocks * size_t(nrhs), &part));
  k_dot2_partial<T, T><<<dim3(kRedBlocks, nrhs), kRedThreads, 0, ctx->stream>>>(r, r, r, z, n, ld, part,
                                                                                 Finish{nullptr, 4, S, counters(ctx)});
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status cg_init_scalars<double>(mf_ctx*, const double*, const double*, int64_t, int64_t, int, double*);
template mf_status cg_init_scalars<float>(mf_ctx*, const float*, const float*, int64_t, int64_t, int, double*);

mf_status stencil125_apply(mf_ctx* ctx, const void* Sv, const float* scale, const float* p, float* y, int nx, int ny,
                           int nz, double* Scg) {
  const __half* S = static_cast<const __half*>(Sv);
  const int64_t np = int64_t(nx + 1) * (ny + 1) * (nz + 1);
  if (np >= (int64_t(1) << 30)) return fail(MF_EUNSUPPORTED, "stencil grid too large for 32-bit indices");
  const int g = int(std::min<int64_t>((np + kRedThreads - 1) / kRedThreads, kRedBlocks));
  if (Scg) {
    double* part;
    MF_TRY(scratch(ctx, 2 * kRedBlocks, &part));
    k_stencil125<true><<<g, kRedThreads, 0, ctx->stream>>>(S, scale, p, y, nx, ny, nz, part,
                                                         Finish{nullptr, 1, Scg, counters(ctx)});
  } else {
    k_stencil125<false><<<g, kRedThreads, 0, ctx->stream>>>(S, scale, p, y, nx, ny, nz, nullptr, Finish{});
  }
  LAUNCH_CHECK();
  return MF_OK;
}

mf_status stencil_diag_inverse(mf_ctx* ctx, const void* S, const float* scale, int64_t n, float* pinv) {
  k_stencil_diag_inverse<<<unsigned((n + 255) / 256), 256, 0, ctx->stream>>>(static_cast<const __half*>(S), scale, n,
                                                                             pinv);
  LAUNCH_CHECK();
  return MF_OK;
}

template <typename T>
mf_status cg_update_p(mf_ctx* ctx, int64_t n, int64_t ld, int nrhs, const T* z, T* p, double* S, bool skip_inactive) {
  k_cg_p<T><<<dim3(grid_for(n), nrhs), 256, 0, ctx->stream>>>(n, ld, z, p, S, skip_inactive);
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status cg_update_p<double>(mf_ctx*, int64_t, int64_t, int, const double*, double*, double*, bool);
template mf_status cg_update_p<float>(mf_ctx*, int64_t, int64_t, int, const float*, float*, double*, bool);

template <typename T>
mf_status cheb_init(mf_ctx* ctx, int64_t n, int64_t ld, int nrhs, const T* r, const T* dinv, double inv_theta, T* d) {
  k_cheb_init<T><<<dim3(grid_for(n), nrhs), 256, 0, ctx->stream>>>(n, ld, r, dinv, T(inv_theta), d);
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status cheb_init<double>(mf_ctx*, int64_t, int64_t, int, const double*, const double*, double, double*);
template mf_status cheb_init<float>(mf_ctx*, int64_t, int64_t, int, const float*, const float*, double, float*);

template <typename T, int W>
static void cheb_launch(mf_ctx* ctx, dim3 grid, int64_t n, int64_t ld, T* z, const T* res_in, T* res, const T* Ad,
                        T* d, const T* dinv, T c1, T c2, bool first, bool last) {
  if (first && last)
    k_cheb_step<T, true, true, W><<<grid, 256, 0, ctx->stream>>>(n, ld, z, res_in, res, Ad, d, dinv, c1, c2);
  else if (first)
    k_cheb_step<T, true, false, W><<<grid, 256, 0, ctx->stream>>>(n, ld, z, res_in, res, Ad, d, dinv, c1, c2);
  else if (last)
    k_cheb_step<T, false, true, W><<<grid, 256, 0, ctx->stream>>>(n, ld, z, res_in, res, Ad, d, dinv, c1, c2);
  else
    k_cheb_step<T, false, false, W><<<grid, 256, 0, ctx->stream>>>(n, ld, z, res_in, res, Ad, d, dinv, c1, c2);
}

template <typename T>
mf_status cheb_step(mf_ctx* ctx, int64_t n, int64_t ld, int nrhs, T* z, const T* res_in, T* res, const T* Ad, T* d,
                    const T* dinv, double c1, double c2, bool first, bool last) {
  const dim3 grid(grid_for(n), nrhs);
  const auto a16 = [&](const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
  const bool words = a16(z) && a16(res_in) && a16(res) && a16(Ad) && a16(d) && a16(dinv) &&
                     (nrhs == 1 || (ld * int64_t(sizeof(T))) % 16 == 0);
  if (words)
    cheb_launch<T, int(16 / sizeof(T))>(ctx, grid, n, ld, z, res_in, res, Ad, d, dinv, T(c1), T(c2), first, last);
  else
    cheb_launch<T, 1>(ctx, grid, n, ld, z, res_in, res, Ad, d, dinv, T(c1), T(c2), first, last);
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status cheb_step<double>(mf_ctx*, int64_t, int64_t, int, double*, const double*, double*, const double*,
                                     double*, const double*, double, double, bool, bool);
template mf_status cheb_step<float>(mf_ctx*, int64_t, int64_t, int, float*, const float*, float*, const float*, float*,
                                    const float*, double, double, bool, bool);

// p starts on a 16-byte boundary and so does every vector ld elements further on
template <typename T> bool words16(const T* p, int64_t ld) {
  return reinterpret_cast<uintptr_t>(p) % 16 == 0 && (ld * int64_t(sizeof(T))) % 16 == 0;
}

template <typename T> mf_status multidot(mf_ctx* ctx, const T* V, int64_t ld, int k, const T* w, int64_t n, double* h) {
  if (k > 64) return fail(MF_EINVAL, "multidot: at most 64 vectors");
  const int g = kRedBlocks;
  double* part;
  MF_TRY(scratch(ctx, size_t(g) * (k + 1) + 64, &part));
  if (words16(V, ld) && words16(w, 0))
    k_multidot<T, 16 / sizeof(T)><<<g, kRedThreads, 0, ctx->stream>>>(V, ld, k, w, n, part);
  else
    k_multidot<T, 1><<<g, kRedThreads, 0, ctx->stream>>>(V, ld, k, w, n, part);
  LAUNCH_CHECK();
  k_multidot_finish<<<k, kRedThreads, 0, ctx->stream>>>(part, g, h);
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status multidot<double>(mf_ctx*, const double*, int64_t, int, const double*, int64_t, double*);
template mf_status multidot<float>(mf_ctx*, const float*, int64_t, int, const float*, int64_t, double*);

// groups up to 6 fp32 or 2 fp64 vectors: within the 64 registers of 4 blocks per SM (larger groups
// spill, and go to the two separate kernels)
template <typename T> constexpr int kAxpyDotMax = sizeof(T) == 4 ? 6 : 2;

template <typename T, int W>
static void launch_axpy_multidot(mf_ctx* ctx, const T* V, int64_t ld, int k, const double* h, double sign, T* w,
                                 int64_t n, double* part) {
  const int g = kRedBlocks;
  switch (k) {
    case 1: k_axpy_multidot<T, 1, W><<<g, kRedThreads, 0, ctx->stream>>>(V, ld, h, sign, w, n, part); break;
    case 2: k_axpy_multidot<T, 2, W><<<g, kRedThreads, 0, ctx->stream>>>(V, ld, h, sign, w, n, part); break;
    case 3:
      if constexpr (kAxpyDotMax<T> >= 3)
        k_axpy_multidot<T, 3, W><<<g, kRedThreads, 0, ctx->stream>>>(V, ld, h, sign, w, n, part);
      break;
    case 4:
      if constexpr (kAxpyDotMax<T> >= 4)
        k_axpy_multidot<T, 4, W><<<g, kRedThreads, 0, ctx->stream>>>(V, ld, h, sign, w, n, part);
      break;
    case 5:
      if constexpr (kAxpyDotMax<T> >= 5)
        k_axpy_multidot<T, 5, W><<<g, kRedThreads, 0, ctx->stream>>>(V, ld, h, sign, w, n, part);
      break;
    default:
      if constexpr (kAxpyDotMax<T> >= 6)
        k_axpy_multidot<T, 6, W><<<g, kRedThreads, 0, ctx->stream>>>(V, ld, h, sign, w, n, part);
      break;
  }
}

template <typename T>
mf_status axpy_multidot(mf_ctx* ctx, const T* V, int64_t ld, int k, const double* h, double sign, T* w, int64_t n,
                        double* h2) {
  if (k > kAxpyDotMax<T>) {
    MF_TRY(multiaxpy<T>(ctx, V, ld, k, h, sign, w, n));
    return multidot<T>(ctx, V, ld, k, w, n, h2);
  }
  if (k < 1) return MF_OK;
  const int g = kRedBlocks;
  double* part;
  MF_TRY(scratch(ctx, size_t(g) * (k + 1) + 64, &part));
  if (words16(V, ld) && words16(w, 0))
    launch_axpy_multidot<T, 16 / sizeof(T)>(ctx, V, ld, k, h, sign, w, n, part);
  else
    launch_axpy_multidot<T, 1>(ctx, V, ld, k, h, sign, w, n, part);
  LAUNCH_CHECK();
  k_multidot_finish<<<k, kRedThreads, 0, ctx->stream>>>(part, g, h2);
  LAUNCH_CHECK();
  return MF_OK;
}

template <typename T>
mf_status multiaxpy(mf_ctx* ctx, const T* V, int64_t ld, int k, const double* h, double sign, T* w, int64_t n,
                    double* norm2) {
  if (k > 64) return fail(MF_EINVAL, "multiaxpy: at most 64 vectors");
  if (k < 1 && !norm2) return MF_OK;
  const bool words = words16(V, ld) && words16(w, 0);
  const int g = grid_for(n);
  if (norm2) {
    double* part;
    MF_TRY(scratch(ctx, size_t(g), &part));
    const Finish fin{norm2, 0, nullptr, counters(ctx)};
    if (words)
      k_multiaxpy<T, 16 / sizeof(T), true><<<g, 256, 0, ctx->stream>>>(V, ld, k, h, sign, w, n, part, fin);
    else
      k_multiaxpy<T, 1, true><<<g, 256, 0, ctx->stream>>>(V, ld, k, h, sign, w, n, part, fin);
  } else if (words) {
    k_multiaxpy<T, 16 / sizeof(T), false><<<g, 256, 0, ctx->stream>>>(V, ld, k, h, sign, w, n, nullptr, Finish{});
  } else {
    k_multiaxpy<T, 1, false><<<g, 256, 0, ctx->stream>>>(V, ld, k, h, sign, w, n, nullptr, Finish{});
  }
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status multiaxpy<double>(mf_ctx*, const double*, int64_t, int, const double*, double, double*, int64_t,
                                     double*);
template mf_status multiaxpy<float>(mf_ctx*, const float*, int64_t, int, const double*, double, float*, int64_t,
                                    double*);
template mf_status axpy_multidot<double>(mf_ctx*, const double*, int64_t, int, const double*, double, double*, int64_t,
                                         double*);
template mf_status axpy_multidot<float>(mf_ctx*, const float*, int64_t, int, const double*, double, float*, int64_t,
                                        double*);

mf_status fill_splitmix(mf_ctx* ctx, uint64_t seed, double* v, int64_t n) {
  k_splitmix<<<grid_for(n), 256, 0, ctx->stream>>>(seed, v, n);
  LAUNCH_CHECK();
  return MF_OK;
}

mf_status set_list(mf_ctx* ctx, double* v, const int32_t* list, int64_t n, double val) {
  if (n == 0) return MF_OK;
  k_set_list<<<int((n + 255) / 256), 256, 0, ctx->stream>>>(v, list, n, val);
  LAUNCH_CHECK();
  return MF_OK;
}
template <typename T> mf_status zero_list(mf_ctx* ctx, T* v, const int32_t* list, int64_t n) {
  if (n == 0) return MF_OK;
  k_zero_list<T><<<int((n + 255) / 256), 256, 0, ctx->stream>>>(v, list, n);
  LAUNCH_CHECK();
  return MF_OK;
}
template mf_status zero_list<double>(mf_ctx*, double*, const int32_t*, int64_t);
template mf_status zero_list<float>(mf_ctx*, float*, const int32_t*, int64_t);

// ---------------------------------------------------------------------------------------
// Allocation-free inner products (mf_dot_noalloc).
//
// Some callers cannot let this library call cudaMalloc: an application that owns all device
// memory through its own pool and gives libraries a fixed budget, a latency-critical loop in
// which an allocation could implicitly synchronise the device and stall other streams, or code
// that has no mf_ctx (creating one allocates the context's reduction workspace).  For them the
// block partial sums live in one statically sized device array of this file instead of the
// context workspace.  Every GPU that loads the library holds the array until the process exits.
// Host code may not use the array's name as a device address (on the host it only stands in for
// the symbol), so its device address is looked up once per device with cudaGetSymbolAddress,
// with that device current, on the first call made on that device; that first call should come
// before any stream capture.  All calls share the array and it keeps the last call's partials:
// nothing in it needs to start at zero, because the partial kernel writes every slot that the
// finishing kernel then reads.  Calls that overlap on the GPU (several streams, several host
// threads) race on the array; callers must serialise them.
constexpr int kNoAllocMaxVec = 16;
static __device__ __align__(256) double g_noalloc_partials[2 * kRedBlocks * kNoAllocMaxVec];

namespace {
std::mutex g_noalloc_mutex;
double* g_noalloc_address[256] = {};
}  // namespace

static mf_status noalloc_workspace(double** out) {
  int dev = -1;
  MF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(MF_EINVAL, "device index outside the allocation-free table");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_address[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p)
      return fail(MF_ECUDA, std::string("cudaGetSymbolAddress of the allocation-free workspace: ") +
                                cudaGetErrorString(e));
    g_noalloc_address[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_address[dev];
  return MF_OK;
}

template <typename T>
static mf_status dot_noalloc(const T* x, const T* y, int64_t n, int64_t ld, int nvec, double* out, cudaStream_t s) {
  double* part = nullptr;
  MF_TRY(noalloc_workspace(&part));
  k_dot2_partial<T, T><<<dim3(kRedBlocks, nvec), kRedThreads, 0, s>>>(x, y, nullptr, nullptr, n, ld, part,
                                                                       Finish{nullptr, 0, nullptr, nullptr});
  MF_CUDA_TRY(cudaGetLastError());
  k_finish<<<nvec, kRedThreads, 0, s>>>(part, kRedBlocks, out, 0, nullptr);
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

}  // namespace mf

extern "C" mf_status mf_dot_noalloc(const void* x, const void* y, int64_t n, int64_t ld, int nvec, int dtype,
                                    double* out, void* cuda_stream) {
  using namespace mf;
  try {
    if (!x || !y || !out) return fail(MF_EINVAL, "NULL argument");
    if (nvec < 1 || nvec > kNoAllocMaxVec)
      return fail(MF_EINVAL, "mf_dot_noalloc: nvec must be in 1.." + std::to_string(kNoAllocMaxVec) +
                                 " (size of its static workspace)");
    if (n < 0 || (nvec > 1 && ld < n)) return fail(MF_EINVAL, "need n >= 0 and ld >= n");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (dtype == MF_F64) return dot_noalloc<double>((const double*)x, (const double*)y, n, ld, nvec, out, s);
    if (dtype == MF_F32) return dot_noalloc<float>((const float*)x, (const float*)y, n, ld, nvec, out, s);
    return fail(MF_EUNSUPPORTED, "dot precision must be MF_F64 or MF_F32");
  } catch (...) {
    return fail(MF_EINVAL, "exception in mf_dot_noalloc");
  }
}
