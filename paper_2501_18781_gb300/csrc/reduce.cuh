// Device-side pieces of the deterministic reductions (internal): block sums, compensated fp32
// dot products, and the finishing step that the last block of a reduction runs.
#pragma once

#include "vec.cuh"

namespace mf {
namespace {

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kRedThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < kRedThreads / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;  // valid in thread 0
}

// fp32 data: GB300's fp64 pipe (1/64 of the fp32 rate) cannot keep up with HBM if every
// element is converted and accumulated in fp64 (a conversion and an fp64 FMA per 4-byte
// element).  Within a thread, fp32 products and sums are therefore carried as unevaluated
// pairs of floats: the product error by an FMA (a*b = p + e exactly) and the sum error by
// Knuth's two-sum, i.e. the compensated dot product of Ogita, Rump and Oishi ("Accurate sum
// and dot product", SIAM J. Sci. Comput. 26, 2005), whose result is as accurate as a dot
// product evaluated in twice the working precision.  Partials leave the thread as
// double(s) + double(c) and are reduced in fp64.
struct Dot2f {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float t = s + p;
    const float z = t - s;
    c += ((s - (t - z)) + (p - z)) + e;
    s = t;
  }
  __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

// What the sum of a row of g partials feeds (row r; mode 0: out[r] = sum; 1: pAp and alpha;
// 2: rr, rz (second row), beta; 3: rz and beta; 4: rr and rz; 5: rr).  count: one arrival
// counter per row (zero between launches); NULL when a separate k_finish launch does the sum.
struct Finish {
  double* out;
  int mode;
  double* S;
  unsigned* count;
};

// Sums row r of the partials in a fixed order (so results are reproducible bit for bit) and
// applies the mode.  The loads go to L2: in the fused form other blocks of the same launch
// wrote the partials.
__device__ void finish_row(const double* part, int g, int r, const Finish& f) {
  const double* pr = part + int64_t(r) * 2 * g;
  double s = 0.0;
  for (int i = threadIdx.x; i < g; i += blockDim.x) s += __ldcg(pr + i);
  s = block_sum(s);
  double s2 = 0.0;
  if (f.mode == 2 || f.mode == 4) {
    for (int i = threadIdx.x; i < g; i += blockDim.x) s2 += __ldcg(pr + g + i);
    s2 = block_sum(s2);
  }
  if (threadIdx.x == 0) {
    double* Sr = f.S ? f.S + r * S_NSCAL : nullptr;
    if (f.mode == 0) f.out[r] = s;
    else if (f.mode == 1) {
      Sr[S_PAP] = s;
      Sr[S_ALPHA] = (Sr[S_ACTIVE] != 0.0 && s != 0.0) ? Sr[S_RZ] / s : 0.0;
    } else if (f.mode == 2 || f.mode == 3) {
      const double rz = f.mode == 2 ? s2 : s;
      if (f.mode == 2) Sr[S_RR] = s;
      Sr[S_RZN] = rz;
      Sr[S_BETA] = (Sr[S_ACTIVE] != 0.0 && Sr[S_RZ] != 0.0) ? rz / Sr[S_RZ] : 0.0;
      Sr[S_RZ] = rz;
    } else if (f.mode == 4) {
      Sr[S_RR] = s;
      Sr[S_RZ] = s2;
    } else if (f.mode == 5) {
      Sr[S_RR] = s;
    }
  }
}

// Called by every thread after thread 0 stored the block's partials of row blockIdx.y: the last
// block of the row to arrive sums the row (finish_row) and resets the counter for the next launch.
__device__ __forceinline__ void finish_if_last(const double* part, const Finish& f) {
  if (!f.count) return;
  __shared__ unsigned last;
  __threadfence();  // this block's partials are visible device-wide before it is counted
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(f.count + blockIdx.y, 1u) == gridDim.x - 1 ? 1u : 0u;
  __syncthreads();
  if (!last) return;
  __threadfence();
  finish_row(part, gridDim.x, blockIdx.y, f);
  if (threadIdx.x == 0) f.count[blockIdx.y] = 0u;
}

}  // namespace
}  // namespace mf
