// Double-float apply of the conservative level-set reinitialisation operator on adaptively refined
// (octree) meshes with hanging-node constraints: (1/dtau) M + eps N_n, N_n(u, v) = int (n.grad u)
// (n.grad v) (Section 2.3 reinitialisation, Appendix B matrix-free evaluation), n the unit normal of
// the level set per Gauss point (the operator's fp64 table, as float pairs).
//
// One thread per leaf, cells in the map's processing order (unconstrained first).  The cell's 27
// values are gathered through the cell map in fp64 (a hanging node as the weighted sum of its
// masters), scaled by one power of two per warp and split into float pairs; values and derivatives
// at the Gauss points run in double-float on the fp32 pipes.  Every flux of this operator is
// s n with s = w eps h (n . grad u), so one pass forms s at the 27 Gauss points, parked in a second
// shared-memory column (55 KB per block, four blocks per SM; kept in registers it spilled 3 KB and ran
// 10 % slower on eight right-hand sides);
// the test side is then accumulated one z-plane at a time: the value term and the z part
// sum_q' D[q'][qc] s n_z, then the x and y parts s n_x, s n_y through the plane's transposed sweeps,
// parked in the thread's shared-memory column; the z sweep runs at the end.  The cell's contributions
// are joined to doubles and added to the free DoFs, hanging ones through the constraint weights.
#include "df_pairs.cuh"

namespace mf {

MF_DEFINE_TABLE_UPLOAD

OctGeom oct_geom(const mf_dofmap* m);

namespace {

constexpr int kOctThreads = 128;

struct DfOctArgs {
  const double* src;
  double* dst;
  int nrhs;           // right-hand sides, one per blockIdx.y
  int64_t ld;         // distance between right-hand sides
  const float* nh;    // [3][27][ncells] unit normal per Gauss point, high parts
  const float* nl;    //                 low parts
  int64_t ncells;     // stride of the normal table
  float eh_h, eh_l;   // eps h0 (h0: edge of a level-0 cell)
  float mh_h, mh_l;   // m h0^3 (m: value coefficient 1 / dtau)
};

__device__ __forceinline__ dd dd_scale2(dd a, float s) { return {a.h * s, a.l * s}; }   // s a power of two
__device__ __forceinline__ float pow2f_oct(int e) { return __uint_as_float(unsigned(e + 127) << 23); }

__global__ void __launch_bounds__(kOctThreads, 4) k_reinit_df_octree(DfOctArgs A, OctGeom og) {
  extern __shared__ float oct_smem[];
  float(*sh)[kOctThreads] = reinterpret_cast<float(*)[kOctThreads]>(oct_smem);
  float(*sl)[kOctThreads] = reinterpret_cast<float(*)[kOctThreads]>(oct_smem + 27 * kOctThreads);
  float(*zh)[kOctThreads] = reinterpret_cast<float(*)[kOctThreads]>(oct_smem + 54 * kOctThreads);
  float(*zl)[kOctThreads] = reinterpret_cast<float(*)[kOctThreads]>(oct_smem + 81 * kOctThreads);
  const int t = threadIdx.x;
  const int64_t slot = int64_t(blockIdx.x) * kOctThreads + t;
  const bool active = slot < og.ncells;
  const int64_t cell = active ? __ldg(og.order + slot) : 0;
  const int lev = active ? __ldg(og.level + cell) : 0;
  const double* __restrict__ src = A.src + int64_t(blockIdx.y) * A.ld;
  int bias = 0;
  {
    // the map entries live only here and are read again for the scatter (fewer live registers)
    int32_t id[27];
#pragma unroll
    for (int l = 0; l < 27; ++l) id[l] = active ? __ldg(og.cmap + l * og.ncp + cell) : 0;
    double X[27];
#pragma unroll
    for (int l = 0; l < 27; ++l) X[l] = active ? __ldg(src + (id[l] >= 0 ? id[l] : 0)) : 0.0;
    if (active) {
#pragma unroll
      for (int l = 0; l < 27; ++l) {
        if (id[l] >= 0) {
          if (og.dflag && __ldg(og.dflag + id[l])) X[l] = 0.0;
          continue;
        }
        const int r = -1 - id[l];
        double v = 0.0;
        for (int e = __ldg(og.rowptr + r); e < __ldg(og.rowptr + r + 1); ++e) {
          const int32_t m = __ldg(og.cols + e);
          if (!(og.dflag && __ldg(og.dflag + m))) v += __ldg(og.w64 + e) * __ldg(src + m);
        }
        X[l] = v;
      }
    }
    int emax = 0;
#pragma unroll
    for (int l = 0; l < 27; ++l) emax = max(emax, (__double2hiint(X[l]) >> 20) & 0x7FF);
    emax = int(__reduce_max_sync(0xffffffffu, unsigned(emax)));
    bias = emax ? emax - 1023 : 0;
    dd U[27];
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
  auto nrm = [&](int d, int q) {
    const int64_t o = (d * 27 + q) * A.ncells + cell;
    return active ? dd{__ldg(A.nh + o), __ldg(A.nl + o)} : dd{0.f, 0.f};
  };
  auto W3 = [&](int q) { return dd{cW3h[q], cW3l[q]}; };
  // w eps h at the cell's level (h = h0 2^-level, an exact power-of-two scale)
  const dd eh = dd_scale2(dd{A.eh_h, A.eh_l}, pow2f_oct(-lev));
  // s(q) = w eps h (n . grad u) at the 27 Gauss points
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const int qa = q % 3, qb = (q / 3) % 3, qc = q / 9;
    const int bx = q - qa, by = q - 3 * qb, bz = q - 9 * qc;
    const dd gx = ddline(qa, Uq(bx), Uq(bx + 1), Uq(bx + 2));
    const dd gy = ddline(qb, Uq(by), Uq(by + 3), Uq(by + 6));
    const dd gz = ddline(qc, Uq(bz), Uq(bz + 9), Uq(bz + 18));
    const dd ng = dd_fma(dd_fma(dd_mul(nrm(0, q), gx), nrm(1, q), gy), nrm(2, q), gz);
    const dd sq = dd_norm(dd_mul(dd_mul(W3(q), eh), dd_norm(ng)));
    zh[q][t] = sq.h;
    zl[q][t] = sq.l;
  }
  auto S = [&](int q) { return dd{zh[q][t], zl[q][t]}; };
  // w m h^3 at the cell's level
  const dd mh = dd_scale2(dd{A.mh_h, A.mh_l}, pow2f_oct(-3 * lev));
#pragma unroll
  for (int qc = 0; qc < 3; ++qc) {
    dd R[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      const int q = p + 9 * qc;
      dd acc = dd_mul(dd_mul(W3(q), mh), Uq(q));
#pragma unroll
      for (int c2 = 0; c2 < 3; ++c2)
        if (c2 != 1 || qc != 1) acc = dd_fma(acc, cD(c2, qc), dd_mul(S(p + 9 * c2), nrm(2, p + 9 * c2)));
      R[p] = acc;
    }
#pragma unroll
    for (int qb = 0; qb < 3; ++qb)
#pragma unroll
      for (int qa = 0; qa < 3; ++qa) {
        const int p = qa + 3 * qb, q = p + 9 * qc;
        const dd sq = S(q);
        const dd fx = dd_mul(sq, nrm(0, q)), fy = dd_mul(sq, nrm(1, q));
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
  if (!active) return;
  dd R[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) R[q] = Uq(q);
  dsweep_t<2>(R);
  double* __restrict__ dst = A.dst + int64_t(blockIdx.y) * A.ld;
#pragma unroll
  for (int l = 0; l < 27; ++l) {
    const double v = f2d_bits(R[l].h, bias) + f2d_bits(R[l].l, bias);
    const int32_t idl = __ldg(og.cmap + l * og.ncp + cell);
    if (idl >= 0) {
      if (!(og.dflag && __ldg(og.dflag + idl))) atomicAdd(dst + idl, v);
      continue;
    }
    const int r = -1 - idl;
    for (int e = __ldg(og.rowptr + r); e < __ldg(og.rowptr + r + 1); ++e) {
      const int32_t m = __ldg(og.cols + e);
      if (!(og.dflag && __ldg(og.dflag + m))) atomicAdd(dst + m, __ldg(og.w64 + e) * v);
    }
  }
}

}  // namespace

mf_status launch_reinit_df_octree(mf_ctx* ctx, const mf_dofmap* m, const double* src, double* dst, int nrhs,
                                  int64_t ld, const float* nh, const float* nl, double eps, double mass) {
  if (m->uniform || m->degree != 2) return fail(MF_EINVAL, "the double-float octree kernel takes octree Q2 maps");
  MF_CUDA_TRY(upload_tables_here());
  const OctGeom og = oct_geom(m);
  DfOctArgs a{};
  a.src = src;
  a.dst = dst;
  a.nrhs = nrhs;
  a.ld = ld;
  a.nh = nh;
  a.nl = nl;
  a.ncells = m->n_cells;
  const double h0 = m->mesh->h0, eh = eps * h0, mh = mass * h0 * h0 * h0;
  a.eh_h = float(eh);
  a.eh_l = float(eh - double(a.eh_h));
  a.mh_h = float(mh);
  a.mh_l = float(mh - double(a.mh_h));
  const dim3 grid(unsigned((m->n_cells + kOctThreads - 1) / kOctThreads), unsigned(nrhs));
  static bool attrs = false;
  if (!attrs) {
    MF_CUDA_TRY(cudaFuncSetAttribute(k_reinit_df_octree, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(108 * kOctThreads * sizeof(float))));
    attrs = true;
  }
  k_reinit_df_octree<<<grid, kOctThreads, 108 * kOctThreads * sizeof(float), ctx->stream>>>(a, og);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

}  // namespace mf
