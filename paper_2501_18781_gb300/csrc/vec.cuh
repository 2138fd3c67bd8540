// Vector kernels of the Krylov solvers (internal): deterministic fp64-accumulated dot
// products, fused CG / Chebyshev updates, CGS2 multi-dot and multi-axpy for GMRES.
#pragma once

#include "internal.h"

namespace mf {

constexpr int kRedBlocks = 608;   // 4 x 152 SMs: fixed grid, so reductions are deterministic
constexpr int kRedThreads = 256;
constexpr size_t kScratchDoubles = size_t(2) * kRedBlocks * 64;  // up to 64 right-hand sides

// partial sums (kRedBlocks doubles) then one-block finish into out[0]
template <typename TX, typename TY>
mf_status dot(mf_ctx* ctx, const TX* x, const TY* y, int64_t n, double* out);
mf_status norm2_sq(mf_ctx* ctx, const double* x, int64_t n, double* out);
// out[k] = x_k . y_k for nvec vector pairs ld apart (device out; fp64 accumulation for fp64
// data, compensated fp32 pairs within a thread for fp32 data, fp64 across threads)
template <typename T>
mf_status dot_batched(mf_ctx* ctx, const T* x, const T* y, int64_t n, int64_t ld, int nvec, double* out);

// y = a x + b y (host scalars), mixed precisions allowed
template <typename TX, typename TY>
mf_status axpby(mf_ctx* ctx, int64_t n, double a, const TX* x, double b, TY* y);
// z = d .* r (Jacobi); d may be NULL (identity)
template <typename T> mf_status pointwise_mul(mf_ctx* ctx, int64_t n, const T* d, const T* r, T* z);
// Oseen block Jacobi: z_u = B^-1 r_u per node, z_p = pinv .* r_p
template <typename T>
mf_status block_jacobi(mf_ctx* ctx, int64_t nu, int64_t np, const double* blk, const double* pinv, const T* r, T* z);
template <typename TS, typename TD> mf_status convert(mf_ctx* ctx, int64_t n, const TS* s, TD* d);
// velocity part only, fp32 block inverses stored entry-major (entry e of node i at e nu + i):
// z_u = B^-1 r_u per node
mf_status block_jacobi_u32(mf_ctx* ctx, int64_t nu, const float* blk, const float* r, float* z);
// velocity part only: dst = s[0] src (s device; dst may equal src), then z_u = B^-1 dst per node
mf_status block_jacobi_u32_scaled(mf_ctx* ctx, int64_t nu, const float* blk, const double* s, const float* src,
                                  float* dst, float* z);

// Batched CG pieces: nrhs systems, vectors ld apart, device scalars S[r * S_NSCAL + k]:
// 0 rz, 1 pAp, 2 alpha, 3 beta, 4 rr, 5 rz_new, 6 active (1 = still iterating)
enum { S_RZ = 0, S_PAP = 1, S_ALPHA = 2, S_BETA = 3, S_RR = 4, S_RZN = 5, S_ACTIVE = 6, S_NSCAL = 8 };
// S[pAp] = p.Ap, S[alpha] = active ? rz / pAp : 0
template <typename T> mf_status cg_alpha(mf_ctx* ctx, const T* p, const T* Ap, int64_t n, int64_t ld, int nrhs, double* S);
// x += alpha p; r -= alpha Ap; then (zmode 1) z = dinv .* r, S[rz] = r.z, beta; (zmode 0) z := r
// implicitly (S[rz] = r.r); (zmode 2) only S[rr].  skip_inactive: systems whose active flag is 0
// are left untouched (an inner CG with an on-device stopping test)
template <typename T>
mf_status cg_update_xr(mf_ctx* ctx, int64_t n, int64_t ld, int nrhs, T* x, T* r, const T* p, const T* Ap,
                       const T* dinv, T* z, int zmode, double* S, bool skip_inactive = false);
// S[rz] = r.z and beta (preconditioner applied separately)
template <typename T> mf_status cg_rz(mf_ctx* ctx, const T* r, const T* z, int64_t n, int64_t ld, int nrhs, double* S);
// 125-point stencils on a grid of n nodes (offsets o = (ox + 2) + 5 (oy + 2) + 25 (oz + 2)) are
// stored as fp16 entries scaled by a per-row fp32 factor (the row's largest magnitude, so every
// entry lies in [-1, 1] and keeps 11 bits relative to the row's largest), rows padded to 128
// entries (the last three 0), in tiles of 32 rows: within a tile, entry group o / 8 of all 32 rows,
// then the next group, each row's eight entries one 16-byte word.  A warp's 16 coefficient loads
// are then 16 consecutive 512-byte runs.  stencil_at: where entry o of row i lives (in halves);
// stencil_halves: the size; the scales are a separate array of n floats.
__host__ __device__ inline int64_t stencil_at(int o, int64_t i) {
  return (i >> 5) * (128 * 32) + (o >> 3) * 256 + (i & 31) * 8 + (o & 7);
}
inline int64_t stencil_halves(int64_t n) { return (n + 31) / 32 * (128 * 32); }
// y = S p for a 125-point stencil on the (nx + 1) x (ny + 1) x (nz + 1) grid (S: the fp16 entries,
// scale: the row factors); with Scg non-NULL also Scg[pAp] = p.y and Scg[alpha] as cg_alpha sets
// them, in the same launch, and nothing at all once Scg's active flag is 0
mf_status stencil125_apply(mf_ctx* ctx, const void* S, const float* scale, const float* p, float* y, int nx, int ny,
                           int nz, double* Scg);
// pinv[i] = 1 / (the stencil's diagonal entry of row i) where that is positive, else unchanged
mf_status stencil_diag_inverse(mf_ctx* ctx, const void* S, const float* scale, int64_t n, float* pinv);
// p = z + beta p (z = r when z is NULL); skip_inactive as for cg_update_xr
template <typename T>
mf_status cg_update_p(mf_ctx* ctx, int64_t n, int64_t ld, int nrhs, const T* z, T* p, double* S,
                      bool skip_inactive = false);
// S[rr] = r.r, S[rz] = r.z (initial)
template <typename T> mf_status cg_init_scalars(mf_ctx* ctx, const T* r, const T* z, int64_t n, int64_t ld, int nrhs, double* S);

// Chebyshev (nrhs vectors ld apart, one diagonal).  The iteration z_0 = 0, res_0 = r,
// d_0 = dinv r / theta, then per step k: z_{k+1} = z_k + d_k, res_{k+1} = res_k - A d_k,
// d_{k+1} = c1 d_k + c2 dinv res_{k+1}, and the result z_m + d_m after the last step m - 1.
// cheb_init writes d_0 only; the first step reads r for res_0 and writes z = d_0 without reading it;
// the last step writes z_m + d_m and neither res nor d (same sums in the same order).
template <typename T>
mf_status cheb_init(mf_ctx* ctx, int64_t n, int64_t ld, int nrhs, const T* r, const T* dinv, double inv_theta, T* d);
template <typename T>
mf_status cheb_step(mf_ctx* ctx, int64_t n, int64_t ld, int nrhs, T* z, const T* res_in, T* res, const T* Ad, T* d,
                    const T* dinv, double c1, double c2, bool first, bool last);

// GMRES: h[0..k) = V^T w (V: k vectors of length n, stride ld), into device h (fp64 sums)
template <typename T> mf_status multidot(mf_ctx* ctx, const T* V, int64_t ld, int k, const T* w, int64_t n, double* h);
// w += sign V h (h device, k entries); with norm2 non-NULL also *norm2 = |w|^2 of the result
// (device, fp64 sum), in the same launch
template <typename T>
mf_status multiaxpy(mf_ctx* ctx, const T* V, int64_t ld, int k, const double* h, double sign, T* w, int64_t n,
                    double* norm2 = nullptr);
// w += sign V h, then h2[0..k) = V^T w: the first Gram-Schmidt pass's update and the second
// pass's products, in one sweep over V for up to 6 fp32 / 2 fp64 vectors (the same results as
// multiaxpy then multidot, which it calls for more)
template <typename T>
mf_status axpy_multidot(mf_ctx* ctx, const T* V, int64_t ld, int k, const double* h, double sign, T* w, int64_t n,
                        double* h2);
// splitmix64 uniform [-1,1) vector (own implementation of the published generator)
mf_status fill_splitmix(mf_ctx* ctx, uint64_t seed, double* v, int64_t n);
// v[list[i]] = val
mf_status set_list(mf_ctx* ctx, double* v, const int32_t* list, int64_t n, double val);
template <typename T> mf_status zero_list(mf_ctx* ctx, T* v, const int32_t* list, int64_t n);

}  // namespace mf
