// Krylov solvers on the matrix-free operators (Appendix B: CG for symmetric and GMRES for
// nonsymmetric systems), Jacobi / Chebyshev / block-Jacobi preconditioning, mixed-precision
// defect correction, the heat-step adjoint gradient and the apply autotuner.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <memory>
#include <type_traits>
#include <vector>

#include "ops.h"
#include "vec.cuh"

namespace mf {

template <typename T>
mf_status apply_impl(mf_op* op, const T* src, T* dst, int nrhs, int64_t ld, bool transpose, int prec = -1);
mf_status diag64(mf_op* op, double** out);
mf_status oseen_blocks32(mf_op* op, float* blk, float* pinv);
mf_status check_fields(const mf_op* op);
bool heat_convection(const mf_op* op);
int qk_degree(const mf_op* op);
bool heat_tabulated(const mf_op* op);
mf_status ensure_tables(mf_op* op);
int scalar_kind(const mf_op* op);
double value_coef(const mf_op* op);
template <typename T> ScalarArgs<T> scalar_args(const mf_op* op, const T* src, T* dst, int nrhs, int64_t ld);
template <typename T> mf_status oseen_coupling(mf_op* op, int which, const T* src, T* dst);
// device-side stopping test and Givens kernels of the inner solves (solver_kernels.cu)
mf_status dev_cg_tol_init(mf_ctx* c, double* S, double tol2);
mf_status dev_cg_tol_check(mf_ctx* c, double* S, double* steps);
mf_status dev_cg_tol_init_batched(mf_ctx* c, double* S, double tol2, int nrhs);
mf_status dev_cg_tol_check_batched(mf_ctx* c, double* S, double* steps, int nrhs);
mf_status dev_gmres_begin(mf_ctx* c, const double* nrm2, double* G, int m);
mf_status dev_gmres_column(mf_ctx* c, const double* h, double* G, int m, int j);
mf_status dev_gmres_solve(mf_ctx* c, const double* G, int m, int j, double* y);
// small device helpers (solver_kernels.cu)
template <typename T> mf_status dev_scale_mul(mf_ctx* c, const double* s, const double* v, T* out, int64_t n);
template <typename T> mf_status dev_scale_mul_back(mf_ctx* c, const double* s, const T* v, double* out, int64_t n);

namespace {

using clk = std::chrono::steady_clock;

// Work vector of a solver: inside a solve its memory comes from the context's block pool and goes
// back there when the vector dies; elsewhere it is a plain device buffer.
template <typename T> struct Vec {
  DevBuf b;
  BlockPool* pool = nullptr;
  void* blk = nullptr;
  size_t nb = 0;
  T* p = nullptr;
  Vec() = default;
  Vec(const Vec&) = delete;
  Vec& operator=(const Vec&) = delete;
  ~Vec() { drop(); }
  void drop() {
    if (blk) pool->put(blk, nb);
    blk = nullptr;
    pool = nullptr;
    b.release();
    p = nullptr;
  }
  // exchange two vectors' memory (pooled or not) and ownership
  void swap_with(Vec& o) {
    std::swap(b.p, o.b.p);
    std::swap(b.bytes, o.b.bytes);
    std::swap(pool, o.pool);
    std::swap(blk, o.blk);
    std::swap(nb, o.nb);
    std::swap(p, o.p);
  }
  mf_status alloc(int64_t n) {
    drop();
    const size_t bytes = sizeof(T) * size_t(n);
    if (tl_pool && bytes > 0) {
      MF_TRY(tl_pool->get(bytes, &blk));
      pool = tl_pool;
      nb = bytes;
      p = static_cast<T*>(blk);
    } else {
      MF_TRY(b.alloc(bytes));
      p = b.as<T>();
    }
    return MF_OK;
  }
};

mf_status sync_copy(mf_ctx* c, double* host, const double* dev, size_t n) {
  MF_CUDA_TRY(cudaMemcpyAsync(host, dev, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MF_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return MF_OK;
}

// Krylov basis vectors are stored this many elements apart: n rounded up to 64, so that every
// vector starts on a 256-byte boundary and the CGS2 kernels move 16-byte words.
inline int64_t basis_stride(int64_t n) { return (n + 63) / 64 * 64; }

// Records what fn launches on the context's stream into an executable graph.  The capture runs
// on a private stream (nothing executes during a capture, so the work queued on the context's
// stream needs no fence); *kernels = the kernel launches the graph holds, which each replay adds
// to the context's launch count.
template <typename F> mf_status capture_graph(mf_ctx* c, F&& fn, cudaGraphExec_t* exec, int64_t* kernels) {
  if (!c->capture_stream) {
    MF_CUDA_TRY(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
    MF_CUDA_TRY(cudaEventCreateWithFlags(&c->fence, cudaEventDisableTiming));
  }
  cudaGraph_t g;
  cudaStream_t orig = c->stream;
  const int64_t before = c->launches;
  c->stream = c->capture_stream;
  MF_CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  mf_status st = fn();
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  c->stream = orig;
  *kernels = c->launches - before;
  c->launches = before;
  if (st != MF_OK) {
    if (e == cudaSuccess) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(MF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(MF_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return MF_OK;
}

// largest eigenvalue of the symmetric tridiagonal (a, b) by Sturm-sequence bisection
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int m = int(a.size());
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {  // eigenvalues < x
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
      d = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-14 * std::max(1.0, std::fabs(hi)); ++it) {
    double mid = 0.5 * (lo + hi);
    if (count_below(mid) == m) hi = mid;
    else lo = mid;
  }
  return hi;
}

// Givens rotation of column j of the (m+1) x m Hessenberg H (row-major, m columns) with the
// previous rotations, then the new rotation that zeroes H[j+1][j]; updates g.
void givens_column(std::vector<double>& H, int m, int j, std::vector<double>& cs, std::vector<double>& sn,
                   std::vector<double>& g) {
  for (int i = 0; i < j; ++i) {
    const double tmp = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
    H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
    H[i * m + j] = tmp;
  }
  const double den = std::hypot(H[j * m + j], H[(j + 1) * m + j]);
  cs[j] = den > 0 ? H[j * m + j] / den : 1.0;
  sn[j] = den > 0 ? H[(j + 1) * m + j] / den : 0.0;
  H[j * m + j] = den;
  H[(j + 1) * m + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
}

// y = R^-1 g for the leading j x j upper triangle of H (m columns)
void back_substitute(const std::vector<double>& H, int m, int j, const std::vector<double>& g, std::vector<double>& y) {
  for (int i = j - 1; i >= 0; --i) {
    double s = g[i];
    for (int k = i + 1; k < j; ++k) s -= H[i * m + k] * y[k];
    y[i] = H[i * m + i] != 0.0 ? s / H[i * m + i] : 0.0;
  }
}

// Block upper-triangular preconditioner of the Oseen saddle-point system [[A, B^T], [B, 0]]:
//   P = [[A, B^T], [0, -S]],  P^-1 r:  z_p = -S^-1 r_p,  z_u = A^-1 (r_u - B^T z_p),
// with S ~ S~ = B D^-1 B^T (D: the 3x3 nodal blocks of A), assembled once as a 125-point stencil
// on the pressure grid and solved by Jacobi-CG (Jacobi: its inverse diagonal), and A^-1 by a few
// D^-1-preconditioned GMRES steps.  Both inner solves keep fp32 vectors and fp32 operator
// arithmetic (the Schur CG on the stencil, stored as row-scaled fp16; the velocity GMRES on the
// whole operator applied to [v; 0]); inner products accumulate in fp64, and the stopping test,
// Givens rotations and triangular solve run on the device, so a preconditioner call needs no host
// round trip.
struct OseenBlockTri {
  mf_op* op = nullptr;
  int64_t n = 0, nu = 0, nu3 = 0, np = 0;
  int ku = 10, smax = 30;
  double stol = 0.1;
  Vec<float> blk32, ua, pinv32, xp, rp, zp, pp, sp, V, t, w;
  DevBuf stil;        // S~ = B D^-1 B^T as a 125-point stencil on the pressure grid (fp16 entries)
  Vec<float> stscale;  // and its row factors
  int gn[3] = {0, 0, 0};  // cells per axis
  int64_t ldv = 0;  // stride of the basis vectors in V
  Vec<double> gst, y;
  // graph replay: a call launches the same sequence every time (several hundred small kernels),
  // so it is recorded once, between fixed input and output vectors, and replayed
  bool use_graph = false;
  int calls = 0;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_kernels = 0;
  Vec<double> rin, zout;

  ~OseenBlockTri() {
    if (exec) cudaGraphExecDestroy(exec);
  }

  mf_status setup(mf_op* o, int velocity_steps, int schur_maxit, double schur_tol) {
    op = o;
    mf_ctx* c = op->ctx;
    n = op->n;
    nu = op->map[0]->n_dofs;
    nu3 = 3 * nu;
    np = op->map[1]->n_dofs;
    ku = velocity_steps > 0 ? velocity_steps : 10;
    if (ku > 60) return fail(MF_EINVAL, "velocity_steps must be at most 60");
    smax = schur_maxit > 0 ? schur_maxit : 30;
    stol = schur_tol > 0 ? schur_tol : 0.1;
    // fp32 3x3 block inverses and inverse pressure scaling, computed in fp32 (the preconditioner
    // applies them in fp32)
    MF_TRY(blk32.alloc(9 * nu));
    for (Vec<float>* v : {&pinv32, &xp, &rp, &zp, &pp, &sp}) MF_TRY(v->alloc(np));
    MF_TRY(oseen_blocks32(op, blk32.p, pinv32.p));
    for (int d = 0; d < 3; ++d) gn[d] = op->map[0]->mesh->n[d];
    MF_TRY(stil.alloc(2 * size_t(stencil_halves(np))));
    MF_TRY(stscale.alloc(np));
    MF_TRY(launch_schur_assemble_f32(c, op->map[0], blk32.p, stil.p, stscale.p));
    MF_TRY(ua.alloc(nu3));
    // Jacobi of the Schur CG: diag(S~)^-1 (the pressure scaling above where it is not positive)
    MF_TRY(stencil_diag_inverse(c, stil.p, stscale.p, np, pinv32.p));
    ldv = basis_stride(n);
    MF_TRY(V.alloc(ldv * (ku + 1)));
    MF_TRY(t.alloc(n));
    MF_TRY(w.alloc(n));
    MF_CUDA_TRY(cudaMemsetAsync(t.p, 0, sizeof(float) * n, c->stream));  // its pressure block stays 0
    MF_CUDA_TRY(cudaMemsetAsync(schur_steps(), 0, sizeof(double), c->stream));
    MF_TRY(gst.alloc(ku * ku + 3 * ku + 2));
    MF_TRY(y.alloc(ku));
    return MF_OK;
  }

  // device counter of the Schur CG steps taken while still iterating, over all calls
  double* schur_steps() { return op->ctx->scalars.as<double>() + kScalarsTri + 144; }

  // xp = S~^-1 r_p (r_p fp64): Jacobi-PCG from 0, smax steps; once ||r_k|| <= stol ||r_0|| (or
  // p.S~p <= 0) the remaining steps' kernels return at once and x stays as it is.
  mf_status schur_solve(const double* r) {
    mf_ctx* c = op->ctx;
    double* S = c->scalars.as<double>() + kScalarsTri + 128;
    MF_CUDA_TRY(cudaMemsetAsync(xp.p, 0, sizeof(float) * np, c->stream));
    MF_TRY((convert<double, float>(c, np, r, rp.p)));
    MF_TRY(pointwise_mul<float>(c, np, pinv32.p, rp.p, zp.p));
    MF_CUDA_TRY(cudaMemcpyAsync(pp.p, zp.p, sizeof(float) * np, cudaMemcpyDeviceToDevice, c->stream));
    MF_TRY(cg_init_scalars<float>(c, rp.p, zp.p, np, np, 1, S));
    MF_TRY(dev_cg_tol_init(c, S, stol * stol));
    for (int k = 0; k < smax; ++k) {
      // sp = S~ pp and alpha in one launch
      MF_TRY(stencil125_apply(c, stil.p, stscale.p, pp.p, sp.p, gn[0], gn[1], gn[2], S));
      MF_TRY(cg_update_xr<float>(c, np, np, 1, xp.p, rp.p, pp.p, sp.p, pinv32.p, zp.p, 1, S, true));
      MF_TRY(dev_cg_tol_check(c, S, schur_steps()));
      MF_TRY(cg_update_p<float>(c, np, np, 1, zp.p, pp.p, S, true));
    }
    return MF_OK;
  }

  // z_u = A^-1 rhs_u (z fp64) by ku steps of GMRES from 0, right-preconditioned by D^-1.  rhs
  // is w: a full-length vector whose pressure block is zero, read before the first step only.
  mf_status velocity_solve(double* z) {
    mf_ctx* c = op->ctx;
    double* ds = c->scalars.as<double>() + kScalarsTri;  // 2 (m + 1) + 1 CGS2 coefficients
    const int m = ku;
    double* G = gst.p;
    double* inv = G + 3 * m + 1;
    MF_TRY((dot<float, float>(c, w.p, w.p, nu3, ds)));
    MF_TRY(dev_gmres_begin(c, ds, G, m));
    for (int j = 0; j < m; ++j) {
      float* vj = V.p + j * ldv;
      float* vj1 = V.p + (j + 1) * ldv;
      // V_j = inv * (w or the previous step's unnormalised vector), t = D^-1 V_j, in one pass;
      // only the velocity blocks of the basis are ever read
      MF_TRY(block_jacobi_u32_scaled(c, nu, blk32.p, inv, j == 0 ? w.p : vj, vj, t.p));
      MF_TRY(apply_impl<float>(op, t.p, vj1, 1, n, false));
      MF_TRY(multidot<float>(c, V.p, ldv, j + 1, vj1, nu3, ds));
      MF_TRY(axpy_multidot<float>(c, V.p, ldv, j + 1, ds, -1.0, vj1, nu3, ds + (m + 1)));
      MF_TRY(multiaxpy<float>(c, V.p, ldv, j + 1, ds + (m + 1), -1.0, vj1, nu3, ds + 2 * (m + 1)));
      MF_TRY(dev_gmres_column(c, ds, G, m, j));  // sets inv = 1 / |V_{j+1}|
    }
    MF_TRY(dev_gmres_solve(c, G, m, m, y.p));
    MF_CUDA_TRY(cudaMemsetAsync(w.p, 0, sizeof(float) * nu3, c->stream));
    MF_TRY(multiaxpy<float>(c, V.p, ldv, m, y.p, 1.0, w.p, nu3));
    MF_TRY(block_jacobi_u32(c, nu, blk32.p, w.p, t.p));
    return convert<float, double>(c, nu3, t.p, z);
  }

  // z = P^-1 r through the recorded graph.  The first call runs directly, which also leaves every
  // lazily built table of the operator in place before the capture.
  mf_status apply_replayed(const double* r, double* z) {
    mf_ctx* c = op->ctx;
    if (!use_graph || calls++ == 0) return apply(r, z);
    if (!exec) {
      MF_TRY(rin.alloc(n));
      MF_TRY(zout.alloc(n));
      MF_TRY(capture_graph(c, [&]() { return apply(rin.p, zout.p); }, &exec, &graph_kernels));
    }
    MF_CUDA_TRY(cudaMemcpyAsync(rin.p, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    MF_CUDA_TRY(cudaGraphLaunch(exec, c->stream));
    c->launches += graph_kernels;
    MF_CUDA_TRY(cudaMemcpyAsync(z, zout.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    return MF_OK;
  }

  // z = P^-1 r (fp64 vectors of length n)
  mf_status apply(const double* r, double* z) {
    mf_ctx* c = op->ctx;
    MF_TRY(schur_solve(r + nu3));
    // z_p = -x_p; velocity right-hand side r_u - B^T z_p = r_u + B^T x_p
    MF_TRY((axpby<float, double>(c, np, -1.0, xp.p, 0.0, z + nu3)));
    MF_TRY(oseen_coupling<float>(op, 0, xp.p, ua.p));
    MF_TRY((axpby<double, float>(c, nu3, 1.0, r, 0.0, w.p)));
    MF_TRY((axpby<float, float>(c, nu3, 1.0, ua.p, 1.0, w.p)));
    MF_CUDA_TRY(cudaMemsetAsync(w.p + nu3, 0, sizeof(float) * np, c->stream));
    return velocity_solve(z);
  }
};

// Preconditioner in precision T for nrhs vectors: none, Jacobi, Chebyshev (on D^-1 A), the
// Oseen block Jacobi, or (fp64 only) the Oseen block-triangular preconditioner.
template <typename T> struct Prec {
  mf_op* op = nullptr;
  int kind = MF_PREC_NONE;
  int degree = 4;
  double lmin = 0, lmax = 0;
  Vec<T> dinv, res, d, Ad;
  int nrhs = 1;
  // block-triangular parameters (set before setup) and state
  int tri_velocity_steps = 10, tri_schur_maxit = 30;
  double tri_schur_tol = 0.1;
  bool tri_graph = false;
  std::unique_ptr<OseenBlockTri> tri;

  mf_status setup(mf_op* o, int k, int deg, double ratio, int lanczos_steps, int nr) {
    op = o;
    kind = k;
    degree = deg;
    nrhs = nr;
    const int64_t n = op->n;
    if (kind == MF_PREC_NONE) return MF_OK;
    if (kind == MF_PREC_BLOCK_JACOBI) {
      if (op->p.kind != MF_OP_OSEEN) return fail(MF_EINVAL, "block Jacobi is for the Oseen operator");
      return diag64(op, nullptr);
    }
    if (kind == MF_PREC_BLOCK_TRIANGULAR) {
      if (op->p.kind != MF_OP_OSEEN) return fail(MF_EINVAL, "the block-triangular preconditioner is for the Oseen operator");
      if (!std::is_same<T, double>::value || nrhs != 1)
        return fail(MF_EUNSUPPORTED, "the block-triangular preconditioner runs inside fp64 GMRES");
      tri = std::make_unique<OseenBlockTri>();
      tri->use_graph = tri_graph;
      return tri->setup(op, tri_velocity_steps, tri_schur_maxit, tri_schur_tol);
    }
    if (op->p.kind == MF_OP_OSEEN) return fail(MF_EUNSUPPORTED, "Oseen: use block Jacobi or block triangular");
    double* d64;
    MF_TRY(diag64(op, &d64));
    Vec<double> inv64;
    MF_TRY(inv64.alloc(n));
    // dinv = 1 / diag
    std::vector<double> ones;
    MF_TRY(dinv.alloc(n));
    MF_TRY(reciprocal(d64, inv64.p, n));
    if (sizeof(T) == 8) MF_CUDA_TRY(cudaMemcpyAsync(dinv.p, inv64.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, op->ctx->stream));
    else MF_TRY(convert<double, float>(op->ctx, n, inv64.p, reinterpret_cast<float*>(dinv.p)));
    if (kind == MF_PREC_CHEBYSHEV) {
      MF_TRY(res.alloc(n * nrhs));
      MF_TRY(d.alloc(n * nrhs));
      MF_TRY(Ad.alloc(n * nrhs));
      double lm;
      if (op->lanczos_ready && op->lanczos_steps == lanczos_steps && op->lanczos_prec == op->f32_prec) {
        lm = op->lanczos_lmax;
      } else {
        MF_TRY(lanczos(inv64.p, lanczos_steps, &lm));
        op->lanczos_lmax = lm;
        op->lanczos_steps = lanczos_steps;
        op->lanczos_prec = op->f32_prec;
        op->lanczos_ready = true;
      }
      lmax = 1.1 * lm;
      lmin = lmax / ratio;
    }
    return MF_OK;
  }

  mf_status reciprocal(const double* d, double* out, int64_t n) {
    // out = 1/d via axpby-free path: copy then invert on device with a tiny helper
    MF_CUDA_TRY(cudaMemcpyAsync(out, d, sizeof(double) * n, cudaMemcpyDeviceToDevice, op->ctx->stream));
    return invert_inplace(op->ctx, out, n);
  }

  static mf_status invert_inplace(mf_ctx* c, double* v, int64_t n);

  // lambda_max of D^-1 A (Lanczos on D^-1/2 A D^-1/2).  Only a preconditioner parameter (it is
  // scaled by 1.1), so the operator applies run in fp32 whatever the solve precision; the
  // Lanczos vectors and scalars are fp64.
  mf_status lanczos(const double* inv64, int steps, double* out) {
    mf_ctx* c = op->ctx;
    const int64_t n = op->n;
    Vec<double> s, v, vp, w;
    MF_TRY(s.alloc(n));
    MF_TRY(v.alloc(n));
    MF_TRY(vp.alloc(n));
    MF_TRY(w.alloc(n));
    Vec<float> tv, tw;
    MF_TRY(tv.alloc(n));
    MF_TRY(tw.alloc(n));
    MF_TRY(sqrt_of(c, inv64, s.p, n));
    MF_TRY(fill_splitmix(c, 0x5eed5eedull, v.p, n));
    double* hs = c->host_scalars;
    double* ds = c->scalars.as<double>() + kScalarsLanczos;
    MF_TRY(norm2_sq(c, v.p, n, ds));
    MF_TRY(sync_copy(c, hs, ds, 1));
    MF_TRY(axpby<double, double>(c, n, 1.0 / std::sqrt(hs[0]), v.p, 0.0, v.p));
    MF_CUDA_TRY(cudaMemsetAsync(vp.p, 0, sizeof(double) * n, c->stream));
    std::vector<double> al, be;
    double beta = 0.0;
    for (int k = 0; k < steps; ++k) {
      MF_TRY(dev_scale_mul<float>(c, s.p, v.p, tv.p, n));  // tv = s .* v (fp32)
      MF_TRY(apply_impl<float>(op, tv.p, tw.p, 1, n, false));
      MF_TRY(dev_scale_mul_back<float>(c, s.p, tw.p, w.p, n));  // w = s .* tw
      MF_TRY(axpby<double, double>(c, n, -beta, vp.p, 1.0, w.p));
      MF_TRY(dot<double, double>(c, w.p, v.p, n, ds));
      MF_TRY(sync_copy(c, hs, ds, 1));
      const double alpha = hs[0];
      MF_TRY(axpby<double, double>(c, n, -alpha, v.p, 1.0, w.p));
      MF_TRY(norm2_sq(c, w.p, n, ds));
      MF_TRY(sync_copy(c, hs, ds, 1));
      al.push_back(alpha);
      beta = std::sqrt(hs[0]);
      if (beta == 0.0 || !std::isfinite(beta)) break;
      be.push_back(beta);
      vp.swap_with(v);
      MF_TRY(axpby<double, double>(c, n, 1.0 / beta, w.p, 0.0, v.p));
    }
    if (al.empty()) return fail(MF_EINVAL, "Lanczos failed");
    be.resize(al.size() - 1);
    *out = tridiag_max_eig(al, be);
    return MF_OK;
  }

  static mf_status sqrt_of(mf_ctx* c, const double* in, double* out, int64_t n);
  static mf_status scale_mul(mf_ctx* c, const double* s, const double* v, T* out, int64_t n);
  static mf_status scale_mul_back(mf_ctx* c, const double* s, const T* v, double* out, int64_t n);

  // z = P r for nrhs vectors
  mf_status apply(const T* r, T* z) {
    mf_ctx* c = op->ctx;
    const int64_t n = op->n;
    switch (kind) {
      case MF_PREC_NONE:
        MF_CUDA_TRY(cudaMemcpyAsync(z, r, sizeof(T) * n * nrhs, cudaMemcpyDeviceToDevice, c->stream));
        return MF_OK;
      case MF_PREC_JACOBI:
        for (int k = 0; k < nrhs; ++k) MF_TRY(pointwise_mul<T>(c, n, dinv.p, r + k * n, z + k * n));
        return MF_OK;
      case MF_PREC_BLOCK_JACOBI: {
        const int64_t nu = op->map[0]->n_dofs, np = op->map[1]->n_dofs;
        for (int k = 0; k < nrhs; ++k)
          MF_TRY(block_jacobi<T>(c, nu, np, op->blk64.as<double>(), op->pdiag64.as<double>(), r + k * n, z + k * n));
        return MF_OK;
      }
      case MF_PREC_BLOCK_TRIANGULAR:
        if constexpr (std::is_same<T, double>::value) return tri->apply_replayed(r, z);
        return fail(MF_EUNSUPPORTED, "block-triangular preconditioner in fp32");
      case MF_PREC_CHEBYSHEV: {
        const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
        double rho = 1.0 / sigma;
        MF_TRY(cheb_init<T>(c, n, n, nrhs, r, dinv.p, 1.0 / theta, d.p));
        if (degree < 1) {   // z = d_0
          MF_CUDA_TRY(cudaMemcpyAsync(z, d.p, sizeof(T) * n * nrhs, cudaMemcpyDeviceToDevice, c->stream));
          return MF_OK;
        }
        for (int k = 0; k < degree; ++k) {
          MF_TRY(apply_impl<T>(op, d.p, Ad.p, nrhs, n, false));
          const double rho_new = 1.0 / (2.0 * sigma - rho);
          MF_TRY(cheb_step<T>(c, n, n, nrhs, z, k == 0 ? r : res.p, res.p, Ad.p, d.p, dinv.p, rho_new * rho,
                              2.0 * rho_new / delta, k == 0, k == degree - 1));
          rho = rho_new;
        }
        return MF_OK;
      }
    }
    return fail(MF_EINVAL, "unknown preconditioner");
  }
};

}  // namespace

// small device helpers defined in solver_kernels.cu
mf_status dev_invert(mf_ctx* c, double* v, int64_t n);
mf_status dev_sqrt(mf_ctx* c, const double* in, double* out, int64_t n);
template <typename T> mf_status dev_scale_mul(mf_ctx* c, const double* s, const double* v, T* out, int64_t n);
template <typename T> mf_status dev_scale_mul_back(mf_ctx* c, const double* s, const T* v, double* out, int64_t n);
mf_status dev_scale_rhs(mf_ctx* c, const double* in, float* out, const double* scale, int64_t n, int nrhs);
mf_status dev_add_scaled(mf_ctx* c, const float* d, double* x, const double* scale, int64_t n, int nrhs);

template <typename T> mf_status Prec<T>::invert_inplace(mf_ctx* c, double* v, int64_t n) { return dev_invert(c, v, n); }
template <typename T> mf_status Prec<T>::sqrt_of(mf_ctx* c, const double* in, double* out, int64_t n) {
  return dev_sqrt(c, in, out, n);
}
template <typename T>
mf_status Prec<T>::scale_mul(mf_ctx* c, const double* s, const double* v, T* out, int64_t n) {
  return dev_scale_mul<T>(c, s, v, out, n);
}
template <typename T>
mf_status Prec<T>::scale_mul_back(mf_ctx* c, const double* s, const T* v, double* out, int64_t n) {
  return dev_scale_mul_back<T>(c, s, v, out, n);
}

namespace {

// Batched preconditioned CG in precision T from x = 0: nrhs systems stored n apart.
// Stops each system at ||r_k|| <= tol_r ||b_r|| (recursive residual).
template <typename T> struct CG {
  static constexpr int kGraphSteps = 8;              // CG steps per graph replay on small systems
  static constexpr int64_t kSmallSystem = 1 << 20;   // unknowns (times right-hand sides) of a small system
  mf_op* op;
  Prec<T>* P;
  int nrhs;
  Vec<T> r, z, p, Ap;
  int check_every = 1;
  bool use_graph = false;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_kernels = 0;

  ~CG() {
    if (exec) cudaGraphExecDestroy(exec);
  }

  mf_status setup(mf_op* o, Prec<T>* pr, int nr) {
    op = o;
    P = pr;
    nrhs = nr;
    const int64_t n = op->n * nrhs;
    MF_TRY(r.alloc(n));
    MF_TRY(p.alloc(n));
    MF_TRY(Ap.alloc(n));
    if (P->kind != MF_PREC_NONE) MF_TRY(z.alloc(n));
    return MF_OK;
  }

  // One CG step for every system.  With steps (the on-device stopping test): systems whose active
  // flag is 0 are left untouched, and the test runs at the end of the step.
  mf_status iteration(T* x, double* S, double* steps = nullptr) {
    mf_ctx* c = op->ctx;
    const int64_t n = op->n;
    const bool skip = steps != nullptr;
    MF_TRY(apply_impl<T>(op, p.p, Ap.p, nrhs, n, false));
    MF_TRY(cg_alpha<T>(c, p.p, Ap.p, n, n, nrhs, S));
    if (P->kind == MF_PREC_JACOBI) {
      MF_TRY(cg_update_xr<T>(c, n, n, nrhs, x, r.p, p.p, Ap.p, P->dinv.p, z.p, 1, S, skip));
      MF_TRY(cg_update_p<T>(c, n, n, nrhs, z.p, p.p, S, skip));
    } else if (P->kind == MF_PREC_NONE) {
      MF_TRY(cg_update_xr<T>(c, n, n, nrhs, x, r.p, p.p, Ap.p, nullptr, nullptr, 0, S, skip));
      MF_TRY(cg_update_p<T>(c, n, n, nrhs, r.p, p.p, S, skip));
    } else {
      MF_TRY(cg_update_xr<T>(c, n, n, nrhs, x, r.p, p.p, Ap.p, nullptr, nullptr, 2, S, skip));
      MF_TRY(P->apply(r.p, z.p));
      MF_TRY(cg_rz<T>(c, r.p, z.p, n, n, nrhs, S));
      MF_TRY(cg_update_p<T>(c, n, n, nrhs, z.p, p.p, S, skip));
    }
    if (steps) MF_TRY(dev_cg_tol_check_batched(c, S, steps, nrhs));
    return MF_OK;
  }

  // b, x: nrhs vectors (x overwritten).  rr0[r] = ||b_r||^2 on return; iters, final ||r||/||b||.
  mf_status solve(const T* b, T* x, double tol, int maxit, int* iters, std::vector<double>& relres) {
    mf_ctx* c = op->ctx;
    const int64_t n = op->n;
    double* S = c->scalars.as<double>();
    double* hS = c->host_scalars;
    MF_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * n * nrhs, c->stream));
    MF_CUDA_TRY(cudaMemcpyAsync(r.p, b, sizeof(T) * n * nrhs, cudaMemcpyDeviceToDevice, c->stream));
    T* zz = P->kind == MF_PREC_NONE ? r.p : z.p;
    if (P->kind != MF_PREC_NONE) MF_TRY(P->apply(r.p, z.p));
    MF_CUDA_TRY(cudaMemcpyAsync(p.p, zz, sizeof(T) * n * nrhs, cudaMemcpyDeviceToDevice, c->stream));
    for (int k = 0; k < nrhs; ++k) hS[k * S_NSCAL + S_ACTIVE] = 1.0;
    // active flags first, then r.r and r.z
    for (int k = 0; k < nrhs; ++k)
      MF_CUDA_TRY(cudaMemcpyAsync(S + k * S_NSCAL + S_ACTIVE, hS + k * S_NSCAL + S_ACTIVE, sizeof(double),
                                  cudaMemcpyHostToDevice, c->stream));
    MF_TRY(cg_init_scalars<T>(c, r.p, zz, n, n, nrhs, S));
    MF_TRY(sync_copy(c, hS, S, size_t(nrhs) * S_NSCAL));
    std::vector<double> bb(nrhs), rr(nrhs);
    std::vector<char> done(nrhs, 0);
    relres.assign(nrhs, 0.0);
    int ndone = 0;
    for (int k = 0; k < nrhs; ++k) {
      bb[k] = hS[k * S_NSCAL + S_RR];
      if (bb[k] == 0.0) {
        done[k] = 1;
        ++ndone;
        hS[k * S_NSCAL + S_ACTIVE] = 0.0;
        MF_CUDA_TRY(cudaMemcpyAsync(S + k * S_NSCAL + S_ACTIVE, hS + k * S_NSCAL + S_ACTIVE, sizeof(double),
                                    cudaMemcpyHostToDevice, c->stream));
      }
    }
    int it = 0;
    // With graph replay the stopping test runs on the device after every step, and on small
    // systems (launch-bound steps) a replay holds kGraphSteps steps, so the host waits once per
    // kGraphSteps steps; steps after a system has stopped leave it untouched (their applies still
    // run, which is why large systems replay one step at a time), and the device counts the steps
    // each system took.
    double* steps = use_graph ? c->scalars.as<double>() + kScalarsCGSteps : nullptr;
    const int per = use_graph ? (n * nrhs <= kSmallSystem ? kGraphSteps : 1) : check_every;
    if (steps) {
      MF_CUDA_TRY(cudaMemsetAsync(steps, 0, sizeof(double) * nrhs, c->stream));
      MF_TRY(dev_cg_tol_init_batched(c, S, tol * tol, nrhs));
    }
    if (use_graph && !exec)
      MF_TRY(capture_graph(c, [&]() {
        for (int k = 0; k < per; ++k) MF_TRY(iteration(x, S, steps));
        return MF_OK;
      }, &exec, &graph_kernels));
    std::vector<double> hsteps(nrhs, 0.0);
    while (ndone < nrhs && it < maxit) {
      if (exec && maxit - it >= per) {
        MF_CUDA_TRY(cudaGraphLaunch(exec, c->stream));
        c->launches += graph_kernels;
        it += per;
      } else {
        const int m = std::min(per, maxit - it);
        for (int k = 0; k < m; ++k) MF_TRY(iteration(x, S, steps));
        it += m;
      }
      if (steps) MF_CUDA_TRY(cudaMemcpyAsync(hsteps.data(), steps, sizeof(double) * nrhs, cudaMemcpyDeviceToHost,
                                             c->stream));
      MF_TRY(sync_copy(c, hS, S, size_t(nrhs) * S_NSCAL));
      for (int k = 0; k < nrhs; ++k) {
        if (done[k]) continue;
        const double rk = hS[k * S_NSCAL + S_RR];
        if (!std::isfinite(rk)) return fail(MF_ENOTCONV, "CG breakdown (non-finite residual)");
        if (steps) {   // the device stopped this system: converged, or p.Ap <= 0 (breakdown)
          if (hS[k * S_NSCAL + S_ACTIVE] == 0.0) {
            if (!(rk <= tol * tol * bb[k])) return fail(MF_ENOTCONV, "CG breakdown (p.Ap <= 0)");
            done[k] = 1;
            ++ndone;
          }
        } else if (rk <= tol * tol * bb[k]) {
          done[k] = 1;
          ++ndone;
          hS[k * S_NSCAL + S_ACTIVE] = 0.0;
          MF_CUDA_TRY(cudaMemcpyAsync(S + k * S_NSCAL + S_ACTIVE, hS + k * S_NSCAL + S_ACTIVE, sizeof(double),
                                      cudaMemcpyHostToDevice, c->stream));
        }
      }
    }
    MF_CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < nrhs; ++k) relres[k] = bb[k] > 0 ? std::sqrt(hS[k * S_NSCAL + S_RR] / bb[k]) : 0.0;
    *iters = steps ? int(*std::max_element(hsteps.begin(), hsteps.end())) : it;
    return ndone == nrhs ? MF_OK : MF_ENOTCONV;
  }
};

// true residual ||b - A x|| / ||b|| per RHS in fp64 (r receives b - A x)
mf_status true_residual(mf_op* op, const double* b, const double* x, double* r, int nrhs, std::vector<double>& rel,
                        std::vector<double>* rnorm = nullptr, bool transpose = false) {
  mf_ctx* c = op->ctx;
  const int64_t n = op->n;
  MF_TRY(apply_impl<double>(op, x, r, nrhs, n, transpose));
  rel.assign(nrhs, 0.0);
  if (rnorm) rnorm->assign(nrhs, 0.0);
  double* ds = c->scalars.as<double>() + kScalarsResid;
  for (int k = 0; k < nrhs; ++k) {
    MF_TRY(axpby<double, double>(c, n, 1.0, b + k * n, -1.0, r + k * n));
    MF_TRY(norm2_sq(c, r + k * n, n, ds + 2 * k));
    MF_TRY(norm2_sq(c, b + k * n, n, ds + 2 * k + 1));
  }
  std::vector<double> h(2 * nrhs);
  MF_TRY(sync_copy(c, h.data(), ds, 2 * nrhs));
  for (int k = 0; k < nrhs; ++k) {
    rel[k] = h[2 * k + 1] > 0 ? std::sqrt(h[2 * k] / h[2 * k + 1]) : 0.0;
    if (rnorm) (*rnorm)[k] = std::sqrt(h[2 * k]);
  }
  return MF_OK;
}

// |x|^2 into device out (fp64 sum)
inline mf_status nrm2sq(mf_ctx* c, const double* x, int64_t n, double* out) { return norm2_sq(c, x, n, out); }
inline mf_status nrm2sq(mf_ctx* c, const float* x, int64_t n, double* out) { return dot<float, float>(c, x, x, n, out); }

// Restarted GMRES(m), right preconditioning, classical Gram-Schmidt with one
// reorthogonalisation (CGS2), Givens rotations on the host.  One RHS; T = double (the solver),
// or float (the inner solve of defect correction on a nonsymmetric operator).
template <typename T>
mf_status gmres(mf_op* op, Prec<T>& P, const T* b, T* x, int m, double tol, int maxit, bool transpose, int* iters,
                double* relres) {
  mf_ctx* c = op->ctx;
  const int64_t n = op->n;
  // a preconditioner that changes from call to call (inner Krylov solves) needs the flexible
  // variant (FGMRES): keep Z_j = P^-1 V_j and update x with Z y
  const bool flexible = P.kind == MF_PREC_BLOCK_TRIANGULAR;
  if (flexible && transpose) return fail(MF_EUNSUPPORTED, "block-triangular preconditioner: forward operator only");
  Vec<T> V, t, r, Z;
  const int64_t ldv = basis_stride(n);
  MF_TRY(V.alloc(ldv * (m + 1)));
  MF_TRY(t.alloc(n));
  MF_TRY(r.alloc(n));
  if (flexible) MF_TRY(Z.alloc(ldv * m));
  double* dh = c->scalars.as<double>() + kScalarsGmres;  // room for 2 (m+1) <= 128 values
  if (2 * (m + 1) > 128) return fail(MF_EINVAL, "GMRES restart too long (max 63)");
  double* hh = c->host_scalars + kScalarsGmres;
  MF_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * n, c->stream));
  MF_TRY(nrm2sq(c, b, n, dh));
  MF_TRY(sync_copy(c, hh, dh, 1));
  const double bn = std::sqrt(hh[0]);
  *iters = 0;
  if (bn == 0.0) {
    *relres = 0.0;
    return MF_OK;
  }
  MF_CUDA_TRY(cudaMemcpyAsync(r.p, b, sizeof(T) * n, cudaMemcpyDeviceToDevice, c->stream));
  double beta = bn;
  int it = 0;
  std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  while (it < maxit) {
    MF_TRY((axpby<T, T>(c, n, 1.0 / beta, r.p, 0.0, V.p)));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    bool conv = false;
    for (; j < m && it < maxit; ++j) {
      T* w = V.p + (j + 1) * ldv;
      T* zj = flexible ? Z.p + j * ldv : t.p;
      MF_TRY(P.apply(V.p + j * ldv, zj));
      MF_TRY(apply_impl<T>(op, zj, w, 1, n, transpose));
      MF_TRY(multidot(c, V.p, ldv, j + 1, w, n, dh));
      MF_TRY(axpy_multidot(c, V.p, ldv, j + 1, dh, -1.0, w, n, dh + (m + 1)));
      MF_TRY(multiaxpy(c, V.p, ldv, j + 1, dh + (m + 1), -1.0, w, n, dh + 2 * (m + 1) - 1));  // and |w|^2
      MF_TRY(sync_copy(c, hh, dh, 2 * (m + 1)));
      for (int i = 0; i <= j; ++i) H[i * m + j] = hh[i] + hh[(m + 1) + i];
      double hn = std::sqrt(hh[2 * (m + 1) - 1]);
      H[(j + 1) * m + j] = hn;
      if (hn > 0) MF_TRY((axpby<T, T>(c, n, 1.0 / hn, w, 0.0, w)));
      givens_column(H, m, j, cs, sn, g);
      ++it;
      if (std::fabs(g[j + 1]) <= tol * bn || hn == 0.0) {
        ++j;
        conv = true;
        break;
      }
    }
    // y = H^-1 g (upper triangular), x += M^-1 V y  (flexible: x += Z y)
    back_substitute(H, m, j, g, y);
    for (int i = 0; i < j; ++i) hh[i] = y[i];
    MF_CUDA_TRY(cudaMemcpyAsync(dh, hh, sizeof(double) * j, cudaMemcpyHostToDevice, c->stream));
    if (flexible) {
      MF_TRY(multiaxpy(c, Z.p, ldv, j, dh, 1.0, x, n));
    } else {
      MF_CUDA_TRY(cudaMemsetAsync(r.p, 0, sizeof(T) * n, c->stream));
      MF_TRY(multiaxpy(c, V.p, ldv, j, dh, 1.0, r.p, n));
      MF_TRY(P.apply(r.p, t.p));
      MF_TRY((axpby<T, T>(c, n, 1.0, t.p, 1.0, x)));
    }
    // true residual
    MF_TRY(apply_impl<T>(op, x, r.p, 1, n, transpose));
    MF_TRY((axpby<T, T>(c, n, 1.0, b, -1.0, r.p)));
    MF_TRY(nrm2sq(c, r.p, n, dh));
    MF_TRY(sync_copy(c, hh, dh, 1));
    beta = std::sqrt(hh[0]);
    *relres = beta / bn;
    if (!std::isfinite(beta)) return fail(MF_ENOTCONV, "GMRES breakdown (non-finite residual)");
    if (beta <= tol * bn) break;
    (void)conv;
  }
  *iters = it;
  return *relres <= tol ? MF_OK : MF_ENOTCONV;
}

}  // namespace

mf_status solve_impl(mf_op* op, const mf_solver_params* sp, const double* b, double* x, int nrhs, mf_solve_info* info,
                     bool transpose) {
  auto t0 = clk::now();
  mf_ctx* c = op->ctx;
  const int64_t n = op->n;
  MF_TRY(check_fields(op));
  PoolScope pool_scope(&c->pool);  // the work vectors below come from (and go back to) the context's pool
  // fp64 applies of this solve run on the fp64 pipes or in double-float
  struct Restore {
    mf_op* op;
    int prev;
    ~Restore() { op->f64_prec = prev; }
  } restore{op, op->f64_prec};
  op->f64_prec = (sp->fp64_arith == 1 || (sp->fp64_arith == 2 && op->df64_faster)) ? PREC_DF64 : PREC_F64;
  // fp32 applies of the inner solve in fp32 or packed 16-bit arithmetic
  struct Restore32 {
    mf_op* op;
    ~Restore32() { op->f32_prec = PREC_F32; }
  } restore32{op};
  if (sp->inner_arith == MF_F16 || sp->inner_arith == MF_BF16) {
    if (sp->solver != MF_SOLVER_DEFECT_CORRECTION)
      return fail(MF_EINVAL, "16-bit inner arithmetic belongs to defect correction");
    op->f32_prec = sp->inner_arith == MF_F16 ? PREC_F16 : PREC_BF16;
  } else if (sp->inner_arith == MF_INNER_TENSOR_CORES) {
    if (sp->solver != MF_SOLVER_DEFECT_CORRECTION)
      return fail(MF_EINVAL, "tensor-core inner arithmetic belongs to defect correction");
    if (qk_degree(op) != 3) return fail(MF_EUNSUPPORTED, "tensor-core inner applies: Q3 Helmholtz operators");
    op->f32_prec = PREC_TC;
  } else if (sp->inner_arith != 0 && sp->inner_arith != MF_F32) {
    return fail(MF_EINVAL, "inner_arith must be MF_F32, MF_F16, MF_BF16 or MF_INNER_TENSOR_CORES");
  }
  mf_solve_info inf{};
  mf_status st = MF_OK;
  const double tol = sp->tol > 0 ? sp->tol : 1e-10;
  const int maxit = sp->maxit > 0 ? sp->maxit : 5000;
  const int lsteps = sp->lanczos_steps > 0 ? sp->lanczos_steps : 20;
  const double ratio = sp->cheby_ratio > 0 ? sp->cheby_ratio : 30.0;
  const int deg = sp->cheby_degree > 0 ? sp->cheby_degree : 4;
  std::vector<double> rel;
  if (sp->precond == MF_PREC_BLOCK_TRIANGULAR && sp->solver != MF_SOLVER_GMRES)
    return fail(MF_EINVAL, "the block-triangular preconditioner needs the GMRES solver");
  if (sp->solver == MF_SOLVER_CG) {
    if (transpose && heat_convection(op)) return fail(MF_EINVAL, "CG on a nonsymmetric operator");
    Prec<double> P;
    MF_TRY(P.setup(op, sp->precond, deg, ratio, lsteps, nrhs));
    inf.lambda_max = P.lmax;
    CG<double> cg;
    MF_TRY(cg.setup(op, &P, nrhs));
    cg.use_graph = sp->use_graph != 0;
    int its = 0, total = 0;
    // restart from the true residual if the recursion drifted (at most 3 times)
    Vec<double> rt, e;
    MF_TRY(rt.alloc(n * nrhs));
    MF_TRY(e.alloc(n * nrhs));
    st = cg.solve(b, x, tol, maxit, &its, rel);
    total += its;
    for (int rs = 0; rs < 3 && (st == MF_OK); ++rs) {
      std::vector<double> rn;
      MF_TRY(true_residual(op, b, x, rt.p, nrhs, rel, &rn));
      double worst = *std::max_element(rel.begin(), rel.end());
      if (worst <= tol) break;
      // correction: solve A e = r with the tolerance that brings ||b - A x|| under tol ||b||
      double tol2 = 1.0;
      for (int k = 0; k < nrhs; ++k)
        if (rel[k] > 0) tol2 = std::min(tol2, 0.5 * tol / rel[k]);
      st = cg.solve(rt.p, e.p, tol2, maxit - total, &its, rel);
      total += its;
      MF_TRY(axpby<double, double>(c, n * nrhs, 1.0, e.p, 1.0, x));
    }
    MF_TRY(true_residual(op, b, x, rt.p, nrhs, rel));
    inf.iterations = total;
  } else if (sp->solver == MF_SOLVER_GMRES) {
    Prec<double> P;
    P.tri_velocity_steps = sp->velocity_steps;
    P.tri_schur_maxit = sp->schur_maxit;
    P.tri_schur_tol = sp->schur_tol;
    P.tri_graph = sp->use_graph != 0;
    MF_TRY(P.setup(op, sp->precond, deg, ratio, lsteps, 1));
    inf.lambda_max = P.lmax;
    const int m = sp->restart > 0 ? sp->restart : 50;
    rel.assign(nrhs, 0.0);
    for (int k = 0; k < nrhs; ++k) {
      int its = 0;
      double rr = 0;
      mf_status s2 = gmres(op, P, b + k * n, x + k * n, m, tol, maxit, transpose, &its, &rr);
      if (s2 != MF_OK && s2 != MF_ENOTCONV) return s2;
      if (s2 == MF_ENOTCONV) st = s2;
      inf.iterations += its;
      rel[k] = rr;
    }
    if (P.tri) {
      MF_TRY(sync_copy(c, c->host_scalars + kScalarsTri + 144, P.tri->schur_steps(), 1));
      inf.inner_steps = int(c->host_scalars[kScalarsTri + 144]);
    }
  } else if (sp->solver == MF_SOLVER_DEFECT_CORRECTION) {
    if (sp->inner_dtype != MF_F32) return fail(MF_EUNSUPPORTED, "inner precision must be MF_F32");
    if (op->p.kind == MF_OP_OSEEN) return fail(MF_EUNSUPPORTED, "defect correction: scalar operators");
    // inner fp32 solve: CG on the symmetric operators, GMRES on the convective heat operator (and
    // its transpose)
    const bool nonsym = heat_convection(op);
    if (nonsym && sp->precond == MF_PREC_CHEBYSHEV)
      return fail(MF_EINVAL, "Chebyshev needs a symmetric operator (the convective inner GMRES takes Jacobi)");
    const bool tr = nonsym && transpose;
    const int m = sp->restart > 0 ? sp->restart : 30;
    Prec<float> P;
    MF_TRY(P.setup(op, sp->precond, deg, ratio, lsteps, nonsym ? 1 : nrhs));
    inf.lambda_max = P.lmax;
    CG<float> cg;
    if (!nonsym) {
      MF_TRY(cg.setup(op, &P, nrhs));
      cg.use_graph = sp->use_graph != 0;
      cg.check_every = 1;
    }
    Vec<double> r;
    Vec<float> r32, d32;
    MF_TRY(r.alloc(n * nrhs));
    MF_TRY(r32.alloc(n * nrhs));
    MF_TRY(d32.alloc(n * nrhs));
    double* dscale = c->scalars.as<double>() + kScalarsScale;
    MF_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n * nrhs, c->stream));
    MF_CUDA_TRY(cudaMemcpyAsync(r.p, b, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, c->stream));
    std::vector<double> rn(nrhs), bnorm(nrhs);
    {
      std::vector<double> rl;
      MF_TRY(true_residual(op, b, x, r.p, nrhs, rl, &bnorm, tr));  // x = 0: r = b
    }
    const double itol = sp->inner_tol > 0 ? sp->inner_tol : 1e-4;
    const int imax = sp->inner_maxit > 0 ? sp->inner_maxit : 100;
    int outer = 0;
    rel.assign(nrhs, 1.0);
    while (outer < maxit) {
      if (*std::max_element(rel.begin(), rel.end()) <= tol) break;
      for (int k = 0; k < nrhs; ++k) rn[k] = rel[k] * bnorm[k];
      // inner fp32 solve on the unit-norm residual
      std::vector<double> sc(nrhs);
      for (int k = 0; k < nrhs; ++k) sc[k] = rn[k] > 0 ? 1.0 / rn[k] : 0.0;
      MF_CUDA_TRY(cudaMemcpyAsync(dscale, sc.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, c->stream));
      MF_TRY(dev_scale_rhs(c, r.p, r32.p, dscale, n, nrhs));
      int its = 0;
      if (nonsym) {
        for (int k = 0; k < nrhs; ++k) {
          int ik = 0;
          double rr = 0;
          const mf_status si = gmres<float>(op, P, r32.p + k * n, d32.p + k * n, m, itol, imax, tr, &ik, &rr);
          if (si != MF_OK && si != MF_ENOTCONV) return si;
          its += ik;
        }
      } else {
        std::vector<double> irel;
        const mf_status si = cg.solve(r32.p, d32.p, itol, imax, &its, irel);
        if (si != MF_OK && si != MF_ENOTCONV) return si;
      }
      inf.iterations += its;
      for (int k = 0; k < nrhs; ++k) sc[k] = rn[k];
      MF_CUDA_TRY(cudaMemcpyAsync(dscale, sc.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, c->stream));
      MF_TRY(dev_add_scaled(c, d32.p, x, dscale, n, nrhs));
      ++outer;
      MF_TRY(true_residual(op, b, x, r.p, nrhs, rel, nullptr, tr));
      for (double v : rel)
        if (!std::isfinite(v)) {
          inf.outer_iterations = outer;
          inf.rel_residual = v;
          if (info) *info = inf;
          return fail(MF_ENOTCONV, "defect correction broke down (non-finite residual)");
        }
    }
    inf.outer_iterations = outer;
    if (*std::max_element(rel.begin(), rel.end()) > tol) st = MF_ENOTCONV;
  } else {
    return fail(MF_EINVAL, "unknown solver");
  }
  MF_CUDA_TRY(cudaStreamSynchronize(c->stream));
  inf.rel_residual = rel.empty() ? 0.0 : *std::max_element(rel.begin(), rel.end());
  inf.seconds = std::chrono::duration<double>(clk::now() - t0).count();
  if (info) *info = inf;
  if (st == MF_ENOTCONV) return fail(MF_ENOTCONV, "solver did not reach the tolerance within maxit");
  return st;
}

}  // namespace mf

using namespace mf;

extern "C" {

mf_status mf_solve(mf_op* op, const mf_solver_params* sp, const double* b, double* x, int nrhs, mf_solve_info* info) {
  try {
    if (!op || !sp || !b || !x) return fail(MF_EINVAL, "NULL argument");
    if (nrhs < 1 || nrhs > 64) return fail(MF_EINVAL, "nrhs must be in 1..64");
    const mf_status st = solve_impl(op, sp, b, x, nrhs, info, false);
    // the solve has synchronised: a tensor-core apply inside it that timed out is reported here
    const mf_status tc = tc_take_error();
    return tc != MF_OK ? tc : st;
  } catch (...) {
    return fail(MF_ENOMEM, "exception in mf_solve");
  }
}

mf_status mf_laser_load(mf_op* op, const mf_laser* lz, double* dst, double* dF) {
  if (!op || !lz || !dst) return fail(MF_EINVAL, "NULL argument");
  if (op->p.kind != MF_OP_HEAT) return fail(MF_EINVAL, "laser load belongs to heat operators");
  if (!(lz->radius > 0) || !(lz->power > 0)) return fail(MF_EINVAL, "laser power and radius must be > 0");
  const double p[5] = {lz->power, lz->radius, lz->x0, lz->y0, lz->absorptivity};
  return launch_laser(op->ctx, op->map[0], p, dst, dF);
}

mf_status mf_heat_step_gradient(mf_op* op, const mf_laser* lz, const mf_solver_params* sp, const double* theta_prev,
                                const double* theta_target, double box_half, double box_depth, double* J,
                                double* dJ_dlaser, double* dJ_dkq, double* theta_out, double* lambda_out) {
  try {
    if (!op || !lz || !sp || !theta_prev || !theta_target || !J || !dJ_dlaser) return fail(MF_EINVAL, "NULL argument");
    if (op->p.kind != MF_OP_HEAT) return fail(MF_EINVAL, "heat operators only");
    if (dJ_dkq && !op->kq_user) return fail(MF_EINVAL, "dJ/dk_q needs MF_FIELD_K_QPOINT");
    if (op->rhocp_user || op->betaq_user) return fail(MF_EUNSUPPORTED, "heat-step gradient with Gauss-point rho_cp / beta");
    mf_ctx* c = op->ctx;
    const mf_dofmap* m = op->map[0];
    if (!m->uniform) return fail(MF_EUNSUPPORTED, "heat-step gradient on octree maps");
    const int64_t n = op->n;
    DevBuf buf;
    MF_TRY(buf.alloc(sizeof(double) * n * 9));
    double* f = buf.as<double>();
    double* dF = f + n;           // 4 n
    double* bvec = dF + 4 * n;
    double* th = bvec + n;
    double* e = th + n;
    double* lam = e + n;
    // b = rho_cp/dt M theta_prev + f_laser (Dirichlet rows 0)
    MF_TRY(mf_laser_load(op, lz, f, dF));
    ScalarArgs<double> a = scalar_args<double>(op, theta_prev, bvec, 1, n);
    a.mass = op->p.rhocp / op->p.dt;
    MF_CUDA_TRY(cudaMemsetAsync(bvec, 0, sizeof(double) * n, c->stream));
    MF_TRY(launch_scalar_apply(c, m, K_MASS, 1, false, false, PREC_F64, &a));
    MF_TRY(axpby<double, double>(c, n, 1.0, f, 1.0, bvec));
    MF_TRY(zero_list<double>(c, bvec, m->d_dir_list.as<int32_t>(), int64_t(m->dirichlet_list.size())));
    mf_solve_info inf;
    mf_status st = solve_impl(op, sp, bvec, th, 1, &inf, false);
    if (st != MF_OK) return st;
    // J = 1/2 e^T M_box e, dJ/dtheta = M_box e
    MF_TRY(axpby<double, double>(c, n, 1.0, th, 0.0, e));
    MF_TRY(axpby<double, double>(c, n, -1.0, theta_target, 1.0, e));
    ScalarArgs<double> mb = scalar_args<double>(op, e, f, 1, n);
    mb.mass = 1.0;
    mb.use_box = 1;
    mb.box_half = box_half;
    mb.box_zmin = m->mesh->hi[2] - box_depth;
    for (int d = 0; d < 3; ++d) mb.lo[d] = m->mesh->lo[d];
    MF_CUDA_TRY(cudaMemsetAsync(f, 0, sizeof(double) * n, c->stream));
    MF_TRY(launch_scalar_apply(c, m, K_MASS, 1, false, false, PREC_F64, &mb));
    double* ds = c->scalars.as<double>() + kScalarsHeat;
    MF_TRY(dot<double, double>(c, e, f, n, ds));
    MF_TRY(zero_list<double>(c, f, m->d_dir_list.as<int32_t>(), int64_t(m->dirichlet_list.size())));
    // adjoint: A^T lambda = dJ/dtheta
    st = solve_impl(op, sp, f, lam, 1, &inf, true);
    if (st != MF_OK) return st;
    for (int p = 0; p < 4; ++p) MF_TRY(dot<double, double>(c, dF + p * n, lam, n, ds + 1 + p));
    double hs[5];
    MF_TRY(sync_copy(c, hs, ds, 5));
    *J = 0.5 * hs[0];
    for (int p = 0; p < 4; ++p) dJ_dlaser[p] = hs[1 + p];
    if (dJ_dkq) MF_TRY(launch_grad_kq(c, m, lam, th, dJ_dkq));
    if (theta_out) MF_CUDA_TRY(cudaMemcpyAsync(theta_out, th, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    if (lambda_out) MF_CUDA_TRY(cudaMemcpyAsync(lambda_out, lam, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    MF_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return MF_OK;
  } catch (...) {
    return fail(MF_ENOMEM, "exception in mf_heat_step_gradient");
  }
}

}  // extern "C"

namespace {

// The configuration that decides which variant is fastest: operator kind and degree, mesh type
// and sizes, the optional fields, the melt-pool flags and the device's SM count.
std::string tune_key(const mf_op* op) {
  const mf_dofmap* m = op->map[0];
  char buf[320];
  std::snprintf(buf, sizeof buf, "kind=%d deg=%d %s dofs=%lld cells=%lld con=%lld beta=%d kq=%d rhocp=%d betaq=%d "
                "mode=%d flags=%d sms=%d", op->p.kind, m->degree, m->uniform ? "uniform" : "octree",
                (long long)op->n, (long long)op->ncells, (long long)(m->con_rowptr.empty() ? 0 : m->con_rowptr.size() - 1), op->beta ? 1 : 0,
                op->kq_user ? 1 : 0, op->rhocp_user ? 1 : 0, op->betaq_user ? 1 : 0, op->p.coef_mode,
                op->p.oseen_flags, op->ctx->sm_count);
  return buf;
}

std::string tune_choice(const mf_op* op) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "\"mode64\": %d, \"mode32\": %d, \"block\": %d, \"persistent_blocks\": %d, "
                "\"df64_faster\": %d, \"oseen_qouter64\": %d, \"qk_f32_tc\": %d, \"q2_line64\": %d, "
                "\"q2_line32\": %d", op->mode64, op->mode32, op->block, op->persistent_blocks, op->df64_faster ? 1 : 0,
                op->oseen_qouter64, op->qk_f32_tc, op->q2_line64, op->q2_line32);
  return buf;
}

bool read_int(const std::string& line, const char* name, int* out) {
  const std::string tag = std::string("\"") + name + "\": ";
  const size_t at = line.find(tag);
  return at != std::string::npos && std::sscanf(line.c_str() + at + tag.size(), "%d", out) == 1;
}

// The last record of cache_path whose key matches this operator, applied to it; false if none.
bool apply_cached_choice(mf_op* op, const char* cache_path) {
  FILE* fp = std::fopen(cache_path, "r");
  if (!fp) return false;
  const std::string want = "\"key\": \"" + tune_key(op) + "\"";
  std::string hit, line;
  char chunk[1024];
  while (std::fgets(chunk, sizeof chunk, fp)) {
    line += chunk;
    if (line.empty() || line.back() != '\n') continue;
    if (line.find(want) != std::string::npos) hit = line;
    line.clear();
  }
  std::fclose(fp);
  int v[7];
  const char* names[7] = {"mode64", "mode32", "block", "persistent_blocks", "df64_faster", "oseen_qouter64", "qk_f32_tc"};
  if (hit.empty()) return false;
  for (int i = 0; i < 7; ++i)
    if (!read_int(hit, names[i], &v[i])) return false;
  if ((v[0] | v[1]) & ~1 || (v[2] != 64 && v[2] != 128) || v[3] < 0 || v[3] > 64) return false;
  op->mode64 = v[0];
  op->mode32 = v[1];
  op->block = v[2];
  op->persistent_blocks = v[3];
  op->df64_faster = v[4] != 0;
  op->oseen_qouter64 = v[5] != 0;
  op->qk_f32_tc = v[6] != 0;
  // records written before the line kernel was a choice leave it off
  int l64 = 0, l32 = 0;
  read_int(hit, "q2_line64", &l64);
  read_int(hit, "q2_line32", &l32);
  op->q2_line64 = l64 != 0;
  op->q2_line32 = l32 != 0;
  op->tune_record = hit.substr(0, hit.size() - 1);
  return true;
}

mf_status autotune_measure(mf_op* op) {
  try {
    MF_TRY(check_fields(op));
    mf_ctx* c = op->ctx;
    const int64_t n = op->n;
    if (qk_degree(op) == 4) {  // Q4: one kernel variant per precision, nothing to choose
      op->tune_record = "{\"variants\": \"helmholtz_q4: one\"}";
      return MF_OK;
    }
    if (qk_degree(op) == 3) {
      // fp32 applies: the sum-factorised CUDA-core kernel or the dense tensor-core kernel
      op->qk_f32_tc = 0;
      DevBuf s, d;
      MF_TRY(s.alloc(sizeof(float) * n));
      MF_TRY(d.alloc(sizeof(float) * n));
      MF_CUDA_TRY(cudaMemsetAsync(s.p, 0, sizeof(float) * n, c->stream));
      cudaEvent_t a0, a1;
      cudaEventCreate(&a0);
      cudaEventCreate(&a1);
      double ms[2] = {1e30, 1e30};
      for (int v = 0; v < 2; ++v) {
        for (int rep = 0; rep < 4; ++rep) {
          cudaEventRecord(a0, c->stream);
          MF_TRY(apply_impl<float>(op, s.as<float>(), d.as<float>(), 1, n, false, v ? PREC_TC : PREC_F32));
          cudaEventRecord(a1, c->stream);
          MF_CUDA_TRY(cudaEventSynchronize(a1));
          float t;
          cudaEventElapsedTime(&t, a0, a1);
          if (rep > 0) ms[v] = std::min(ms[v], double(t));
        }
      }
      cudaEventDestroy(a0);
      cudaEventDestroy(a1);
      op->qk_f32_tc = ms[1] < ms[0] ? 1 : 0;
      char buf[256];
      std::snprintf(buf, sizeof buf, "{\"kind\": %d, \"n\": %lld, \"q3_f32_cuda_core_ms\": %.6g, \"q3_f32_tensor_core_ms\": %.6g}",
                    op->p.kind, (long long)n, ms[0], ms[1]);
      op->tune_record = buf;
      return MF_OK;
    }
    if (op->p.kind == MF_OP_OSEEN) {
      // fp64 kernel variant: component loop outside (fewer registers) or Gauss-point loop outside
      // (fewer fp64 operations, spills)
      MF_TRY(ensure_tables(op));
      DevBuf s, d;
      MF_TRY(s.alloc(sizeof(double) * n));
      MF_TRY(d.alloc(sizeof(double) * n));
      MF_TRY(fill_splitmix(c, 7, s.as<double>(), n));
      cudaEvent_t a0, a1;
      cudaEventCreate(&a0);
      cudaEventCreate(&a1);
      double ms[2] = {1e30, 1e30};
      for (int v = 0; v < 2; ++v) {
        op->oseen_qouter64 = v;
        for (int rep = 0; rep < 4; ++rep) {
          cudaEventRecord(a0, c->stream);
          MF_TRY(apply_impl<double>(op, s.as<double>(), d.as<double>(), 1, n, false, PREC_F64));
          cudaEventRecord(a1, c->stream);
          MF_CUDA_TRY(cudaEventSynchronize(a1));
          float t;
          cudaEventElapsedTime(&t, a0, a1);
          if (rep > 0) ms[v] = std::min(ms[v], double(t));
        }
      }
      op->oseen_qouter64 = ms[1] < ms[0] ? 1 : 0;
      // fp64-accurate arithmetic: the fp64 pipes or double-float pairs
      double df_ms = 1e30;
      {
        for (int rep = 0; rep < 4; ++rep) {
          cudaEventRecord(a0, c->stream);
          MF_TRY(apply_impl<double>(op, s.as<double>(), d.as<double>(), 1, n, false, PREC_DF64));
          cudaEventRecord(a1, c->stream);
          MF_CUDA_TRY(cudaEventSynchronize(a1));
          float t;
          cudaEventElapsedTime(&t, a0, a1);
          if (rep > 0) df_ms = std::min(df_ms, double(t));
        }
      }
      op->df64_faster = df_ms < std::min(ms[0], ms[1]);
      cudaEventDestroy(a0);
      cudaEventDestroy(a1);
      char buf[256];
      std::snprintf(buf, sizeof buf, "{\"kind\": %d, \"n\": %lld, \"component_outer_ms\": %.6g, \"qpoint_outer_ms\": %.6g, "
                    "\"df64_ms\": %.6g}", op->p.kind, (long long)n, ms[0], ms[1], df_ms);
      op->tune_record = buf;
      return MF_OK;
    }
    MF_TRY(ensure_tables(op));
    DevBuf src, dst;
    MF_TRY(src.alloc(sizeof(double) * n));
    MF_TRY(dst.alloc(sizeof(double) * n));
    MF_TRY(fill_splitmix(c, 7, src.as<double>(), n));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool forced = heat_tabulated(op);
    DevBuf s32, d32;
    MF_TRY(s32.alloc(sizeof(float) * n));
    MF_TRY(d32.alloc(sizeof(float) * n));
    MF_TRY(convert<double, float>(c, n, src.as<double>(), s32.as<float>()));
    // the launch shape of octree operators is timed on a batch of eight right-hand sides (their
    // batched reinitialisation; one and eight right-hand sides prefer different shapes)
    const int shape_rhs = op->map[0]->uniform ? 1 : 8;
    DevBuf sb, db;
    if (shape_rhs > 1) {
      MF_TRY(sb.alloc(sizeof(float) * n * shape_rhs));
      MF_TRY(db.alloc(sizeof(float) * n * shape_rhs));
      for (int r = 0; r < shape_rhs; ++r)
        MF_CUDA_TRY(cudaMemcpyAsync(sb.as<float>() + r * n, s32.as<float>(), sizeof(float) * n,
                                    cudaMemcpyDeviceToDevice, c->stream));
    }
    // median-free best-of-5 event timing of one apply variant
    auto time_variant = [&](int prec, double* out_ms, int nr = 1) -> mf_status {
      double best = 1e30;
      for (int rep = 0; rep < 6; ++rep) {
        cudaEventRecord(e0, c->stream);
        if (prec == PREC_F32 && nr > 1)
          MF_TRY(apply_impl<float>(op, sb.as<float>(), db.as<float>(), nr, n, false, PREC_F32));
        else if (prec == PREC_F32) MF_TRY(apply_impl<float>(op, s32.as<float>(), d32.as<float>(), 1, n, false, PREC_F32));
        else MF_TRY(apply_impl<double>(op, src.as<double>(), dst.as<double>(), 1, n, false, prec));
        cudaEventRecord(e1, c->stream);
        MF_CUDA_TRY(cudaEventSynchronize(e1));
        float ms;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, double(ms));
      }
      *out_ms = best;
      return MF_OK;
    };
    // 1) coefficient evaluation: in the kernel from nodal fields, or tabulated per Gauss point
    double mode_ms[2][2] = {{1e30, 1e30}, {1e30, 1e30}};
    for (int pi = 0; pi < 2; ++pi)
      for (int mode = 0; mode < 2; ++mode) {
        if (forced && mode == 0) continue;
        if (pi == 1 && mode == 0 && op->p.kind == MF_OP_REINIT) continue;  // fp64-evaluated normals only
        (pi == 0 ? op->mode64 : op->mode32) = mode;
        MF_TRY(time_variant(pi == 0 ? PREC_F64 : PREC_F32, &mode_ms[pi][mode]));
      }
    op->mode64 = mode_ms[0][0] < mode_ms[0][1] ? 0 : 1;
    op->mode32 = (op->p.kind != MF_OP_REINIT && mode_ms[1][0] < mode_ms[1][1]) ? 0 : 1;
    // 2) launch shape on the fp32 apply: cells per block (octree) and persistent grids
    const int shapes[5][2] = {{128, 0}, {64, 0}, {128, 2}, {128, 4}, {64, 8}};
    double shape_ms[5];
    int best_shape = 0;
    for (int si = 0; si < 5; ++si) {
      shape_ms[si] = 1e30;
      if (op->map[0]->uniform && shapes[si][0] != 128) continue;
      op->block = shapes[si][0];
      op->persistent_blocks = shapes[si][1];
      MF_TRY(time_variant(PREC_F32, &shape_ms[si], shape_rhs));
      if (shape_ms[si] < shape_ms[best_shape]) best_shape = si;
    }
    op->block = shapes[best_shape][0];
    op->persistent_blocks = shapes[best_shape][1];
    // 3) fp64-accurate arithmetic: fp64 pipes vs double-float on the fp32 pipes; on uniform Q2
    //    Helmholtz / heat operators also the line-per-thread kernel in fp64 and fp32 (small meshes)
    double f64_ms, df_ms, line64_ms = -1.0, line32_ms = -1.0;
    op->q2_line64 = op->q2_line32 = 0;
    MF_TRY(time_variant(PREC_F64, &f64_ms));
    MF_TRY(time_variant(PREC_DF64, &df_ms));
    const int kind = scalar_kind(op);
    if (op->map[0]->uniform && op->map[0]->degree == 2 && (kind == K_HELM || kind == K_HEAT) && !heat_convection(op) &&
        !op->rhocp_user) {
      op->q2_line64 = 1;
      MF_TRY(time_variant(PREC_F64, &line64_ms));
      op->q2_line64 = 0;
      op->q2_line32 = 1;
      MF_TRY(time_variant(PREC_F32, &line32_ms));
      op->q2_line64 = line64_ms < f64_ms ? 1 : 0;
      op->q2_line32 = line32_ms < shape_ms[best_shape] ? 1 : 0;
    }
    op->df64_faster = df_ms < (op->q2_line64 ? line64_ms : f64_ms);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    char buf[512];
    std::snprintf(buf, sizeof buf,
                  "{\"kind\": %d, \"n\": %lld, \"f64_inkernel_ms\": %.6g, \"f64_tabulated_ms\": %.6g, "
                  "\"f32_inkernel_ms\": %.6g, \"f32_tabulated_ms\": %.6g, \"block\": %d, \"persistent_blocks\": %d, "
                  "\"f32_shape_ms\": %.6g, \"f64_ms\": %.6g, \"df64_ms\": %.6g, \"f64_line_ms\": %.6g, "
                  "\"f32_line_ms\": %.6g}",
                  op->p.kind, (long long)n, mode_ms[0][0], mode_ms[0][1], mode_ms[1][0], mode_ms[1][1], op->block,
                  op->persistent_blocks, shape_ms[best_shape], f64_ms, df_ms, line64_ms, line32_ms);
    op->tune_record = buf;
    return MF_OK;
  } catch (...) {
    return fail(MF_ENOMEM, "exception in mf_autotune");
  }
}

}  // namespace

extern "C" {

mf_status mf_autotune(mf_op* op, const char* cache_path) {
  try {
    if (!op) return fail(MF_EINVAL, "NULL argument");
    MF_TRY(check_fields(op));
    if (cache_path && apply_cached_choice(op, cache_path)) return MF_OK;
    MF_TRY(autotune_measure(op));
    const std::string rec = "{\"key\": \"" + tune_key(op) + "\", " + tune_choice(op) + ", \"timings\": " +
                            op->tune_record + "}";
    op->tune_record = rec;
    if (cache_path) {
      FILE* fp = std::fopen(cache_path, "a");
      if (fp) {
        std::fprintf(fp, "%s\n", rec.c_str());
        std::fclose(fp);
      }
    }
    return MF_OK;
  } catch (...) {
    return fail(MF_ENOMEM, "exception in mf_autotune");
  }
}

}  // extern "C"
