// C ABI of libmfgb: contexts, meshes, DoF maps, operators, apply / transpose / diagonal.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "ops.h"
#include "vec.cuh"

namespace mf {

static thread_local std::string g_error;

// The device this process is bound to (-1: none yet).  Constant tables, the tensor-core operand
// image and the host-mapped error flags are uploaded once per process, so every context must
// live on the same device.
static std::atomic<int> g_bound_device{-1};

void set_error(const std::string& msg) { g_error = msg; }
mf_status fail(mf_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

// every live context's pool, so that a failed allocation anywhere can free the kept blocks
static std::mutex g_pools_mu;
static std::vector<BlockPool*> g_pools;
thread_local BlockPool* tl_pool = nullptr;

BlockPool::BlockPool() {
  std::lock_guard<std::mutex> lk(g_pools_mu);
  g_pools.push_back(this);
}
BlockPool::~BlockPool() {
  trim();
  std::lock_guard<std::mutex> lk(g_pools_mu);
  g_pools.erase(std::remove(g_pools.begin(), g_pools.end(), this), g_pools.end());
}
mf_status BlockPool::get(size_t n, void** out) {
  const size_t r = rounded(n);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = keep.find(r);
    if (it != keep.end()) {
      *out = it->second;
      keep.erase(it);
      kept -= r;
      return MF_OK;
    }
  }
  if (cudaMalloc(out, r) != cudaSuccess) {
    cudaGetLastError();
    trim_block_pools();
    if (cudaMalloc(out, r) != cudaSuccess) {
      cudaGetLastError();
      *out = nullptr;
      return fail(MF_ENOMEM, "cudaMalloc of " + std::to_string(r) + " bytes failed");
    }
  }
  return MF_OK;
}
void BlockPool::put(void* blk, size_t n) {
  const size_t r = rounded(n);
  std::lock_guard<std::mutex> lk(mu);
  keep.emplace(r, blk);
  kept += r;
}
// cudaFree waits for the device, so work still queued on a block finishes before it is freed
void BlockPool::trim() {
  std::lock_guard<std::mutex> lk(mu);
  for (auto& kv : keep) cudaFree(kv.second);
  keep.clear();
  kept = 0;
}
void trim_block_pools() {
  std::lock_guard<std::mutex> lk(g_pools_mu);
  for (BlockPool* p : g_pools) p->trim();
}

}  // namespace mf

using namespace mf;

#define MF_GUARD_BEGIN try {
#define MF_GUARD_END                                                         \
  }                                                                          \
  catch (const std::bad_alloc&) { return fail(MF_ENOMEM, "host allocation failed"); } \
  catch (...) { return fail(MF_EINVAL, "internal exception"); }

extern "C" {

const char* mf_last_error(void) { return mf::g_error.c_str(); }

mf_status mf_context_create(int device, void* cuda_stream, mf_ctx** out) {
  MF_GUARD_BEGIN
  if (!out) return fail(MF_EINVAL, "out is NULL");
  *out = nullptr;
  if (device < 0) return fail(MF_EINVAL, "device index out of range");
  {
    const int bound = g_bound_device.load();
    if (bound >= 0 && bound != device)
      return fail(MF_EUNSUPPORTED, "this process is bound to CUDA device " + std::to_string(bound) +
                                       ": the library serves one device per process");
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    int expect = -1;   // nothing can run without a device; the first request still fixes the binding
    g_bound_device.compare_exchange_strong(expect, device);
    return fail(MF_ECUDA, "no CUDA device visible");
  }
  if (device >= ndev) return fail(MF_EINVAL, "device index out of range");
  {
    int expect = -1;
    if (!g_bound_device.compare_exchange_strong(expect, device) && expect != device)
      return fail(MF_EUNSUPPORTED, "this process is bound to CUDA device " + std::to_string(expect) +
                                       ": the library serves one device per process");
  }
  MF_CUDA_TRY(cudaSetDevice(device));
  auto* c = new mf_ctx();
  c->device = device;
  if (cuda_stream) c->stream = static_cast<cudaStream_t>(cuda_stream);
  else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return fail(MF_ECUDA, "cudaStreamCreate failed");
    }
    c->own_stream = true;
  }
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  mf_status st = c->scratch.alloc(kScratchDoubles * sizeof(double));
  if (st == MF_OK) st = c->scalars.alloc(sizeof(double) * kScalarsTotal);
  if (st == MF_OK) st = c->counters.alloc(sizeof(unsigned) * 64);
  // zeroed on the context's stream (a non-blocking stream is not ordered after the legacy one)
  if (st == MF_OK && (cudaMemsetAsync(c->counters.p, 0, sizeof(unsigned) * 64, c->stream) != cudaSuccess ||
                      cudaStreamSynchronize(c->stream) != cudaSuccess))
    st = fail(MF_ECUDA, "zeroing the reduction counters failed");
  if (st == MF_OK && cudaMallocHost(&c->host_scalars, sizeof(double) * kScalarsTotal) != cudaSuccess)
    st = fail(MF_ENOMEM, "pinned host allocation failed");
  if (st != MF_OK) {
    mf_context_destroy(c);
    return st;
  }
  *out = c;
  return MF_OK;
  MF_GUARD_END
}

void mf_context_destroy(mf_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->host_scalars) cudaFreeHost(c->host_scalars);
  c->scratch.release();
  c->scalars.release();
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  if (c->fence) cudaEventDestroy(c->fence);
  delete c;
}

mf_status mf_context_set_stream(mf_ctx* c, void* s) {
  if (!c) return fail(MF_EINVAL, "ctx is NULL");
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  c->own_stream = false;
  c->stream = static_cast<cudaStream_t>(s);
  return MF_OK;
}

int64_t mf_context_launch_count(const mf_ctx* c) { return c ? c->launches : 0; }

mf_status mf_mesh_uniform(mf_ctx* c, const int n[3], const double lo[3], const double hi[3], mf_mesh** out) {
  MF_GUARD_BEGIN
  if (!n || !lo || !hi || !out) return fail(MF_EINVAL, "NULL argument");
  *out = nullptr;
  double h[3];
  for (int d = 0; d < 3; ++d) {
    if (n[d] <= 0 || n[d] > 4096) return fail(MF_EINVAL, "cells per axis must be in 1..4096");
    if (!(hi[d] > lo[d])) return fail(MF_EINVAL, "empty box");
    h[d] = (hi[d] - lo[d]) / n[d];
  }
  if (std::fabs(h[1] - h[0]) > 1e-12 * h[0] || std::fabs(h[2] - h[0]) > 1e-12 * h[0])
    return fail(MF_EINVAL, "uniform cells must be cubes");
  auto* m = new mf_mesh();
  m->ctx = c;
  for (int d = 0; d < 3; ++d) {
    m->n[d] = n[d];
    m->lo[d] = lo[d];
    m->hi[d] = hi[d];
  }
  m->h0 = h[0];
  *out = m;
  return MF_OK;
  MF_GUARD_END
}

mf_status mf_mesh_octree(mf_ctx* c, int base, int levels, const double lo[3], const double hi[3], const int32_t* leaves,
                         int64_t nleaves, mf_mesh** out) {
  MF_GUARD_BEGIN
  if (!lo || !hi || !out || (!leaves && nleaves)) return fail(MF_EINVAL, "NULL argument");
  *out = nullptr;
  if (base <= 0 || levels < 0 || levels > 10) return fail(MF_EINVAL, "base must be > 0 and levels in 0..10");
  const int64_t nf = int64_t(base) << levels;
  if (nf > 1024) return fail(MF_EINVAL, "finest level finer than 1024 cells per axis");
  for (int d = 0; d < 3; ++d)
    if (!(hi[d] > lo[d]) || std::fabs((hi[d] - lo[d]) - (hi[0] - lo[0])) > 1e-12 * (hi[0] - lo[0]))
      return fail(MF_EINVAL, "octree domain must be a cube");
  if (nleaves <= 0) return fail(MF_EINVAL, "no leaves");
  // tiling and 2:1 balance on the finest grid
  std::vector<int8_t> lev(size_t(nf * nf * nf), -1);
  for (int64_t t = 0; t < nleaves; ++t) {
    const int32_t* lf = leaves + 4 * t;
    const int l = lf[0];
    if (l < 0 || l > levels) return fail(MF_EINVAL, "leaf level out of range");
    const int64_t nl = int64_t(base) << l, s = int64_t(1) << (levels - l);
    for (int d = 1; d < 4; ++d)
      if (lf[d] < 0 || lf[d] >= nl) return fail(MF_EINVAL, "leaf coordinate out of range");
    for (int64_t z = lf[3] * s; z < (lf[3] + 1) * s; ++z)
      for (int64_t y = lf[2] * s; y < (lf[2] + 1) * s; ++y)
        for (int64_t x = lf[1] * s; x < (lf[1] + 1) * s; ++x) {
          int8_t& v = lev[size_t((z * nf + y) * nf + x)];
          if (v != -1) return fail(MF_EINVAL, "leaves overlap");
          v = int8_t(l);
        }
  }
  for (size_t i = 0; i < lev.size(); ++i)
    if (lev[i] < 0) return fail(MF_EINVAL, "leaves do not cover the domain");
  for (int64_t z = 0; z < nf; ++z)
    for (int64_t y = 0; y < nf; ++y)
      for (int64_t x = 0; x < nf; ++x) {
        const int a = lev[size_t((z * nf + y) * nf + x)];
        for (int dz = 0; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              if (dz == 0 && (dy < 0 || (dy == 0 && dx <= 0))) continue;
              const int64_t X = x + dx, Y = y + dy, Z = z + dz;
              if (X < 0 || Y < 0 || X >= nf || Y >= nf || Z >= nf) continue;
              const int b = lev[size_t((Z * nf + Y) * nf + X)];
              if (a - b > 1 || b - a > 1) return fail(MF_EINVAL, "leaves are not 2:1 balanced");
            }
      }
  lev.clear();
  lev.shrink_to_fit();
  // Morton order of the finest-level anchors
  std::vector<std::pair<uint64_t, int64_t>> key(nleaves);
  auto spread = [](uint64_t v) {
    uint64_t r = 0;
    for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1ull) << (3 * b);
    return r;
  };
  for (int64_t t = 0; t < nleaves; ++t) {
    const int32_t* lf = leaves + 4 * t;
    const int sh = levels - lf[0];
    key[t] = {spread(uint64_t(lf[1]) << sh) | (spread(uint64_t(lf[2]) << sh) << 1) | (spread(uint64_t(lf[3]) << sh) << 2), t};
  }
  std::sort(key.begin(), key.end());
  auto* m = new mf_mesh();
  m->ctx = c;
  m->octree = true;
  m->base = base;
  m->levels = levels;
  for (int d = 0; d < 3; ++d) {
    m->n[d] = base;
    m->lo[d] = lo[d];
    m->hi[d] = hi[d];
  }
  m->h0 = (hi[0] - lo[0]) / base;
  m->leaves.resize(4 * nleaves);
  for (int64_t t = 0; t < nleaves; ++t) std::memcpy(&m->leaves[4 * t], leaves + 4 * key[t].second, 4 * sizeof(int32_t));
  *out = m;
  return MF_OK;
  MF_GUARD_END
}

void mf_mesh_destroy(mf_mesh* m) { delete m; }

mf_status mf_dofmap_create(mf_mesh* mesh, int degree, uint32_t faces, mf_dofmap** out) {
  MF_GUARD_BEGIN
  if (!mesh || !out) return fail(MF_EINVAL, "NULL argument");
  *out = nullptr;
  if (degree < 1 || degree > 4) return fail(MF_EUNSUPPORTED, "degree must be 1 to 4");
  if (degree > 2 && mesh->octree) return fail(MF_EUNSUPPORTED, "degrees 3 and 4 on uniform meshes only");
  if (faces >> 6) return fail(MF_EINVAL, "dirichlet_faces has bits above 5");
  auto* m = new mf_dofmap();
  m->mesh = mesh;
  m->degree = degree;
  m->nb = (degree + 1) * (degree + 1) * (degree + 1);
  m->dirichlet_faces = faces;
  mf_status st = mesh->octree ? build_octree_dofmap(m) : build_uniform_dofmap(m);
  if (st == MF_OK && mesh->ctx) st = upload_dofmap(m);  // host-only maps (NULL context) stay on the host
  if (st != MF_OK) {
    delete m;
    return st;
  }
  *out = m;
  return MF_OK;
  MF_GUARD_END
}

void mf_dofmap_destroy(mf_dofmap* m) { delete m; }

mf_status mf_dofmap_query(const mf_dofmap* m, int64_t* nd, int64_t* nc, int64_t* ncon, int64_t* nent) {
  if (!m) return fail(MF_EINVAL, "map is NULL");
  if (nd) *nd = m->n_dofs;
  if (nc) *nc = m->n_cells;
  if (ncon) *ncon = m->uniform ? 0 : int64_t(m->con_rowptr.size()) - 1;
  if (nent) *nent = m->uniform ? 0 : int64_t(m->con_cols.size());
  return MF_OK;
}

mf_status mf_dofmap_export(const mf_dofmap* m, int32_t* cell_map, int64_t* con_rowptr, int32_t* con_cols, double* con_w,
                           double* coords, uint8_t* dirichlet) {
  MF_GUARD_BEGIN
  if (!m) return fail(MF_EINVAL, "map is NULL");
  const int k = m->degree, nb = m->nb;
  const int64_t Rx = m->R[0] + 1, Ry = m->R[1] + 1;
  if (cell_map) {
    if (m->uniform) {
      const int nx = m->mesh->n[0], ny = m->mesh->n[1], nz = m->mesh->n[2];
      int64_t c = 0;
      for (int cz = 0; cz < nz; ++cz)
        for (int cy = 0; cy < ny; ++cy)
          for (int cx = 0; cx < nx; ++cx, ++c)
            for (int i = 0, l = 0; i <= k; ++i)
              for (int j = 0; j <= k; ++j)
                for (int a = 0; a <= k; ++a, ++l) {
                  const int64_t x = int64_t(k) * cx + a, y = int64_t(k) * cy + j, z = int64_t(k) * cz + i;
                  cell_map[c * nb + l] = int32_t(x + Rx * (y + Ry * z));
                }
    } else {
      std::memcpy(cell_map, m->cell_map.data(), m->cell_map.size() * sizeof(int32_t));
    }
  }
  if (!m->uniform) {
    if (con_rowptr) std::memcpy(con_rowptr, m->con_rowptr.data(), m->con_rowptr.size() * sizeof(int64_t));
    if (con_cols) std::memcpy(con_cols, m->con_cols.data(), m->con_cols.size() * sizeof(int32_t));
    if (con_w) std::memcpy(con_w, m->con_w.data(), m->con_w.size() * sizeof(double));
  } else if (con_rowptr) {
    con_rowptr[0] = 0;
  }
  if (coords) {
    const mf_mesh* me = m->mesh;
    double span[3], lo[3];
    for (int d = 0; d < 3; ++d) {
      span[d] = (me->hi[d] - me->lo[d]) / double(m->R[d]);
      lo[d] = me->lo[d];
    }
    // degrees 3 and 4: lattice coordinate k c + a sits at the Gauss-Lobatto point xi_a of cell c
    double xi[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (k == 3) {
      const double r = 1.0 / std::sqrt(5.0);
      xi[1] = 0.5 * (1.0 - r);
      xi[2] = 0.5 * (1.0 + r);
      xi[3] = 1.0;
    } else if (k == 4) {
      const double r = std::sqrt(3.0 / 7.0);
      xi[1] = 0.5 * (1.0 - r);
      xi[2] = 0.5;
      xi[3] = 0.5 * (1.0 + r);
      xi[4] = 1.0;
    }
    for (int64_t d = 0; d < m->n_dofs; ++d) {
      const int64_t key = m->uniform ? d : m->free_keys[d];
      const int64_t p[3] = {key % Rx, (key / Rx) % Ry, key / (Rx * Ry)};
      for (int a = 0; a < 3; ++a) {
        if (k <= 2) {
          coords[3 * d + a] = lo[a] + double(p[a]) * span[a];
        } else {
          const int64_t n = m->R[a] / k, c = std::min<int64_t>(p[a] / k, n - 1);
          coords[3 * d + a] = lo[a] + (double(c) + xi[p[a] - k * c]) * ((me->hi[a] - me->lo[a]) / double(n));
        }
      }
    }
  }
  if (dirichlet) std::memcpy(dirichlet, m->dirichlet.data(), m->dirichlet.size());
  return MF_OK;
  MF_GUARD_END
}

// ------------------------------------------------------------------------ operators

static bool is_q2(const mf_dofmap* m) { return m && m->degree == 2; }

mf_status mf_operator_create(mf_ctx* c, const mf_op_params* p, const mf_dofmap* const* maps, int nmaps, mf_op** out) {
  MF_GUARD_BEGIN
  if (!c || !p || !maps || !out) return fail(MF_EINVAL, "NULL argument");
  *out = nullptr;
  for (int i = 0; i < nmaps; ++i)
    if (!maps[i] || maps[i]->mesh->ctx != c) return fail(MF_EINVAL, "maps must be built on this context's meshes");
  if (p->kind < 0 || p->kind > MF_OP_REINIT) return fail(MF_EINVAL, "unknown operator kind");
  if (p->kind == MF_OP_OSEEN) {
    if (nmaps != 2 || !is_q2(maps[0]) || !maps[1] || maps[1]->degree != 1 || maps[0]->mesh != maps[1]->mesh ||
        !maps[0]->uniform)
      return fail(MF_EINVAL, "Oseen needs a Q2 and a Q1 map on the same uniform mesh");
    if (maps[1]->dirichlet_faces) return fail(MF_EUNSUPPORTED, "Dirichlet pressure DoFs");
  } else if (nmaps == 1 && maps[0] && maps[0]->degree >= 3) {
    if (p->kind != MF_OP_HELMHOLTZ) return fail(MF_EUNSUPPORTED, "degrees 3 and 4: the Helmholtz operator only");
    if (maps[0]->dirichlet_faces) return fail(MF_EUNSUPPORTED, "degrees 3 and 4: no Dirichlet faces");
  } else {
    if (nmaps != 1 || !is_q2(maps[0])) return fail(MF_EINVAL, "scalar operators need one Q2 map");
  }
  if (p->oseen_flags) {
    if (p->kind != MF_OP_OSEEN) return fail(MF_EINVAL, "oseen_flags apply to the Oseen operator");
    if (p->oseen_flags & ~(MF_OSEEN_THREE_PHASE | MF_OSEEN_DARCY | MF_OSEEN_TRACE_CORRECTION))
      return fail(MF_EINVAL, "unknown oseen_flags bit");
    if ((p->oseen_flags & (MF_OSEEN_THREE_PHASE | MF_OSEEN_DARCY)) && !(p->t_liquidus > p->t_solidus))
      return fail(MF_EINVAL, "the solid fraction needs t_liquidus > t_solidus");
    if ((p->oseen_flags & MF_OSEEN_THREE_PHASE) && !(p->rho_s > 0 && p->mu_s >= 0))
      return fail(MF_EINVAL, "three-phase coefficients need rho_s > 0 and mu_s >= 0");
    if ((p->oseen_flags & MF_OSEEN_DARCY) && !(p->darcy_b > 0 && p->darcy_c >= 0))
      return fail(MF_EINVAL, "Darcy damping needs b > 0 and C >= 0");
  }
  if (p->heaviside != 0 && p->heaviside != 1) return fail(MF_EINVAL, "heaviside must be 0 or 1");
  if (p->heaviside == 1 && !(p->eps > 0)) return fail(MF_EINVAL, "sine Heaviside needs eps > 0");
  auto* op = new mf_op();
  op->ctx = c;
  op->p = *p;
  op->nmaps = nmaps;
  for (int i = 0; i < nmaps; ++i) op->map[i] = maps[i];
  op->n = maps[0]->n_dofs * (p->kind == MF_OP_OSEEN ? 3 : 1) + (nmaps == 2 ? maps[1]->n_dofs : 0);
  op->ncells = maps[0]->n_cells;
  op->mode64 = p->kind == MF_OP_OSEEN ? 1 : (p->coef_mode == MF_COEF_INKERNEL ? 0 : 1);
  // reinit: fp32 applies always read the normal evaluated in fp64 (far from the interface phi_h is
  // flat to within fp32 rounding, and a normal computed there in fp32 points anywhere)
  op->mode32 = p->kind == MF_OP_REINIT ? 1 : op->mode64;
  *out = op;
  return MF_OK;
  MF_GUARD_END
}

void mf_operator_destroy(mf_op* op) { delete op; }

mf_status mf_operator_size(const mf_op* op, int64_t* n) {
  if (!op || !n) return fail(MF_EINVAL, "NULL argument");
  *n = op->n;
  return MF_OK;
}

const char* mf_operator_variant(const mf_op* op) { return op ? op->variant.c_str() : ""; }

mf_status mf_operator_set_variant(mf_op* op, const char* name, int value) {
  MF_GUARD_BEGIN
  if (!op || !name) return fail(MF_EINVAL, "NULL argument");
  if (value != 0 && value != 1) return fail(MF_EINVAL, "variant values are 0 or 1");
  if (std::string(name) == "q2_line") {
    op->q2_line64 = op->q2_line32 = value;
    return MF_OK;
  }
  return fail(MF_EINVAL, std::string("unknown variant name: ") + name);
  MF_GUARD_END
}

mf_status mf_operator_set_field(mf_op* op, int field, const void* ptr, int dtype, int64_t n) {
  MF_GUARD_BEGIN
  if (!op || !ptr) return fail(MF_EINVAL, "NULL argument");
  if (dtype != MF_F64) return fail(MF_EUNSUPPORTED, "fields are fp64");
  const int64_t nd = op->map[0]->n_dofs;
  switch (field) {
    case MF_FIELD_PHI:
      if (n != nd) return fail(MF_EINVAL, "PHI must have n_dofs values");
      op->phi = static_cast<const double*>(ptr);
      break;
    case MF_FIELD_T_PREV:
      if (n != nd) return fail(MF_EINVAL, "T_PREV must have n_dofs values");
      op->tprev = static_cast<const double*>(ptr);
      break;
    case MF_FIELD_BETA:
      if (n != 3 * nd) return fail(MF_EINVAL, "BETA must have 3 * n_dofs values");
      op->beta = static_cast<const double*>(ptr);
      break;
    case MF_FIELD_K_QPOINT:
      if (n != op->ncells * 27) return fail(MF_EINVAL, "K_QPOINT must have n_cells * 27 values");
      op->kq_user = static_cast<const double*>(ptr);
      break;
    case MF_FIELD_RHOCP_QPOINT:
      if (op->p.kind != MF_OP_HEAT) return fail(MF_EINVAL, "RHOCP_QPOINT belongs to heat operators");
      if (n != op->ncells * 27) return fail(MF_EINVAL, "RHOCP_QPOINT must have n_cells * 27 values");
      op->rhocp_user = static_cast<const double*>(ptr);
      break;
    case MF_FIELD_BETA_QPOINT:
      if (op->p.kind != MF_OP_HEAT) return fail(MF_EINVAL, "BETA_QPOINT belongs to heat operators");
      if (n != op->ncells * 81) return fail(MF_EINVAL, "BETA_QPOINT must have n_cells * 27 * 3 values");
      op->betaq_user = static_cast<const double*>(ptr);
      break;
    default:
      return fail(MF_EINVAL, "unknown field");
  }
  op->tables_ready = false;
  op->tc_ready = false;
  op->df_ready = false;
  op->diag_ready = false;
  op->lanczos_ready = false;
  op->h16_cnorm = 0.0f;
  // float copy of the in-kernel nodal field
  const double* f = op->p.kind == MF_OP_HEAT ? op->tprev : op->phi;
  if (f && (field == MF_FIELD_PHI || field == MF_FIELD_T_PREV)) {
    MF_TRY(op->field32.alloc(sizeof(float) * nd));
    MF_TRY(convert<double, float>(op->ctx, nd, f, op->field32.as<float>()));
  }
  return MF_OK;
  MF_GUARD_END
}

}  // extern "C"

namespace mf {

int scalar_kind(const mf_op* op) {
  switch (op->p.kind) {
    case MF_OP_HELMHOLTZ: return K_HELM;
    case MF_OP_HEAT: return K_HEAT;
    case MF_OP_REINIT: return K_REINIT;
  }
  return -1;
}

double value_coef(const mf_op* op) {
  switch (op->p.kind) {
    case MF_OP_HELMHOLTZ: return op->p.mass_coef;
    case MF_OP_HEAT: return op->p.rhocp / op->p.dt;
    case MF_OP_REINIT: return 1.0 / op->p.dtau;
  }
  return 0.0;
}

// heat operator with a convection term (nodal or per Gauss point)
bool heat_convection(const mf_op* op) { return op->p.kind == MF_OP_HEAT && (op->beta || op->betaq_user); }

// heat operator whose coefficients must come from the Gauss-point tables
bool heat_tabulated(const mf_op* op) {
  return op->p.kind == MF_OP_HEAT && (op->beta || op->kq_user || op->rhocp_user || op->betaq_user);
}

mf_status apply_tc(mf_op* op, const float* src, float* dst, int nrhs, int64_t ld);

// 3 or 4 for the Q3/Q4 Helmholtz operators, else 0
int qk_degree(const mf_op* op) { return op->map[0] && op->map[0]->degree >= 3 ? op->map[0]->degree : 0; }

mf_status check_fields(const mf_op* op) {
  switch (op->p.kind) {
    case MF_OP_HELMHOLTZ:
      if (!op->phi) return fail(MF_EINVAL, "Helmholtz needs MF_FIELD_PHI");
      break;
    case MF_OP_HEAT:
      if (!op->tprev && !op->kq_user) return fail(MF_EINVAL, "heat needs MF_FIELD_T_PREV or MF_FIELD_K_QPOINT");
      break;
    case MF_OP_OSEEN:
      if (!op->phi || !op->beta) return fail(MF_EINVAL, "Oseen needs MF_FIELD_PHI and MF_FIELD_BETA");
      if ((op->p.oseen_flags & (MF_OSEEN_THREE_PHASE | MF_OSEEN_DARCY)) && !op->tprev)
        return fail(MF_EINVAL, "three-phase / Darcy terms need MF_FIELD_T_PREV (nodal temperature)");
      break;
    case MF_OP_REINIT:
      if (!op->phi) return fail(MF_EINVAL, "reinit needs MF_FIELD_PHI");
      break;
  }
  return MF_OK;
}

mf_status ensure_tables(mf_op* op) {
  if (op->tables_ready) return MF_OK;
  MF_TRY(check_fields(op));
  const int64_t nc = op->ncells;
  const mf_op_params& p = op->p;
  if (p.kind == MF_OP_OSEEN) {
    MF_TRY(op->rho64.alloc(sizeof(double) * 27 * nc));
    MF_TRY(op->rho32.alloc(sizeof(float) * 27 * nc));
    MF_TRY(op->mu64.alloc(sizeof(double) * 27 * nc));
    MF_TRY(op->mu32.alloc(sizeof(float) * 27 * nc));
    MF_TRY(op->qvec64.alloc(sizeof(double) * 81 * nc));
    MF_TRY(op->qvec32.alloc(sizeof(float) * 81 * nc));
    MF_TRY(launch_oseen_qtables(op->ctx, op->map[0], op->phi, op->beta, p.rho_l, p.rho_g, p.mu_l, p.mu_g, p.heaviside,
                                p.eps, op->rho64.as<double>(), op->rho32.as<float>(), op->mu64.as<double>(),
                                op->mu32.as<float>(), op->qvec64.as<double>(), op->qvec32.as<float>()));
    if (p.oseen_flags) {
      MF_TRY(op->kd64.alloc(sizeof(double) * 27 * nc));
      MF_TRY(op->kd32.alloc(sizeof(float) * 27 * nc));
      MF_TRY(op->nrm64.alloc(sizeof(double) * 81 * nc));
      MF_TRY(op->nrm32.alloc(sizeof(float) * 81 * nc));
      MF_TRY(launch_oseen_ext_tables(op->ctx, op->map[0], p, op->phi, op->tprev, op->rho64.as<double>(),
                                     op->rho32.as<float>(), op->mu64.as<double>(), op->mu32.as<float>(),
                                     op->kd64.as<double>(), op->kd32.as<float>(), op->nrm64.as<double>(),
                                     op->nrm32.as<float>()));
    }
    for (mf::DevBuf* b : {&op->cm64, &op->cv64}) MF_TRY(b->alloc(sizeof(double) * 27 * nc));
    for (mf::DevBuf* b : {&op->cm32, &op->cv32}) MF_TRY(b->alloc(sizeof(float) * 27 * nc));
    MF_TRY(op->cb64.alloc(sizeof(double) * 81 * nc));
    MF_TRY(op->cb32.alloc(sizeof(float) * 81 * nc));
    MF_TRY(launch_oseen_fold(op->ctx, op->map[0], p.sigma, op->rho64.as<double>(), op->mu64.as<double>(),
                             p.oseen_flags ? op->kd64.as<double>() : nullptr, op->qvec64.as<double>(),
                             op->cm64.as<double>(), op->cm32.as<float>(), op->cb64.as<double>(), op->cb32.as<float>(),
                             op->cv64.as<double>(), op->cv32.as<float>()));
  } else if (qk_degree(op)) {
    const int64_t P3 = int64_t(qk_degree(op) + 1) * (qk_degree(op) + 1) * (qk_degree(op) + 1);
    MF_TRY(op->qcoef64.alloc(sizeof(double) * P3 * nc));
    MF_TRY(op->qcoef32.alloc(sizeof(float) * P3 * nc));
    MF_TRY(launch_qk_coef(op->ctx, op->map[0], op->phi, p.a_liquid, p.a_gas, p.heaviside, p.eps,
                          op->qcoef64.as<double>(), op->qcoef32.as<float>()));
  } else {
    const int kind = scalar_kind(op);
    MF_TRY(op->qcoef64.alloc(sizeof(double) * 27 * nc));
    MF_TRY(op->qcoef32.alloc(sizeof(float) * 27 * nc));
    const bool vec = (kind == K_REINIT) || heat_convection(op);
    if (vec) {
      MF_TRY(op->qvec64.alloc(sizeof(double) * 81 * nc));
      MF_TRY(op->qvec32.alloc(sizeof(float) * 81 * nc));
    }
    const bool qm = kind == K_HEAT && op->rhocp_user;
    if (qm) {
      MF_TRY(op->qmass64.alloc(sizeof(double) * 27 * nc));
      MF_TRY(op->qmass32.alloc(sizeof(float) * 27 * nc));
    }
    const double* field = kind == K_HEAT ? op->tprev : op->phi;
    MF_TRY(launch_scalar_qtables(op->ctx, op->map[0], kind, field, op->kq_user, kind == K_HEAT ? op->beta : nullptr,
                                 p.k0, 0.5 * p.k0 / (p.t_boil > 0 ? p.t_boil : 1.0), p.a_liquid, p.a_gas, p.heaviside,
                                 p.eps, p.rhocp, op->qcoef64.as<double>(), op->qcoef32.as<float>(),
                                 vec ? op->qvec64.as<double>() : nullptr, vec ? op->qvec32.as<float>() : nullptr,
                                 kind == K_HEAT ? op->rhocp_user : nullptr, kind == K_HEAT ? op->betaq_user : nullptr,
                                 p.dt, qm ? op->qmass64.as<double>() : nullptr, qm ? op->qmass32.as<float>() : nullptr));
  }
  op->tables_ready = true;
  return MF_OK;
}

template <typename T> ScalarArgs<T> scalar_args(const mf_op* op, const T* src, T* dst, int nrhs, int64_t ld) {
  ScalarArgs<T> a{};
  const bool f32 = sizeof(T) == 4;
  a.src = src;
  a.dst = dst;
  a.nrhs = nrhs;
  a.ld = ld;
  a.field = f32 ? reinterpret_cast<const T*>(op->field32.as<float>())
                : reinterpret_cast<const T*>(op->p.kind == MF_OP_HEAT ? op->tprev : op->phi);
  a.qcoef = f32 ? reinterpret_cast<const T*>(op->qcoef32.as<float>()) : reinterpret_cast<const T*>(op->qcoef64.as<double>());
  a.qvec = f32 ? reinterpret_cast<const T*>(op->qvec32.as<float>()) : reinterpret_cast<const T*>(op->qvec64.as<double>());
  a.qmass = !(op->p.kind == MF_OP_HEAT && op->rhocp_user) ? nullptr
            : f32 ? reinterpret_cast<const T*>(op->qmass32.as<float>())
                  : reinterpret_cast<const T*>(op->qmass64.as<double>());
  a.ncp = op->ncells;
  a.mass = T(value_coef(op));
  a.a_l = T(op->p.a_liquid);
  a.a_g = T(op->p.a_gas);
  a.k0 = T(op->p.k0);
  a.k_slope = T(0.5 * op->p.k0 / (op->p.t_boil > 0 ? op->p.t_boil : 1.0));
  a.eps = T(op->p.eps);
  a.heaviside = op->p.heaviside;
  a.block = op->block;
  a.persistent_blocks = op->persistent_blocks;
  return a;
}
template ScalarArgs<double> scalar_args<double>(const mf_op*, const double*, double*, int, int64_t);
template ScalarArgs<float> scalar_args<float>(const mf_op*, const float*, float*, int, int64_t);

template <typename T> OseenArgs<T> oseen_args(const mf_op* op, const T* src, T* dst) {
  OseenArgs<T> a{};
  const bool f32 = sizeof(T) == 4;
  a.src = src;
  a.dst = dst;
  a.nu = op->map[0]->n_dofs;
  a.np = op->map[1]->n_dofs;
  a.rho = f32 ? reinterpret_cast<const T*>(op->rho32.as<float>()) : reinterpret_cast<const T*>(op->rho64.as<double>());
  a.mu = f32 ? reinterpret_cast<const T*>(op->mu32.as<float>()) : reinterpret_cast<const T*>(op->mu64.as<double>());
  a.beta = f32 ? reinterpret_cast<const T*>(op->qvec32.as<float>()) : reinterpret_cast<const T*>(op->qvec64.as<double>());
  a.sigma = T(op->p.sigma);
  a.ext = op->p.oseen_flags ? 1 : 0;
  a.qouter = a.ext ? 1 : op->oseen_qouter64;  // the extensions exist in the Gauss-point-outer kernel
  a.kd = a.ext ? (f32 ? reinterpret_cast<const T*>(op->kd32.as<float>()) : reinterpret_cast<const T*>(op->kd64.as<double>()))
               : nullptr;
  a.nrm = a.ext ? (f32 ? reinterpret_cast<const T*>(op->nrm32.as<float>()) : reinterpret_cast<const T*>(op->nrm64.as<double>()))
                : nullptr;
  auto pick = [&](const mf::DevBuf& b64, const mf::DevBuf& b32) {
    return f32 ? reinterpret_cast<const T*>(b32.as<float>()) : reinterpret_cast<const T*>(b64.as<double>());
  };
  a.cm = pick(op->cm64, op->cm32);
  a.cb = pick(op->cb64, op->cb32);
  a.cv = pick(op->cv64, op->cv32);
  return a;
}
template OseenArgs<double> oseen_args<double>(const mf_op*, const double*, double*);

// the block-triangular preconditioner's fp32 block inverses (entry-major, 9 nu) and inverse pressure
// scaling (n_p), from the fp32 Gauss-point tables
mf_status oseen_blocks32(mf_op* op, float* blk, float* pinv) {
  if (op->p.kind != MF_OP_OSEEN) return fail(MF_EINVAL, "nodal blocks exist for the Oseen operator only");
  MF_TRY(check_fields(op));
  MF_TRY(ensure_tables(op));
  return launch_oseen_blockdiag32(op->ctx, op->map[0], op->map[1], oseen_args<float>(op, nullptr, nullptr), blk, pinv);
}

// Packed 16-bit arithmetic (two right-hand sides per thread) on fp32 vectors: scalar operators
// with tabulated coefficients and no convection.
mf_status apply_h16(mf_op* op, const float* src, float* dst, int nrhs, int64_t ld, bool transpose, int prec) {
  mf_ctx* c = op->ctx;
  MF_TRY(check_fields(op));
  if (op->p.kind == MF_OP_OSEEN) return fail(MF_EUNSUPPORTED, "16-bit arithmetic for the Oseen operator");
  const int kind = scalar_kind(op);
  if (heat_convection(op)) return fail(MF_EUNSUPPORTED, "16-bit arithmetic with convection");
  if (kind == K_HEAT && op->rhocp_user) return fail(MF_EUNSUPPORTED, "16-bit arithmetic with rho_cp per Gauss point");
  (void)transpose;  // the supported operators are symmetric
  MF_TRY(ensure_tables(op));
  if (ld == op->n) MF_CUDA_TRY(cudaMemsetAsync(dst, 0, sizeof(float) * op->n * nrhs, c->stream));
  else
    for (int r = 0; r < nrhs; ++r) MF_CUDA_TRY(cudaMemsetAsync(dst + r * ld, 0, sizeof(float) * op->n, c->stream));
  ScalarArgs<float> a = scalar_args<float>(op, src, dst, nrhs, ld);
  // power of two near sqrt(n): unit-norm vectors get O(1) entries (inside fp16's range)
  const float scale = std::ldexp(1.0f, int(std::lround(0.5 * std::log2(double(std::max<int64_t>(op->n, 1))))));
  if (op->h16_cnorm <= 0.0f) {
    // every coefficient the packed kernel multiplies: the value term mass h^2 (largest h), eps
    // (reinit) and the Gauss-point table (a or k)
    double big = std::fabs(double(a.mass)) * op->map[0]->mesh->h0 * op->map[0]->mesh->h0;
    if (kind == K_REINIT) {
      big = std::max(big, std::fabs(double(a.eps)));
    } else {
      float qmax = 0.0f;
      MF_TRY(abs_max_f32(c, op->qcoef32.as<float>(), int64_t(27) * op->ncells, &qmax));
      big = std::max(big, double(qmax));
    }
    op->h16_cnorm = std::ldexp(1.0f, std::max(0, int(std::ceil(std::log2(std::max(big, 1e-30))))));
  }
  MF_TRY(launch_scalar_apply_h16(c, op->map[0], kind, prec, a, scale, op->h16_cnorm));
  MF_TRY(launch_dirichlet_copy(c, op->map[0], src, dst, nrhs, ld, 0, true));
  op->variant = std::string(kind == K_HELM ? "helmholtz" : kind == K_HEAT ? "heat" : "reinit") +
                (op->map[0]->uniform ? "/uniform" : "/octree") + (prec == PREC_F16 ? "/f16x2" : "/bf16x2") +
                "/tabulated/pairs-of-rhs";
  return MF_OK;
}

// dst = A src (or A^T src), nrhs vectors ld apart, precision T.
// prec: PREC_F64 / PREC_DF64 for fp64 vectors (-1: the operator's fp64 arithmetic), PREC_F32 for fp32.
template <typename T>
mf_status apply_impl(mf_op* op, const T* src, T* dst, int nrhs, int64_t ld, bool transpose, int prec) {
  const bool f32 = sizeof(T) == 4;
  if (f32) prec = (prec == PREC_F16 || prec == PREC_BF16 || prec == PREC_F32 || prec == PREC_TC) ? prec : op->f32_prec;
  else if (prec != PREC_F64 && prec != PREC_DF64) prec = op->f64_prec;
  if (qk_degree(op)) {  // Q3 / Q4 Helmholtz: symmetric, fp64 or fp32 arithmetic (Q3 fp32: or the tensor cores)
    if constexpr (sizeof(T) == 4) {
      if (prec == PREC_TC || (prec == PREC_F32 && op->qk_f32_tc))
        return apply_tc(op, src, dst, nrhs, ld);
    }
    if (prec != PREC_F64 && prec != PREC_F32) return fail(MF_EUNSUPPORTED, "degrees 3 and 4: fp64 or fp32 applies");
    MF_TRY(check_fields(op));
    MF_TRY(ensure_tables(op));
    const T* coef = f32 ? reinterpret_cast<const T*>(op->qcoef32.as<float>())
                        : reinterpret_cast<const T*>(op->qcoef64.as<double>());
    for (int r = 0; r < nrhs; ++r) {
      MF_CUDA_TRY(cudaMemsetAsync(dst + r * ld, 0, sizeof(T) * op->n, op->ctx->stream));
      MF_TRY(launch_helmholtz_qk<T>(op->ctx, op->map[0], src + r * ld, dst + r * ld, coef, op->p.mass_coef));
    }
    op->variant = std::string("helmholtz_q") + std::to_string(qk_degree(op)) + "/uniform" + (f32 ? "/f32" : "/f64") +
                  "/tabulated/line-per-thread";
    return MF_OK;
  }
  if constexpr (sizeof(T) == 4) {
    if (prec == PREC_F16 || prec == PREC_BF16) return apply_h16(op, src, dst, nrhs, ld, transpose, prec);
  }
  const bool df = prec == PREC_DF64;
  mf_ctx* c = op->ctx;
  MF_TRY(check_fields(op));
  const int mode = df ? 1 : (f32 ? op->mode32 : op->mode64);
  const bool needs_tables = op->p.kind == MF_OP_OSEEN || mode == 1 || heat_tabulated(op);
  if (needs_tables) MF_TRY(ensure_tables(op));
  if (ld == op->n) MF_CUDA_TRY(cudaMemsetAsync(dst, 0, sizeof(T) * op->n * nrhs, c->stream));
  else
    for (int r = 0; r < nrhs; ++r) MF_CUDA_TRY(cudaMemsetAsync(dst + r * ld, 0, sizeof(T) * op->n, c->stream));
  const char* pname = f32 ? "/f32" : (df ? "/df64" : "/f64");
  if (op->p.kind == MF_OP_OSEEN) {
    if (transpose) return fail(MF_EUNSUPPORTED, "transpose of the Oseen operator");
    const int64_t nu = op->map[0]->n_dofs;
    if constexpr (sizeof(T) == 8) {
      if (df) {
        // double-float: one warp per velocity component over a brick of 32 cells (the Darcy term is
        // folded into cm; the trace correction reads the interface normal pairs)
        const int64_t nc = op->ncells;
        const bool ext = op->p.oseen_flags != 0;
        if (!op->df_ready) {
          MF_TRY(op->cm_df.alloc(sizeof(float) * 54 * nc));
          MF_TRY(op->cv_df.alloc(sizeof(float) * 54 * nc));
          MF_TRY(op->cb_df.alloc(sizeof(float) * 162 * nc));
          MF_TRY(launch_split_pairs(c, op->cm64.as<double>(), 27 * nc, op->cm_df.as<float>(), op->cm_df.as<float>() + 27 * nc));
          MF_TRY(launch_split_pairs(c, op->cv64.as<double>(), 27 * nc, op->cv_df.as<float>(), op->cv_df.as<float>() + 27 * nc));
          MF_TRY(launch_split_pairs(c, op->cb64.as<double>(), 81 * nc, op->cb_df.as<float>(), op->cb_df.as<float>() + 81 * nc));
          if (ext) {
            MF_TRY(op->nrm_df.alloc(sizeof(float) * 162 * nc));
            MF_TRY(launch_split_pairs(c, op->nrm64.as<double>(), 81 * nc, op->nrm_df.as<float>(),
                                      op->nrm_df.as<float>() + 81 * nc));
          }
          op->df_ready = true;
        }
        for (int r = 0; r < nrhs; ++r) {
          MF_TRY(launch_oseen_df_uniform(c, op->map[0], reinterpret_cast<const double*>(src + r * ld),
                                         reinterpret_cast<double*>(dst + r * ld), op->cm_df.as<float>(),
                                         op->cv_df.as<float>(), op->cb_df.as<float>(),
                                         ext ? op->nrm_df.as<float>() : nullptr));
          MF_TRY(launch_dirichlet_copy(c, op->map[0], src + r * ld, dst + r * ld, 3, nu, 0, false));
        }
        op->variant = std::string("oseen_q2q1/df64/tabulated/warp-per-component") + (ext ? "/meltpool" : "");
        return MF_OK;
      }
    }
    for (int r = 0; r < nrhs; ++r) {
      OseenArgs<T> a = oseen_args<T>(op, src + r * ld, dst + r * ld);
      MF_TRY(launch_oseen_apply(c, op->map[0], prec, &a));
      // the three velocity components' Dirichlet rows, as three vectors nu apart
      MF_TRY(launch_dirichlet_copy(c, op->map[0], src + r * ld, dst + r * ld, 3, nu, 0, f32));
    }
    op->variant = std::string("oseen_q2q1") + pname + "/tabulated" +
                  ((f32 || op->oseen_qouter64 || op->p.oseen_flags) ? "/qpoint-outer" : "/component-outer") +
                  (op->p.oseen_flags ? "/meltpool" : "");
    return MF_OK;
  }
  const int kind = scalar_kind(op);
  const bool beta = heat_convection(op);
  if (transpose && !(kind == K_HEAT && beta)) {
    // symmetric operators: A^T = A
    transpose = false;
  }
  int m = mode;
  if (heat_tabulated(op) && (op->kq_user || op->rhocp_user || op->betaq_user)) m = 1;
  if constexpr (sizeof(T) == 8) {
    // double-float reinitialisation on octree meshes: the plane-by-plane kernel through the cell map
    if (df && !op->map[0]->uniform && kind == K_REINIT && nrhs <= 65535) {
      if (!op->df_ready) {
        MF_TRY(op->qvec_dfh.alloc(sizeof(float) * 81 * op->ncells));
        MF_TRY(op->qvec_dfl.alloc(sizeof(float) * 81 * op->ncells));
        MF_TRY(launch_split_pairs(c, op->qvec64.as<double>(), 81 * op->ncells, op->qvec_dfh.as<float>(),
                                  op->qvec_dfl.as<float>()));
        op->df_ready = true;
      }
      MF_TRY(launch_reinit_df_octree(c, op->map[0], reinterpret_cast<const double*>(src),
                                     reinterpret_cast<double*>(dst), nrhs, ld, op->qvec_dfh.as<float>(),
                                     op->qvec_dfl.as<float>(), op->p.eps, value_coef(op)));
      MF_TRY(launch_dirichlet_copy(c, op->map[0], src, dst, nrhs, ld, 0, false));
      op->variant = "reinit/octree/df64/tabulated/planes";
      return MF_OK;
    }
    // double-float on uniform meshes: the plane-by-plane kernel with the split coefficient table
    // (a value coefficient per Gauss point, rho_cp,q / dt, needs the convective kernel)
    const bool qm = kind == K_HEAT && op->rhocp_user;
    if (df && op->map[0]->uniform && (kind == K_HELM || kind == K_HEAT) && (!qm || beta) && nrhs <= 65535) {
      if (!op->df_ready) {
        MF_TRY(op->qcoef_dfh.alloc(sizeof(float) * 27 * op->ncells));
        MF_TRY(op->qcoef_dfl.alloc(sizeof(float) * 27 * op->ncells));
        MF_TRY(launch_df_coef_split(c, op->map[0], op->qcoef64.as<double>(), op->qcoef_dfh.as<float>(),
                                    op->qcoef_dfl.as<float>()));
        if (beta) {
          MF_TRY(op->qvec_dfh.alloc(sizeof(float) * 81 * op->ncells));
          MF_TRY(op->qvec_dfl.alloc(sizeof(float) * 81 * op->ncells));
          MF_TRY(launch_df_vec_split(c, op->map[0], op->qvec64.as<double>(), op->qvec_dfh.as<float>(),
                                     op->qvec_dfl.as<float>()));
        }
        if (qm) {
          MF_TRY(op->qmass_dfh.alloc(sizeof(float) * 27 * op->ncells));
          MF_TRY(op->qmass_dfl.alloc(sizeof(float) * 27 * op->ncells));
          MF_TRY(launch_df_mass_split(c, op->map[0], op->qmass64.as<double>(), op->qmass_dfh.as<float>(),
                                      op->qmass_dfl.as<float>()));
        }
        op->df_ready = true;
      }
      if (beta)
        MF_TRY(launch_scalar_df_uniform_conv(c, op->map[0], reinterpret_cast<const double*>(src),
                                             reinterpret_cast<double*>(dst), nrhs, ld, op->qcoef_dfh.as<float>(),
                                             op->qcoef_dfl.as<float>(), op->qvec_dfh.as<float>(),
                                             op->qvec_dfl.as<float>(), value_coef(op), transpose,
                                             qm ? op->qmass_dfh.as<float>() : nullptr,
                                             qm ? op->qmass_dfl.as<float>() : nullptr));
      else
        MF_TRY(launch_scalar_df_uniform(c, op->map[0], reinterpret_cast<const double*>(src),
                                        reinterpret_cast<double*>(dst), nrhs, ld, op->qcoef_dfh.as<float>(),
                                        op->qcoef_dfl.as<float>(), value_coef(op)));
      MF_TRY(launch_dirichlet_copy(c, op->map[0], src, dst, nrhs, ld, 0, false));
      op->variant = std::string(kind == K_HELM ? "helmholtz" : "heat") + "/uniform/df64/tabulated/planes" +
                    (beta ? (transpose ? "/conv-T" : "/conv") : "");
      return MF_OK;
    }
  }
  if ((f32 ? op->q2_line32 : op->q2_line64) && (prec == PREC_F64 || prec == PREC_F32) && op->map[0]->uniform &&
      (kind == K_HELM || kind == K_HEAT) && !beta && !transpose && !op->rhocp_user) {
    // small meshes: 9 threads per cell (the degree-2 line kernel), coefficients from the tables
    MF_TRY(ensure_tables(op));
    const T* coef = f32 ? reinterpret_cast<const T*>(op->qcoef32.as<float>())
                        : reinterpret_cast<const T*>(op->qcoef64.as<double>());
    for (int r = 0; r < nrhs; ++r) MF_TRY(launch_q2_line<T>(c, op->map[0], src + r * ld, dst + r * ld, coef, value_coef(op)));
    MF_TRY(launch_dirichlet_copy(c, op->map[0], src, dst, nrhs, ld, 0, f32));
    op->variant = std::string(kind == K_HELM ? "helmholtz" : "heat") + "/uniform" + pname + "/tabulated/line-per-thread";
    return MF_OK;
  }
  ScalarArgs<T> a = scalar_args<T>(op, src, dst, nrhs, ld);
  MF_TRY(launch_scalar_apply(c, op->map[0], kind, m, beta, transpose, prec, &a));
  MF_TRY(launch_dirichlet_copy(c, op->map[0], src, dst, nrhs, ld, 0, f32));
  op->variant = std::string(kind == K_HELM ? "helmholtz" : kind == K_HEAT ? "heat" : "reinit") +
                (op->map[0]->uniform ? "/uniform" : "/octree") + pname +
                (m == 0 ? "/inkernel" : "/tabulated") + (beta ? (transpose ? "/conv-T" : "/conv") : "") + "/block" +
                std::to_string(op->map[0]->uniform ? 128 : op->block) +
                (op->persistent_blocks > 0 ? "/persistent" + std::to_string(op->persistent_blocks) : "");
  return MF_OK;
}
template mf_status apply_impl<double>(mf_op*, const double*, double*, int, int64_t, bool, int);

mf_status diag64(mf_op* op, double** out);

// B^T p (which 0, into the three velocity blocks), B u (which 1, into the pressure block) or the
// approximate Schur complement B D^-1 B^T p (which 2, pressure to pressure; D the 3 x 3 nodal
// blocks of A_uu; work vectors allocated per call)
template <typename T> mf_status oseen_coupling(mf_op* op, int which, const T* src, T* dst) {
  if (op->p.kind != MF_OP_OSEEN) return fail(MF_EINVAL, "coupling blocks exist for the Oseen operator only");
  if (which < 0 || which > 2) return fail(MF_EINVAL, "which must be 0 (B^T p), 1 (B u) or 2 (B D^-1 B^T p)");
  const int64_t nu = op->map[0]->n_dofs, np = op->map[1]->n_dofs;
  if (which == 2) {
    MF_TRY(check_fields(op));
    DevBuf ua, ub;
    if constexpr (sizeof(T) == 4) {
      // the preconditioner's form: the assembled 125-point stencil from the fp32 block inverses
      const int* gn = op->map[0]->mesh->n;
      DevBuf sc, pinv;
      MF_TRY(ua.alloc(sizeof(float) * 9 * size_t(nu)));
      MF_TRY(ub.alloc(2 * size_t(stencil_halves(np))));
      MF_TRY(sc.alloc(sizeof(float) * size_t(np)));
      MF_TRY(pinv.alloc(sizeof(float) * size_t(np)));
      MF_TRY(oseen_blocks32(op, ua.as<float>(), pinv.as<float>()));
      MF_TRY(launch_schur_assemble_f32(op->ctx, op->map[0], ua.as<float>(), ub.p, sc.as<float>()));
      MF_TRY(stencil125_apply(op->ctx, ub.p, sc.as<float>(), src, dst, gn[0], gn[1], gn[2], nullptr));
      MF_CUDA_TRY(cudaStreamSynchronize(op->ctx->stream));  // before sc is freed
    } else {
      MF_TRY(diag64(op, nullptr));
      MF_TRY(ua.alloc(sizeof(T) * 3 * size_t(nu)));
      MF_TRY(ub.alloc(sizeof(T) * 3 * size_t(nu)));
      MF_TRY(oseen_coupling<T>(op, 0, src, ua.as<T>()));
      MF_TRY(block_jacobi<T>(op->ctx, nu, 0, op->blk64.as<double>(), nullptr, ua.as<T>(), ub.as<T>()));
      MF_TRY(oseen_coupling<T>(op, 1, ub.as<T>(), dst));
    }
    MF_CUDA_TRY(cudaStreamSynchronize(op->ctx->stream));  // before the work vectors are freed
    return MF_OK;
  }
  MF_CUDA_TRY(cudaMemsetAsync(dst, 0, sizeof(T) * size_t(which == 0 ? 3 * nu : np), op->ctx->stream));
  if constexpr (sizeof(T) == 4) return launch_oseen_coupling_f32(op->ctx, op->map[0], which, src, dst);
  else return launch_oseen_coupling_f64(op->ctx, op->map[0], which, src, dst);
}
template mf_status oseen_coupling<double>(mf_op*, int, const double*, double*);
template mf_status oseen_coupling<float>(mf_op*, int, const float*, float*);
template mf_status apply_impl<float>(mf_op*, const float*, float*, int, int64_t, bool, int);

mf_status diag64(mf_op* op, double** out) {
  if (!op->diag_ready) {
    MF_TRY(ensure_tables(op));
    if (qk_degree(op)) {
      MF_TRY(op->diag64.alloc(sizeof(double) * op->n));
      MF_TRY(launch_qk_diag(op->ctx, op->map[0], op->qcoef64.as<double>(), op->p.mass_coef, op->diag64.as<double>()));
    } else if (op->p.kind == MF_OP_OSEEN) {
      const int64_t nu = op->map[0]->n_dofs, np = op->map[1]->n_dofs;
      MF_TRY(op->blk64.alloc(sizeof(double) * 9 * nu));
      MF_TRY(op->pdiag64.alloc(sizeof(double) * np));
      OseenArgs<double> a = oseen_args<double>(op, nullptr, nullptr);
      MF_TRY(launch_oseen_blockdiag(op->ctx, op->map[0], op->map[1], a, op->blk64.as<double>(), op->pdiag64.as<double>()));
    } else {
      MF_TRY(op->diag64.alloc(sizeof(double) * op->n));
      ScalarArgs<double> a = scalar_args<double>(op, nullptr, nullptr, 1, op->n);
      const int kind = scalar_kind(op);
      MF_TRY(launch_scalar_diag(op->ctx, op->map[0], kind, heat_convection(op), a, op->diag64.as<double>()));
    }
    op->diag_ready = true;
  }
  if (out) *out = op->diag64.as<double>();
  return MF_OK;
}

}  // namespace mf

extern "C" {

mf_status mf_apply(mf_op* op, const void* src, void* dst, int nrhs, int64_t ld, int dtype) {
  MF_GUARD_BEGIN
  if (!op || !src || !dst) return fail(MF_EINVAL, "NULL argument");
  if (nrhs < 1 || ld < op->n) return fail(MF_EINVAL, "nrhs must be >= 1 and ld >= n");
  if (dtype == MF_F64) return apply_impl<double>(op, (const double*)src, (double*)dst, nrhs, ld, false, PREC_F64);
  if (dtype == MF_DF64) return apply_impl<double>(op, (const double*)src, (double*)dst, nrhs, ld, false, PREC_DF64);
  if (dtype == MF_F32) return apply_impl<float>(op, (const float*)src, (float*)dst, nrhs, ld, false, PREC_F32);
  return fail(MF_EUNSUPPORTED, "apply precision must be MF_F64, MF_DF64 or MF_F32");
  MF_GUARD_END
}

mf_status mf_oseen_coupling(mf_op* op, int which, const void* src, void* dst, int dtype) {
  MF_GUARD_BEGIN
  if (!op || !src || !dst) return fail(MF_EINVAL, "NULL argument");
  if (dtype == MF_F64) return oseen_coupling<double>(op, which, (const double*)src, (double*)dst);
  if (dtype == MF_F32) return oseen_coupling<float>(op, which, (const float*)src, (float*)dst);
  return fail(MF_EUNSUPPORTED, "coupling precision must be MF_F64 or MF_F32");
  MF_GUARD_END
}

mf_status mf_interface_sources(mf_op* op, const mf_evaporation* ev, const double* T, double* f_u, double* f_p,
                               double* f_T) {
  MF_GUARD_BEGIN
  if (!op || !ev || !T) return fail(MF_EINVAL, "NULL argument");
  if (op->p.kind != MF_OP_OSEEN) return fail(MF_EINVAL, "interface sources live on an Oseen operator's maps");
  if (!op->phi) return fail(MF_EINVAL, "interface sources need MF_FIELD_PHI");
  if (!op->map[0]->uniform) return fail(MF_EUNSUPPORTED, "interface sources on octree maps");
  if (ev->mass_flux != MF_MASS_FLUX_KNIGHT && ev->mass_flux != MF_MASS_FLUX_TANASAWA)
    return fail(MF_EINVAL, "unknown mass-flux model");
  if (!(op->p.rho_l > 0 && op->p.rho_g > 0 && op->p.rho_l != op->p.rho_g))
    return fail(MF_EINVAL, "interface sources need distinct positive rho_l, rho_g");
  if (!(ev->rhocp_liquid > 0 && ev->rhocp_gas > 0)) return fail(MF_EINVAL, "rho c_p must be positive");
  if (ev->mass_flux == MF_MASS_FLUX_KNIGHT && !(ev->t_boil > 0 && ev->molar_mass > 0))
    return fail(MF_EINVAL, "Knight's mass flux needs T_v > 0 and M > 0");
  if (!f_u && !f_p && !f_T) return MF_OK;
  return launch_interface_sources(op->ctx, op->map[0], op->map[1], op->p, op->phi, *ev, T, f_u, f_p, f_T);
  MF_GUARD_END
}

mf_status mf_apply_packed16(mf_op* op, const float* src, float* dst, int nrhs, int64_t ld, int format) {
  MF_GUARD_BEGIN
  if (!op || !src || !dst) return fail(MF_EINVAL, "NULL argument");
  if (nrhs < 1 || ld < op->n) return fail(MF_EINVAL, "nrhs must be >= 1 and ld >= n");
  if (format != MF_F16 && format != MF_BF16) return fail(MF_EINVAL, "format must be MF_F16 or MF_BF16");
  return apply_impl<float>(op, src, dst, nrhs, ld, false, format == MF_F16 ? PREC_F16 : PREC_BF16);
  MF_GUARD_END
}

mf_status mf_apply_tc(mf_op* op, const float* src, float* dst, int nrhs, int64_t ld) {
  MF_GUARD_BEGIN
  if (!op || !src || !dst) return fail(MF_EINVAL, "NULL argument");
  if (nrhs < 1 || ld < op->n) return fail(MF_EINVAL, "nrhs must be >= 1 and ld >= n");
  return apply_tc(op, src, dst, nrhs, ld);
  MF_GUARD_END
}

}  // extern "C"

namespace mf {

mf_status apply_tc(mf_op* op, const float* src, float* dst, int nrhs, int64_t ld) {
  if (qk_degree(op) != 3) return fail(MF_EUNSUPPORTED, "tensor-core applies: Q3 Helmholtz operators");
  MF_TRY(check_fields(op));
  MF_TRY(ensure_tables(op));
  if (!op->tc_ready) {
    const int64_t ntiles = (op->ncells + 127) / 128;
    MF_TRY(op->qcoef_tc.alloc(sizeof(float) * ntiles * 128 * 64));
    MF_TRY(launch_tc_coef_layout(op->ctx, op->map[0], op->qcoef32.as<float>(), op->qcoef_tc.as<float>()));
    op->tc_ready = true;
  }
  for (int r = 0; r < nrhs; ++r) {
    MF_CUDA_TRY(cudaMemsetAsync(dst + r * ld, 0, sizeof(float) * op->n, op->ctx->stream));
    MF_TRY(launch_helmholtz_q3_tc(op->ctx, op->map[0], src + r * ld, dst + r * ld, op->qcoef_tc.as<float>(),
                                  op->p.mass_coef));
  }
  op->variant = "helmholtz_q3/uniform/f32/tcgen05-bf16x3/dense";
  return MF_OK;
}

}  // namespace mf

extern "C" {

mf_status mf_apply_transpose(mf_op* op, const void* src, void* dst, int nrhs, int64_t ld, int dtype) {
  MF_GUARD_BEGIN
  if (!op || !src || !dst) return fail(MF_EINVAL, "NULL argument");
  if (nrhs < 1 || ld < op->n) return fail(MF_EINVAL, "nrhs must be >= 1 and ld >= n");
  if (dtype == MF_F64) return apply_impl<double>(op, (const double*)src, (double*)dst, nrhs, ld, true, PREC_F64);
  if (dtype == MF_DF64) return apply_impl<double>(op, (const double*)src, (double*)dst, nrhs, ld, true, PREC_DF64);
  if (dtype == MF_F32) return apply_impl<float>(op, (const float*)src, (float*)dst, nrhs, ld, true, PREC_F32);
  return fail(MF_EUNSUPPORTED, "apply precision must be MF_F64, MF_DF64 or MF_F32");
  MF_GUARD_END
}

mf_status mf_dot(mf_ctx* c, const void* x, const void* y, int64_t n, int64_t ld, int nvec, int dtype, double* out) {
  MF_GUARD_BEGIN
  if (!c || !x || !y || !out) return fail(MF_EINVAL, "NULL argument");
  if (n < 0 || nvec < 1 || nvec > 64 || (nvec > 1 && ld < n)) return fail(MF_EINVAL, "need n >= 0, 1 <= nvec <= 64, ld >= n");
  if (dtype == MF_F64) return dot_batched<double>(c, (const double*)x, (const double*)y, n, ld, nvec, out);
  if (dtype == MF_F32) return dot_batched<float>(c, (const float*)x, (const float*)y, n, ld, nvec, out);
  return fail(MF_EUNSUPPORTED, "dot precision must be MF_F64 or MF_F32");
  MF_GUARD_END
}

mf_status mf_diagonal(mf_op* op, void* dst, int dtype) {
  MF_GUARD_BEGIN
  if (!op || !dst) return fail(MF_EINVAL, "NULL argument");
  if (op->p.kind == MF_OP_OSEEN) return fail(MF_EUNSUPPORTED, "Oseen uses nodal block diagonals");
  double* d;
  MF_TRY(diag64(op, &d));
  if (dtype == MF_F64)
    MF_CUDA_TRY(cudaMemcpyAsync(dst, d, sizeof(double) * op->n, cudaMemcpyDeviceToDevice, op->ctx->stream));
  else if (dtype == MF_F32)
    MF_TRY(convert<double, float>(op->ctx, op->n, d, static_cast<float*>(dst)));
  else
    return fail(MF_EUNSUPPORTED, "diagonal precision must be MF_F64 or MF_F32");
  return MF_OK;
  MF_GUARD_END
}

}  // extern "C"
