// Internal structures of libmfgb (host side).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mfgb.h"

namespace mf {

void set_error(const std::string& msg);
mf_status fail(mf_status st, const std::string& msg);

#define MF_CUDA_TRY(...)                                                                   \
  do {                                                                                     \
    cudaError_t e_ = (__VA_ARGS__);                                                           \
    if (e_ != cudaSuccess)                                                                 \
      return ::mf::fail(MF_ECUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define MF_TRY(...)                  \
  do {                               \
    mf_status s_ = (__VA_ARGS__);    \
    if (s_ != MF_OK) return s_;      \
  } while (0)

// frees the blocks that every context keeps for reuse (after a failed cudaMalloc)
void trim_block_pools();

// Device buffer owned by a handle.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  // a buffer that already has n bytes is kept (its user rewrites it; work queued on the stream
  // before still reads the old contents first)
  mf_status alloc(size_t n) {
    if (p && n == bytes) return MF_OK;
    release();
    if (n == 0) return MF_OK;
    if (cudaMalloc(&p, n) != cudaSuccess) {
      cudaGetLastError();
      trim_block_pools();
      if (cudaMalloc(&p, n) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        return fail(MF_ENOMEM, "cudaMalloc of " + std::to_string(n) + " bytes failed");
      }
    }
    bytes = n;
    return MF_OK;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
  template <class T> mf_status upload(const std::vector<T>& v, cudaStream_t s) {
    MF_TRY(alloc(v.size() * sizeof(T)));
    if (!v.empty()) MF_CUDA_TRY(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return MF_OK;
  }
};

// Device blocks a context keeps for reuse (the solvers' work vectors, allocated and freed on every
// solve).  A block handed back may still be read by work queued on the context's stream; every
// later user queues its work on the same stream, so the reuse needs no synchronisation.  Sizes
// are rounded up (to 512 bytes, or to 2 MiB from 1 MiB on) and matched exactly; when cudaMalloc
// fails, the kept blocks of every context are freed and the allocation is retried.
struct BlockPool {
  std::mutex mu;  // guards keep (trim_block_pools may run on another thread)
  std::multimap<size_t, void*> keep;
  size_t kept = 0;
  BlockPool();
  ~BlockPool();
  BlockPool(const BlockPool&) = delete;
  BlockPool& operator=(const BlockPool&) = delete;
  static size_t rounded(size_t n) {
    const size_t big = size_t(2) << 20, small = 512;
    return n >= (size_t(1) << 20) ? (n + big - 1) / big * big : (n + small - 1) / small * small;
  }
  mf_status get(size_t n, void** out);
  void put(void* blk, size_t n);
  void trim();
};

// the pool of the context whose solve runs on this thread (set by a PoolScope), or NULL
extern thread_local BlockPool* tl_pool;
struct PoolScope {
  BlockPool* prev;
  explicit PoolScope(BlockPool* p) : prev(tl_pool) { tl_pool = p; }
  ~PoolScope() { tl_pool = prev; }
};

}  // namespace mf

// Layout of the device / pinned host scalar areas (doubles).
namespace mf {
constexpr int kScalarsCG = 0;        // 64 RHS x 8 CG scalars
constexpr int kScalarsLanczos = 512;
constexpr int kScalarsResid = 1024;  // 2 x 64
constexpr int kScalarsGmres = 1536;  // 2 (m + 1) <= 128
constexpr int kScalarsScale = 2048;  // 64
constexpr int kScalarsHeat = 2560;   // 8
constexpr int kScalarsTri = 3072;    // Oseen block-triangular inner solves: 2 (k + 1) + 8 <= 512
constexpr int kScalarsCGSteps = 3584;  // 64 step counters of the batched CG's on-device stopping test
constexpr int kScalarsTotal = 4096;
}  // namespace mf

struct mf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t launches = 0;
  int sm_count = 0;
  mf::DevBuf scratch;   // reduction partials (fixed size, allocated with the context)
  mf::DevBuf counters;  // 64 arrival counters of the reductions (zero between launches)
  mf::DevBuf scalars;   // device scalars of the solvers
  double* host_scalars = nullptr;  // pinned
  // CUDA graphs are captured on a private stream (the legacy default stream cannot be
  // captured), fenced against `stream` with an event on both sides.
  cudaStream_t capture_stream = nullptr;
  cudaEvent_t fence = nullptr;
  mf::BlockPool pool;   // work vectors of the solvers, reused in this stream's order
};

struct mf_mesh {
  mf_ctx* ctx = nullptr;
  bool octree = false;
  int n[3] = {0, 0, 0};   // uniform: cells per axis; octree: base cells per axis (cubic)
  int base = 0, levels = 0;
  double lo[3], hi[3];
  double h0 = 0;          // edge of a root (uniform: every) cell
  // octree leaves in Morton order: level, i, j, k
  std::vector<int32_t> leaves;
};

struct mf_dofmap {
  mf_mesh* mesh = nullptr;
  int degree = 2;
  int nb = 27;               // nodes per cell
  uint32_t dirichlet_faces = 0;
  int64_t n_dofs = 0, n_cells = 0;
  int64_t R[3] = {0, 0, 0};  // lattice intervals per axis
  // uniform: implicit lattice (no maps).  octree: explicit maps below.
  bool uniform = true;
  // host copies
  std::vector<int32_t> cell_map;        // [cell][nb] free index or -(1+hang rank)
  std::vector<int64_t> con_rowptr;      // hanging rows
  std::vector<int32_t> con_cols;
  std::vector<double> con_w;
  std::vector<int64_t> free_keys;       // lattice key of each free DoF
  std::vector<uint8_t> dirichlet;       // per free DoF
  std::vector<int32_t> dirichlet_list;  // indices of Dirichlet DoFs
  std::vector<uint8_t> cell_level;      // per cell
  std::vector<int32_t> cell_anchor;     // per cell: i, j, k on its level grid
  // device copies
  mf::DevBuf d_cell_map;     // int32 SoA [nb][n_cells_pad]
  mf::DevBuf d_cell_level;   // uint8 [n_cells]
  mf::DevBuf d_cell_flags;   // uint8 [n_cells]: bit0 = has constrained node
  mf::DevBuf d_con_rowptr;   // int32 [n_con+1]
  mf::DevBuf d_con_cols;     // int32
  mf::DevBuf d_con_w;        // double
  mf::DevBuf d_con_wf;       // float
  mf::DevBuf d_dir_list;     // int32
  mf::DevBuf d_dir_flag;     // uint8 [n_dofs] (octree with Dirichlet faces)
  mf::DevBuf d_order;        // int32 processing order of cells (unconstrained first)
  int64_t n_cells_pad = 0;
  int64_t n_unconstrained = 0;
  int64_t n_constrained_cells = 0;
};

namespace mf {
mf_status build_uniform_dofmap(mf_dofmap* m);
mf_status build_octree_dofmap(mf_dofmap* m);
mf_status upload_dofmap(mf_dofmap* m);
}  // namespace mf
