// Q3 Helmholtz apply on the fifth-generation tensor cores (tcgen05 with the accumulators in tensor
// memory), for fp32 vectors.  The cell operator of the sum-factorised kernel, written densely: with
// G the 256 x 64 matrix of the 64 Q3 shape functions and their three reference derivatives at the
// 64 Gauss points,
//   D1 = U G^T        (128 cells x 256: values and reference gradients at the Gauss points)
//   P  = pointwise(D1) (w c h^3 on the values, w a_q h on the gradients)
//   V  = P G          (128 cells x 64: the cell contributions at the nodes)
// are two dense products per tile of 128 cells.  To keep fp32-class accuracy on the bf16 tensor
// cores every operand x is split into x_hi = bf16(x) and x_lo = bf16(x - x_hi) and each product is
// x_hi y_hi + x_hi y_lo + x_lo y_hi with fp32 accumulation.  One CTA per SM (224 KB of operand
// images and coefficients in shared memory, 320 of the 512 tensor-memory columns), persistent over the tiles; four
// threads per cell gather, apply the coefficients and scatter; thread 0 issues the MMAs.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "ops.h"

namespace mf {

void qk_host_tables(int k, double* S, double* Sp, double* W);

namespace {

constexpr int kM = 128;   // cells per tile (rows of the MMA)
constexpr int kNb = 64;   // Q3 nodes per cell
constexpr int kNq = 256;  // 64 values + 3 x 64 reference gradients
// shared memory image (bytes); the operands in the no-swizzle layouts
constexpr uint32_t kB1H = 0, kB1L = 32768;          // G: B of product 1 (K-major) and of product 2 (MN-major)
constexpr uint32_t kA1H = 65536, kA1L = 81920;      // 128 x 64 nodal values
constexpr uint32_t kA2H = 98304, kA2L = 114688;     // 128 x 64 chunk of P
constexpr uint32_t kStage = 131072;                 // two 128 x 64 fp32 coefficient tiles (TMA)
constexpr uint32_t kBar = 196608, kSlot = 196640, kSmem = 196656;
constexpr uint32_t kImage = 65536;  // the G image, copied from global memory once per CTA
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kStageBytes = 32768;

// byte offset of element (r, c) of a K-major tile with K columns: 8 x 16-byte core matrices,
// adjacent along K (leading offset 128 B), row groups of 8 after all K columns (stride K/8 * 128 B)
__host__ __device__ constexpr uint32_t kmajor(int r, int c, int K) {
  return uint32_t((r & 7) * 16 + (r >> 3) * (K / 8) * 128 + (c & 7) * 2 + (c >> 3) * 128);
}

// shared memory matrix descriptor (no swizzle): start, leading offset 128 B, stride sbo
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo) {
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t(128 >> 4) << 16) | (uint64_t((sbo >> 4) & 0x3FFF) << 32) |
         (uint64_t(1) << 46);
}

// shared memory matrix descriptor (no swizzle) with explicit leading and stride offsets
__device__ __forceinline__ uint64_t sdesc2(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) | (uint64_t((sbo >> 4) & 0x3FFF) << 32) |
         (uint64_t(1) << 46);
}

// instruction descriptor of kind::f16: bf16 A (K-major) and B (K-major, or MN-major with b_mn),
// fp32 D, M x N
__host__ __device__ constexpr uint32_t idesc(int M, int N, bool b_mn = false) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (b_mn ? (1u << 16) : 0u) | (uint32_t(N >> 3) << 17) |
         (uint32_t(M >> 4) << 24);
}

__constant__ float cTcW[64];  // Gauss weights w_q of the 64 points (x fastest)

struct TcArgs {
  const float* src;
  float* dst;
  const float* coef;  // a per Gauss point, per tile of 128 cells: [tile][q][row]
  const uint4* image; // the G images (kImage bytes)
  int* err;           // host-mapped error flag
  int nx, ny;
  int64_t sx, sy, ncells;
  float mass_h3, h;
};

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// wait for the phase of an mbarrier, at most one second (global timer); false on timeout
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t phase) {
  uint64_t t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    if (ok) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 1000000000ull) return false;
  }
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive fp32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 8 consecutive K-elements of one row as bf16 hi and lo parts: two 16-byte stores into the core
// matrices of the hi and lo images
__device__ __forceinline__ void put_split8(unsigned char* sm, uint32_t hi, uint32_t lo, uint32_t off, const float* x) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(x[2 * e], x[2 * e + 1]);
    const __nv_bfloat162 b = __floats2bfloat162_rn(x[2 * e] - __low2float(a), x[2 * e + 1] - __high2float(a));
    h[e] = *reinterpret_cast<const uint32_t*>(&a);
    l[e] = *reinterpret_cast<const uint32_t*>(&b);
  }
  *reinterpret_cast<uint4*>(sm + hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(sm + lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// nodes 16 quarter .. 16 quarter + 15 of a cell (zeros for a cell past the end)
__device__ __forceinline__ void gather16(const TcArgs& A, bool on, int64_t base, int quarter, float* x) {
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const int l = 16 * quarter + e;
    x[e] = on ? __ldg(A.src + base + (l & 3) + A.sx * ((l >> 2) & 3) + A.sy * (l >> 4)) : 0.0f;
  }
}

__device__ __forceinline__ bool tile_cell(const TcArgs& A, int64_t tile, int row, int64_t& base) {
  const int64_t cell = tile * kM + row;
  base = 0;
  if (cell >= A.ncells) return false;
  const int64_t cx = cell % A.nx, cy = (cell / A.nx) % A.ny, cz = cell / (int64_t(A.nx) * A.ny);
  base = 3 * cx + A.sx * (3 * cy) + A.sy * (3 * cz);
  return true;
}

// Four threads per cell: thread t works on row t % 128 of the tile and on quarter t / 128 of its
// columns (warps w, w + 4, w + 8 and w + 12 read the same tensor-memory lanes).  Software-pipelined over the
// CTA's tiles: the next tile's coefficients arrive by a TMA bulk copy and its nodal values are
// loaded while the coefficients of the current one are applied, and its first product runs while
// the current tile is scattered.  Product 2 reads the same G image as product 1, as an MN-major B.
__global__ void __launch_bounds__(512, 1) k_helmholtz_q3_tc(TcArgs A) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sb = static_cast<uint32_t>(__cvta_generic_to_shared(sm));
  const int tid = threadIdx.x, warp = tid >> 5, row = tid & 127, quarter = tid >> 7;
  __shared__ int s_abort;
  const uint32_t bar1 = sb + kBar, bar2 = sb + kBar + 8, bars = sb + kBar + 16;  // bars: 2 stage barriers
  // the G image (once per CTA), the barriers, tensor memory
  for (uint32_t i = tid; i < kImage / 16; i += blockDim.x) reinterpret_cast<uint4*>(sm)[i] = A.image[i];
  if (tid == 0) {
    s_abort = 0;
    for (int b = 0; b < 4; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sb + kBar + 8 * b));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sb + kSlot),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
  uint32_t ph1 = 0, ph2 = 0, phs[2] = {0, 0};
  const uint32_t id1 = idesc(kM, kNq), id2 = idesc(kM, kNb, true);
  const int64_t ntiles = (A.ncells + kM - 1) / kM;
  const uint32_t rowoff = uint32_t((row & 7) * 16 + (row >> 3) * 1024);  // row's place in a 64-column tile
  // asynchronous work committed and not yet waited for; a wait clears its flag and advances its
  // phase only when it succeeds, so timed-out work is waited for again before the exit
  int pend1 = 0, pend2 = 0, pends[2] = {0, 0};
  auto wait1 = [&]() {
    if (wait_phase(bar1, ph1)) { ph1 ^= 1; pend1 = 0; } else { s_abort = 1; }
  };
  auto wait2 = [&]() {
    if (wait_phase(bar2, ph2)) { ph2 ^= 1; pend2 = 0; } else { s_abort = 1; }
  };
  auto waits = [&](int b) {
    if (wait_phase(bars + 8 * b, phs[b])) { phs[b] ^= 1; pends[b] = 0; } else { s_abort = 1; }
  };
  // thread 0: the coefficient tile t into stage buffer b by one bulk copy
  auto fetch_coef = [&](int64_t t, int b) {
    const uint32_t dst = sb + kStage + b * kStageBytes, bar = bars + 8 * b;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kStageBytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(A.coef + t * (kM * 64)), "r"(kStageBytes), "r"(bar)
                 : "memory");
  };
  int64_t tile = blockIdx.x;
  int64_t base = 0;
  bool on = tile < ntiles ? tile_cell(A, tile, row, base) : false;
  // prologue: the first tile's coefficients and nodal values
  if (tile < ntiles && tid == 0) fetch_coef(tile, 0);
  if (tile < ntiles) pends[0] = 1;
  if (tile < ntiles) {
    float x[16];
    gather16(A, on, base, quarter, x);
#pragma unroll
    for (int g = 0; g < 2; ++g) put_split8(sm, kA1H, kA1L, rowoff + (2 * quarter + g) * 128, x + 8 * g);
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + kSlot);
  const uint32_t d1 = tmem, d2 = tmem + 256;
  auto issue_product1 = [&]() {
    for (int t = 0; t < 3; ++t) {
      const uint32_t a = sb + (t == 2 ? kA1L : kA1H), b = sb + (t == 1 ? kB1L : kB1H);
      for (int s = 0; s < 4; ++s) mma_bf16(d1, sdesc(a + s * 256, 1024), sdesc(b + s * 256, 1024), id1, (t | s) != 0);
    }
    commit(bar1);
  };
  if (tile < ntiles && tid == 0) issue_product1();
  pend1 = tile < ntiles ? 1 : 0;
  int sbuf = 0;  // stage buffer of the current tile
  for (; tile < ntiles; tile += gridDim.x, sbuf ^= 1) {
    const int64_t next = tile + gridDim.x;
    // 1. D1 of this tile and its coefficients are ready; the next tile's coefficients are fetched
    wait1();
    waits(sbuf);
    __syncthreads();
    if (s_abort) break;
    fence_after();
    if (next < ntiles && tid == 0) fetch_coef(next, sbuf ^ 1);
    if (next < ntiles) pends[sbuf ^ 1] = 1;
    const float* stage = reinterpret_cast<const float*>(sm + kStage + sbuf * kStageBytes);
    // the next tile's nodal values into registers
    int64_t nbase = 0;
    const bool non = next < ntiles ? tile_cell(A, next, row, nbase) : false;
    float xn[16];
    gather16(A, non, nbase, quarter, xn);
    // 2. per 64-column chunk: coefficients, then V += P_chunk G_chunk
    for (int j = 0; j < 4; ++j) {
      if (j > 0) {
        wait2();
        __syncthreads();
        if (s_abort) break;
        fence_after();
      }
      {
        float v[16];
        const int q0 = quarter * 16;
        tmem_ld16(d1 + lane_base + j * 64 + q0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int q = q0 + i;
          v[i] *= j == 0 ? cTcW[q] * A.mass_h3 : cTcW[q] * stage[q * kM + row] * A.h;
        }
        put_split8(sm, kA2H, kA2L, rowoff + (q0 >> 3) * 128, v);
        put_split8(sm, kA2H, kA2L, rowoff + ((q0 >> 3) + 1) * 128, v + 8);
      }
      fence_async_smem();
      fence_before();
      __syncthreads();
      if (tid == 0) {
        fence_after();
        for (int t = 0; t < 3; ++t) {
          const uint32_t a = sb + (t == 2 ? kA2L : kA2H), b = sb + (t == 1 ? kB1L : kB1H);
          // B = G^T read from the product-1 image as MN-major without swizzle: 8 nodes contiguous
          // (16 B), node groups 128 B apart (the stride offset in this mode), Gauss-point groups of
          // 8 rows 1024 B apart (the leading offset)
          for (int s = 0; s < 4; ++s)
            mma_bf16(d2, sdesc(a + s * 256, 1024), sdesc2(b + (8 * j + 2 * s) * 1024, 1024, 128), id2, (j | t | s) != 0);
        }
        commit(bar2);
      }
      pend2 = 1;
    }
    if (s_abort) break;
    // 3. the next tile's U (its first product reads it while this tile is scattered); D1 of this
    //    tile has been read in full
    if (next < ntiles) {
#pragma unroll
      for (int g = 0; g < 2; ++g) put_split8(sm, kA1H, kA1L, rowoff + (2 * quarter + g) * 128, xn + 8 * g);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (next < ntiles && tid == 0) {
      fence_after();
      issue_product1();
    }
    if (next < ntiles) pend1 = 1;
    // 4. this tile's V, scattered
    wait2();
    __syncthreads();
    if (s_abort) break;
    fence_after();
    {
      float v[16];
      tmem_ld16(d2 + lane_base + quarter * 16, v);
      if (on)
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int l = quarter * 16 + i;
          atomicAdd(A.dst + base + (l & 3) + A.sx * ((l >> 2) & 3) + A.sy * (l >> 4), v[i]);
        }
    }
    on = non;
    base = nbase;
    fence_before();
    __syncthreads();
  }
  if (s_abort) {
    // report, give the work still in flight its time, then free the tensor memory
    if (tid == 0) atomicExch(A.err, 1);
    if (pend1) wait_phase(bar1, ph1);
    if (pend2) wait_phase(bar2, ph2);
    for (int b = 0; b < 2; ++b)
      if (pends[b]) wait_phase(bars + 8 * b, phs[b]);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

// coefficients [cell][64] -> per tile of 128 cells [tile][q][row] (rows past the end: 0)
__global__ void k_tc_coef_layout(const float* __restrict__ in, float* __restrict__ out, int64_t ncells, int64_t ntiles) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= ntiles * kM * 64) return;
  const int64_t t = i / (kM * 64);
  const int q = int((i / kM) % 64), r = int(i % kM);
  const int64_t cell = t * kM + r;
  out[i] = cell < ncells ? in[cell * 64 + q] : 0.0f;
}

// the G image: B of product 1 (256 rows x K = 64, K-major), hi then lo
std::vector<uint16_t> make_image() {
  double S[16], Sp[16], W[4];
  qk_host_tables(3, S, Sp, W);
  std::vector<uint16_t> img(kImage / 2, 0);
  for (int col = 0; col < kNq; ++col) {
    const int part = col / 64, q = col % 64, qa = q % 4, qb = (q / 4) % 4, qc = q / 16;
    for (int l = 0; l < kNb; ++l) {
      const int a = l % 4, b = (l / 4) % 4, c = l / 16;
      const double fa = part == 1 ? Sp[4 * qa + a] : S[4 * qa + a];
      const double fb = part == 2 ? Sp[4 * qb + b] : S[4 * qb + b];
      const double fc = part == 3 ? Sp[4 * qc + c] : S[4 * qc + c];
      const float g = float(fa * fb * fc);
      const __nv_bfloat16 h = __float2bfloat16_rn(g);
      const __nv_bfloat16 lo = __float2bfloat16_rn(g - __bfloat162float(h));
      const uint32_t off = kmajor(col, l, kNb);
      std::memcpy(&img[(kB1H + off) / 2], &h, 2);
      std::memcpy(&img[(kB1L + off) / 2], &lo, 2);
    }
  }
  return img;
}

}  // namespace

mf_status launch_tc_coef_layout(mf_ctx* ctx, const mf_dofmap* m, const float* in, float* out) {
  const int64_t ntiles = (m->n_cells + kM - 1) / kM, n = ntiles * kM * 64;
  k_tc_coef_layout<<<int((n + 255) / 256), 256, 0, ctx->stream>>>(in, out, m->n_cells, ntiles);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

// Host-mapped error flag of the tensor-core kernel: set by a launch whose bounded wait ran out.
static int* g_tc_h_err = nullptr;

mf_status tc_take_error() {
  if (!g_tc_h_err || !*reinterpret_cast<volatile int*>(g_tc_h_err)) return MF_OK;
  *reinterpret_cast<volatile int*>(g_tc_h_err) = 0;   // reported once
  return fail(MF_ETIMEOUT, "a tensor-core apply timed out waiting on its MMAs");
}

mf_status launch_helmholtz_q3_tc(mf_ctx* ctx, const mf_dofmap* m, const float* src, float* dst, const float* coef,
                                 double mass) {
  static DevBuf image;
  static int* d_err = nullptr;
  static bool ready = false;
  int*& h_err = g_tc_h_err;
  if (!ready) {
    const std::vector<uint16_t> img = make_image();
    MF_TRY(image.alloc(kImage));
    MF_CUDA_TRY(cudaMemcpy(image.p, img.data(), kImage, cudaMemcpyHostToDevice));
    double S[16], Sp[16], W[4];
    qk_host_tables(3, S, Sp, W);
    float w[64];
    for (int q = 0; q < 64; ++q) w[q] = float(W[q % 4] * W[(q / 4) % 4] * W[q / 16]);
    MF_CUDA_TRY(cudaMemcpyToSymbol(cTcW, w, sizeof(w)));
    MF_CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&h_err), sizeof(int), cudaHostAllocMapped));
    *h_err = 0;
    MF_CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&d_err), h_err, 0));
    MF_CUDA_TRY(cudaFuncSetAttribute(k_helmholtz_q3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmem + 1024)));
    ready = true;
  }
  MF_TRY(tc_take_error());   // a launch issued earlier on this process timed out
  TcArgs a{};
  a.src = src;
  a.dst = dst;
  a.coef = coef;
  a.image = image.as<const uint4>();
  a.err = d_err;
  a.nx = m->mesh->n[0];
  a.ny = m->mesh->n[1];
  a.sx = m->R[0] + 1;
  a.sy = a.sx * (m->R[1] + 1);
  a.ncells = m->n_cells;
  const double h = m->mesh->h0;
  a.mass_h3 = float(mass * h * h * h);
  a.h = float(h);
  const int64_t ntiles = (m->n_cells + kM - 1) / kM;
  const int grid = int(std::min<int64_t>(ntiles, ctx->sm_count > 0 ? ctx->sm_count : 152));
  k_helmholtz_q3_tc<<<grid, 512, kSmem + 1024, ctx->stream>>>(a);
  ctx->launches++;
  MF_CUDA_TRY(cudaGetLastError());
  return MF_OK;
}

}  // namespace mf
