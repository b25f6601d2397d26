// Shared device helpers of the TSQR kernels: the plan, the shared-memory tile layout that TMA
// fills, TMA and mbarrier wrappers with bounded waits, and block-level reductions.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tsqr {

constexpr int kThreads = 256;     // threads per block of every kernel
constexpr int kMaxLevels = 40;    // tree levels above the chains
constexpr int kMaxArity = 8;
constexpr int kMaxColBlocks = 64; // column blocks of B per apply launch
constexpr int kStatusTimeout = 1;

// Plan::precision: the arithmetic of a factorization.
constexpr int kPrecF64 = 0;      // native FP64
constexpr int kPrecDF = 1;       // double-float (FP32 pairs) everywhere
constexpr int kPrecOzaki = 2;    // native FP64; thin-Q WY products as Ozaki splits on tcgen05
constexpr int kPrecDFOzaki = 3;  // double-float factor and apply; thin Q as in kPrecOzaki
constexpr int kPrecF32 = 16;     // FP32 storage and arithmetic
__host__ __device__ inline bool prec_df(int p) { return p == kPrecDF || p == kPrecDFOzaki; } // bit in the device status word

// Kinds of stacked matrices a Householder QR is taken of (rows that column j's reflector
// touches, besides the pivot row j):
//   PLAIN: one leaf block, rows j+1..N-1 (dense Householder QR).
//   CHAIN: [R; A_k], an upper triangle atop a full block: rows np..N-1 (Algorithm 2 step).
//   NODE : q stacked upper triangles: rows s*np + r with s >= 1, r <= j (eq. fact_2rs).
enum Kind { PLAIN = 0, CHAIN = 1, NODE = 2 };

// Reduction-tree plan.  Leaves are h rows each (the last one ragged); `chain` consecutive
// leaves form one chain, factored by one thread block; chains are the level-0 nodes of an
// arity-q tree whose nodes are numbered level by level.
struct Plan {
  int64_t m;
  int n, np, h;
  int64_t leaves;
  int chain, chains, arity, depth;
  int level_count[kMaxLevels + 1];
  int level_offset[kMaxLevels + 1];
  int total_nodes, tree_nodes;
  int rows_cap;   // rows of the factor kernel's shared tile
  int precision;  // kPrec* below: the arithmetic of the factorization
  int r_only;     // nonzero: R alone; no reflectors, T or tree factors are kept
  int col_major;  // the caller's A, R, Q and B are column-major (element (i, j) at X[j * ld + i])
};

// Offset of element (r, c) of a caller matrix with leading dimension ld, in the plan's layout.
__host__ __device__ __forceinline__ int64_t gidx(const Plan& P, int64_t r, int64_t c, int64_t ld) {
  return P.col_major ? c * ld + r : r * ld + c;
}

__host__ __device__ inline int64_t chain_first_leaf(const Plan& p, int g) { return (int64_t)g * p.chain; }
__host__ __device__ inline int64_t chain_end_leaf(const Plan& p, int g) {
  return (g == p.chains - 1) ? p.leaves : (int64_t)(g + 1) * p.chain;
}

// Device buffers of one factorization (all inside the caller's workspace, except V when the
// reflectors overwrite A).
struct Store {
  double* v;        // m x ldv
  int64_t ldv;
  double* tau_leaf; // leaves x np
  double* t_leaf;   // leaves x np x np
  double* node_r;   // total_nodes x np x np
  double* node_y;   // tree_nodes x (arity-1) x np x np
  double* node_tau; // tree_nodes x np
  double* node_t;   // tree_nodes x np x np
  double* signs;    // np
  int* counters;    // tree_nodes * kMaxColBlocks
  int* status;      // 1
};

// One factorization of a batch, as the batched kernels read it from device memory.
struct __align__(64) BatchItem {
  CUtensorMap mapA;  // A, or its staged copy
  CUtensorMap mapV;  // reflector storage
  Plan plan;
  Store store;
  void* R;           // n x n, leading dimension ldr (double, or float with FP32 storage)
  int64_t ldr;
  void* Q;           // thin Q output of the batched form-Q, leading dimension ldq
  int64_t ldq;
  const float* A32;  // FP32 storage: A (leading dimension lda32), widened into V before the factor
  int64_t lda32;
  int box_rows;
};
// Block b of a batched launch works on chain `chain` (or tree node `chain` of a level) of item.
struct BatchWork {
  int item;
  int chain;
  int level;  // tree level of a form-Q tree step (unused for chain work)
};

// ---------------------------------------------------------------------------------------------
// Shared-memory tile in the layout TMA writes with CU_TENSOR_MAP_SWIZZLE_128B and 16-double
// (128-byte) inner boxes: the columns are split into panels of 16; a panel holds rows_cap rows
// of 128 bytes; inside a row the 16-byte chunk index is XORed with (row & 7).  Both a warp
// reading 32 consecutive columns of one row and a warp reading one column of 32 consecutive
// rows are then free of bank conflicts beyond 2-way.  base must be 1024-byte aligned.
struct Tile {
  char* base;
  int rows_cap;
  __device__ __forceinline__ double* ptr(int r, int c) const {
    uint32_t off = (uint32_t)(c >> 4) * (uint32_t)rows_cap * 128u + (uint32_t)r * 128u +
                   (((((uint32_t)c & 15u) >> 1) ^ ((uint32_t)r & 7u)) << 4) + (((uint32_t)c & 1u) << 3);
    return reinterpret_cast<double*>(base + off);
  }
  __device__ __forceinline__ double& operator()(int r, int c) const { return *ptr(r, c); }
};

// ---------------------------------------------------------------------------------------------
// PTX wrappers: mbarrier, TMA tensor loads/stores, proxy fences.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Invalidates an mbarrier with no operation pending, so its shared memory can take other uses.
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of the barrier for at most ~`cycles` SM clocks; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long cycles) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > cycles) return false;
  }
  return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(x),
               "r"(y), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void tma_store_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void tma_store_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void tma_store_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// About one second at GB300 clocks: no TMA copy of a few hundred KB legitimately takes longer.
constexpr long long kWaitCycles = 2000000000LL;

// Loads rows [row0, row0 + rows) of a row-major matrix described by `map` (box 16 x box_rows)
// into tile rows [dst_row, dst_row + rows) of all np/16 panels, then waits (bounded).  Rows
// past the matrix's end and columns past n arrive as zeros.  Call from all threads; returns
// false in every thread if the copy did not complete in time (the status word is then set).
__device__ inline bool tile_load(const Tile& t, const CUtensorMap* map, uint64_t* bar, uint32_t& phase,
                                 int np, int64_t row0, int rows, int dst_row, int box_rows, int* status,
                                 int* flag) {
  fence_proxy_async_smem();  // order this thread's earlier shared-memory writes before the copy
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t bytes = (uint32_t)rows * (uint32_t)np * 8u;
    mbar_arrive_expect_tx(bar, bytes);
    for (int pnl = 0; pnl < np / 16; ++pnl)
      for (int r = 0; r < rows; r += box_rows)
        tma_load_2d(t.base + (size_t)pnl * t.rows_cap * 128 + (size_t)(dst_row + r) * 128, map, bar, pnl * 16,
                    (int)(row0 + r));
    const bool ok = mbar_wait_bounded(bar, phase, kWaitCycles);
    *flag = ok ? 0 : 1;
    if (!ok) {
      atomicOr(status, kStatusTimeout);
      mbar_wait_bounded(bar, phase, kWaitCycles);  // give the copy in flight one more bounded chance
    }
  }
  phase ^= 1u;
  __syncthreads();
  return *flag == 0;
}

// tile_load split in two, so that other loads can proceed while the copy is in flight: start
// issues it (all threads call; it synchronises the block first), finish waits for it (all
// threads call; false in every thread on timeout, with the status word set).
__device__ inline void tile_load_start(const Tile& t, const CUtensorMap* map, uint64_t* bar, int np, int64_t row0,
                                       int rows, int dst_row, int box_rows) {
  fence_proxy_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, (uint32_t)rows * (uint32_t)np * 8u);
    for (int pnl = 0; pnl < np / 16; ++pnl)
      for (int r = 0; r < rows; r += box_rows)
        tma_load_2d(t.base + (size_t)pnl * t.rows_cap * 128 + (size_t)(dst_row + r) * 128, map, bar, pnl * 16,
                    (int)(row0 + r));
  }
}
__device__ inline bool tile_load_finish(uint64_t* bar, uint32_t& phase, int* status, int* flag) {
  if (threadIdx.x == 0) {
    const bool ok = mbar_wait_bounded(bar, phase, kWaitCycles);
    *flag = ok ? 0 : 1;
    if (!ok) {
      atomicOr(status, kStatusTimeout);
      mbar_wait_bounded(bar, phase, kWaitCycles);  // give the copy in flight one more bounded chance
    }
  }
  phase ^= 1u;
  __syncthreads();
  return *flag == 0;
}

// Stores tile rows [src_row, src_row + rows) to matrix rows [row0, row0 + rows) (TMA clips
// rows and columns outside the matrix).  Call after the tile is final; all threads.
__device__ inline void tile_store(const Tile& t, const CUtensorMap* map, int np, int64_t row0, int rows, int src_row,
                                  int box_rows) {
  fence_proxy_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int pnl = 0; pnl < np / 16; ++pnl)
      for (int r = 0; r < rows; r += box_rows)
        tma_store_2d(map, t.base + (size_t)pnl * t.rows_cap * 128 + (size_t)(src_row + r) * 128, pnl * 16,
                     (int)(row0 + r));
    tma_store_commit();
  }
}
// Before shared rows handed to tile_store are overwritten: the TMA engine has read them.
__device__ inline void tile_store_drain() {
  if (threadIdx.x == 0) tma_store_wait_read();
  __syncthreads();
}

// Sum over the block, returned to every thread.  red holds >= kThreads/32 doubles; the sum is
// taken in a fixed order so every thread gets the same bits.
__device__ inline double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) s += red[w];
  return s;
}

}  // namespace tsqr
