// TSQR factorization kernels: leaves, flat chains and the tree over thread blocks, in one launch
// (the schedule is in factor_chain.cuh), with the flat-tree step on the FP64 (or FP32) pipe.  In
// the Ozaki WY form (mode 2) the 64-column step takes the Gram entries of its T on the tensor
// cores (gram_tc.cuh); everything else, and R bit for bit, is the plain step's.  The double-float
// step (modes 1 and 3) keeps them in its column loop: there the loop is bound by latency, not by
// the FP32 pipe, so the extra dot products cost little and the serial tensor-core pass after the
// loop cost more (factor at m = 2^22, n = 64: 39.6 ms with the loop's Gram, 46.7 ms without).
#include <algorithm>

#include "factor_kernels.h"
#include "factor_chain.cuh"

namespace tsqr {

size_t factor_smem_bytes(const Plan& P) {
  return 1024 + (size_t)P.rows_cap * P.np * 8 + (size_t)tri_size(P.np) * 8 + kThreads * 8 + P.np * 8 + 8 * 8 +
         P.np * 8 + 2 * P.np * 8 + (size_t)P.np * P.np / 4 * 8 + 16 + 16;
}

// kTc: the chain steps take their Gram entries on the tensor cores; the block holds 256 TMEM
// columns (two blocks per SM fit) for its lifetime.
template <class Ar, bool kTc>
__global__ void __launch_bounds__(kThreads, 2)
    factor_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapV, const Plan P,
                  const Store st, typename Ar::Out* __restrict__ R_out, int64_t ldr, int box_rows) {
  extern __shared__ char smem_raw[];
  using E = typename Ar::E;
  const FactorSmem<E> f = carve_factor<E>(smem_raw, P);
  if constexpr (!kTc) {
    factor_chain<Ar>(&mapA, &mapV, P, st, R_out, ldr, box_rows, blockIdx.x, f,
                     [](const FactorSmem<E>& ff, const Plan& p) { return chain_step<Ar>(ff, p); });
  } else {
    if (threadIdx.x < 32) oz::tmem_alloc(f.slot, gram::kTmemCols);
    if (threadIdx.x == 0) {
      mbar_init(f.mbar, 1);
      fence_mbar_init();
    }
    oz::fence_before_sync();
    __syncthreads();
    oz::fence_after_sync();
    const uint32_t tmem = *f.slot;
    uint32_t phase = 0;
    const gram::GramTC tc = gram_resources(f, &phase, tmem, st.status);
    factor_chain<Ar>(&mapA, &mapV, P, st, R_out, ldr, box_rows, blockIdx.x, f,
                     [&](const FactorSmem<E>& ff, const Plan& p) { return chain_step<Ar>(ff, p, &tc); });
    oz::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) oz::tmem_dealloc(tmem, gram::kTmemCols);
  }
}

// Many factorizations in one persistent launch: every block takes the next chain from the work
// list (work[k]: chain work[k].chain of item work[k].item, longest chains first) through the
// counter *next until the list is used up.  No block waits for another (the tree above each
// item's chains is climbed by the last arrival), so any number of resident blocks is safe.
template <class Ar>
__global__ void __launch_bounds__(kThreads, 2)
    factor_batched_kernel(const BatchItem* __restrict__ items, const BatchWork* __restrict__ work, int total,
                          int* __restrict__ next) {
  extern __shared__ char smem_raw[];
  __shared__ int k_s;
  for (;;) {
    if (threadIdx.x == 0) k_s = atomicAdd(next, 1);
    __syncthreads();
    const int k = k_s;
    __syncthreads();  // every thread has read k_s before thread 0 takes the next one
    if (k >= total) return;
    const BatchWork w = work[k];
    const BatchItem& it = items[w.item];
    const FactorSmem<typename Ar::E> f = carve_factor<typename Ar::E>(smem_raw, it.plan);
    factor_chain<Ar>(&it.mapA, &it.mapV, it.plan, it.store, static_cast<typename Ar::Out*>(it.R), it.ldr,
                     it.box_rows, w.chain, f,
                     [](const FactorSmem<typename Ar::E>& ff, const Plan& p) { return chain_step<Ar>(ff, p); });
    // a bounded wait that gave up may leave a copy in flight: take no further work
    __syncthreads();
    if (threadIdx.x == 0) k_s = *reinterpret_cast<volatile int*>(it.store.status) & kStatusTimeout;
    __syncthreads();
    const int failed = k_s;
    __syncthreads();  // every thread has read k_s before thread 0 reuses it
    if (failed) return;
    // the next item carves shared memory by its own plan: retire this item's TMA barrier first
    if (threadIdx.x == 0) mbar_inval(f.bar);
  }
}

cudaError_t prepare_factor_batched(int precision, size_t smem) {
  if (prec_df(precision))
    return cudaFuncSetAttribute(factor_batched_kernel<ArithDF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (precision == kPrecF32)
    return cudaFuncSetAttribute(factor_batched_kernel<ArithF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaFuncSetAttribute(factor_batched_kernel<ArithF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <class Ar>
static cudaError_t factor_batched_blocks_t(int total, size_t smem, int* blocks) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, factor_batched_kernel<Ar>, kThreads, smem);
  if (e != cudaSuccess) return e;
  *blocks = std::max(1, std::min(total, std::max(1, per_sm) * sms));
  return cudaSuccess;
}

cudaError_t factor_batched_blocks(int precision, int total, size_t smem, int* blocks) {
  if (prec_df(precision)) return factor_batched_blocks_t<ArithDF>(total, smem, blocks);
  if (precision == kPrecF32) return factor_batched_blocks_t<ArithF32>(total, smem, blocks);
  return factor_batched_blocks_t<ArithF64>(total, smem, blocks);
}

cudaError_t launch_factor_batched(const BatchItem* items, const BatchWork* work, int total, int* next, int blocks,
                                  int precision, size_t smem, cudaStream_t stream) {
  if (prec_df(precision))
    factor_batched_kernel<ArithDF><<<blocks, kThreads, smem, stream>>>(items, work, total, next);
  else if (precision == kPrecF32)
    factor_batched_kernel<ArithF32><<<blocks, kThreads, smem, stream>>>(items, work, total, next);
  else
    factor_batched_kernel<ArithF64><<<blocks, kThreads, smem, stream>>>(items, work, total, next);
  return cudaGetLastError();
}

// FP32 storage in a batch: blocks (x, i) widen item i's A into its reflector storage.
__global__ void stage_widen_batched_kernel(const BatchItem* __restrict__ items) {
  const BatchItem& it = items[blockIdx.y];
  const float* A = it.A32;
  if (A == nullptr) return;
  const int64_t m = it.plan.m, lda = it.lda32, ldv = it.store.ldv;
  const int n = it.plan.n;
  double* V = it.store.v;
  const int64_t total = m * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / n;
    const int c = (int)(i - r * n);
    V[r * ldv + c] = (double)A[r * lda + c];
  }
}

cudaError_t launch_stage_widen_batched(const BatchItem* items, int count, cudaStream_t stream) {
  stage_widen_batched_kernel<<<dim3(16, (unsigned)count), 256, 0, stream>>>(items);
  return cudaGetLastError();
}

template <class Ar, bool kTc>
static cudaError_t launch_factor_k(const CUtensorMap& mapA, const CUtensorMap& mapV, const Plan& P, const Store& st,
                                   void* R_out, int64_t ldr, int box_rows, size_t smem, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(st.counters, 0, sizeof(int) * (size_t)(P.tree_nodes > 0 ? P.tree_nodes : 1), stream);
  if (e != cudaSuccess) return e;
  factor_kernel<Ar, kTc><<<P.chains, kThreads, smem, stream>>>(mapA, mapV, P, st,
                                                               static_cast<typename Ar::Out*>(R_out), ldr, box_rows);
  return cudaGetLastError();
}

// kTcForm: the precision form whose plans take the Gram entries on the tensor cores (where
// gram_tc_applies and at most two blocks share an SM's 512 TMEM columns); -1 for none.
template <class Ar, int kTcForm>
static cudaError_t launch_factor_t(const CUtensorMap& mapA, const CUtensorMap& mapV, const Plan& P, const Store& st,
                                   void* R_out, int64_t ldr, int box_rows, cudaStream_t stream) {
  const size_t smem = factor_smem_bytes(P);
  cudaError_t e = cudaFuncSetAttribute(factor_kernel<Ar, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if constexpr (kTcForm >= 0) {
    if (P.precision == kTcForm && gram_tc_applies(P)) {
      e = cudaFuncSetAttribute(factor_kernel<Ar, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, factor_kernel<Ar, true>, kThreads, smem);
      if (e != cudaSuccess) return e;
      if (per_sm * (int)gram::kTmemCols <= 512)
        return launch_factor_k<Ar, true>(mapA, mapV, P, st, R_out, ldr, box_rows, smem, stream);
    }
  }
  return launch_factor_k<Ar, false>(mapA, mapV, P, st, R_out, ldr, box_rows, smem, stream);
}

// Copies A (m x n, leading dimension lda) into V (leading dimension ldv): the staging step for
// an A whose row stride or address TMA cannot take (odd lda, or not 16-byte aligned).
__global__ void stage_copy_kernel(const double* __restrict__ A, int64_t lda, double* __restrict__ V, int64_t ldv,
                                  int64_t m, int n) {
  const int64_t total = m * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / n;
    const int c = (int)(i - r * n);
    V[r * ldv + c] = A[r * lda + c];
  }
}

cudaError_t launch_stage_copy(const double* A, int64_t lda, double* V, int64_t ldv, int64_t m, int n,
                              cudaStream_t stream) {
  stage_copy_kernel<<<152 * 8, 256, 0, stream>>>(A, lda, V, ldv, m, n);
  return cudaGetLastError();
}

// FP32 storage: A (float, m x n, leading dimension lda) widened exactly into V's 8-byte slots, from
// which the factorization loads its tiles as for FP64 input.
__global__ void stage_widen_kernel(const float* __restrict__ A, int64_t lda, double* __restrict__ V, int64_t ldv,
                                   int64_t m, int n) {
  const int64_t total = m * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / n;
    const int c = (int)(i - r * n);
    V[r * ldv + c] = (double)A[r * lda + c];
  }
}

cudaError_t launch_stage_widen(const float* A, int64_t lda, double* V, int64_t ldv, int64_t m, int n,
                               cudaStream_t stream) {
  stage_widen_kernel<<<152 * 8, 256, 0, stream>>>(A, lda, V, ldv, m, n);
  return cudaGetLastError();
}

// Column-major A (element (i, j) at A[j * lda + i]) staged into V's row-major 8-byte slots,
// through 32 x 32 shared tiles so that both the reads (down columns) and the writes (along rows)
// are coalesced; FP32 input is widened.
template <class T>
__global__ void stage_transpose_kernel(const T* __restrict__ A, int64_t lda, double* __restrict__ V, int64_t ldv,
                                       int64_t m, int n) {
  __shared__ double tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  const int c0 = blockIdx.y * 32;
  for (int64_t r0 = (int64_t)blockIdx.x * 32; r0 < m; r0 += (int64_t)gridDim.x * 32) {
    for (int cc = ty; cc < 32; cc += 8) {  // read: lanes along the rows of column c0 + cc
      const int64_t r = r0 + tx;
      const int c = c0 + cc;
      tile[cc][tx] = (r < m && c < n) ? (double)A[(int64_t)c * lda + r] : 0.0;
    }
    __syncthreads();
    for (int rr = ty; rr < 32; rr += 8) {  // write: lanes along the columns of row r0 + rr
      const int64_t r = r0 + rr;
      const int c = c0 + tx;
      if (r < m && c < n) V[r * ldv + c] = tile[tx][rr];
    }
    __syncthreads();
  }
}

cudaError_t launch_stage_transpose(const void* A, bool f32, int64_t lda, double* V, int64_t ldv, int64_t m, int n,
                                   cudaStream_t stream) {
  const dim3 grid(152 * 4, (unsigned)((n + 31) / 32));
  if (f32)
    stage_transpose_kernel<float><<<grid, 256, 0, stream>>>(static_cast<const float*>(A), lda, V, ldv, m, n);
  else
    stage_transpose_kernel<double><<<grid, 256, 0, stream>>>(static_cast<const double*>(A), lda, V, ldv, m, n);
  return cudaGetLastError();
}

cudaError_t launch_factor(const CUtensorMap& mapA, const CUtensorMap& mapV, const Plan& P, const Store& st,
                          void* R_out, int64_t ldr, int box_rows, cudaStream_t stream) {
  if (blocked_factor_applies(P)) return launch_factor_blocked(mapA, mapV, P, st, R_out, ldr, box_rows, stream);
  if (prec_df(P.precision))
    return launch_factor_t<ArithDF, -1>(mapA, mapV, P, st, R_out, ldr, box_rows, stream);
  if (P.precision == kPrecF32) return launch_factor_t<ArithF32, -1>(mapA, mapV, P, st, R_out, ldr, box_rows, stream);
  return launch_factor_t<ArithF64, kPrecOzaki>(mapA, mapV, P, st, R_out, ldr, box_rows, stream);
}

}  // namespace tsqr
