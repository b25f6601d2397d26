// Thin Q of an FP32-storage factorization with the compact-WY products on the tensor cores.
//
// Per chain leaf (V = [I; Y], Algorithm 2's reflectors): M = T C and Q_rows = -Y M, then
// C -= M (Sec. 4.1: Q is applied as a broadcast down the tree, leaf by leaf).  M = T C feeds the
// recurrence C -= M along the whole chain and runs on the FP32 pipe; Q_rows = -Y M, the
// (<= 128) x 64 x 64 contraction that holds 2hn^2 of the leaf's flops and feeds nothing
// forward, runs on the tensor cores.  Each FP32 operand value a is split into three bf16 terms,
//   a1 = bf16(a),  a2 = bf16(a - a1),  a3 = bf16(a - a1 - a2),
// where each difference is exact in FP32 and a1 + a2 + a3 carries a's 24 significant bits.  The
// six term products whose weight is 2^-16 of the leading one or more (s + t <= 4) accumulate in
// one FP32 TMEM accumulator through tcgen05.mma kind::f16 (bf16 inputs, FP32 accumulation, M =
// 128, N = 64, K = 16); the dropped products weigh below 2^-24.  The result has FP32-level
// accuracy, the bar of the FP32 storage form.  The first leaf of a chain (V unit lower
// trapezoidal) is computed on the FP32 pipe.  Needs np = 64 and h <= 128.
//
// One block of 256 threads per chain, one SM each (about 190 KB of shared memory); 64 TMEM
// columns.  The leaf's T arrives by a bulk copy and its reflector tile by TMA, both issued when
// the leaf starts; every wait is bounded and the block frees its TMEM on every exit path.
#include "../../include/tsqr.h"
#include "bf16x3_pass.cuh"
#include "factor_kernels.h"

namespace tsqr {
namespace {

using namespace bf3;

// Chain g of one factorization (the body of formq_bf16x3_kernel and of its batched form).
// first_only: only the chain's first leaf, with the block C entering it read from node_r[g]
// (written there by formq_f32_recur_kernel after the chain's other leaves), also without a tree.
__device__ __forceinline__ void formq_bf16x3_chain(const CUtensorMap* mapV_p, const Plan& P, const Store& st,
                                                   float* __restrict__ Q, int64_t ldq, int box_rows, int g,
                                                   char* smem_raw, bool first_only = false) {
  Tc3Smem z = carve_tc3(smem_raw, P.h);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int np = 64, n = P.n, h = P.h;
  if (tid == 0) {
    for (int b = 0; b < 3; ++b) mbar_init(z.bars + b, 1);
    fence_mbar_init();
    *z.flag = 0;
  }
  if (warp == 0) oz::tmem_alloc(z.slot, kTmemCols3);
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  const uint32_t tmem = *z.slot;
  uint32_t mma_phase = 0, y_phase = 0, t_phase = 0;
  // C = this chain's block of Q_tree [D; 0]
  const f32x2* blocks = reinterpret_cast<const f32x2*>(st.node_r);
  for (int i = tid; i < np * np; i += kT3) {
    const int a = i >> 6, b = i & 63;
    z.C[a * kLd + b] = (P.depth == 0 && !first_only) ? ((a == b && a < n) ? (float)__ldcg(st.signs + a) : 0.f)
                                                     : blocks[(size_t)g * np * np + i].hi;
  }
  __syncthreads();
  // rows h..127 of the A terms stay zero (the MMA reads 128 rows; only the first leaf, which is
  // processed last, reuses the buffers as scratch)
  if (h < 128) zero_a_rows(z.a, h);
  const int64_t l0 = chain_first_leaf(P, g), l1 = first_only ? l0 + 1 : chain_end_leaf(P, g);
  bool alive = true;
  for (int64_t leaf = l1 - 1; leaf >= l0 && alive; --leaf) {
    const int64_t row0 = leaf * h;
    const int rows_valid = (int)((P.m - row0 < h) ? (P.m - row0) : h);
    const f32x2* Tg = reinterpret_cast<const f32x2*>(st.t_leaf) + leaf * np * np;
    if (leaf != l0) {
      // ---- both loads of the leaf start now: T by a bulk copy, the reflector tile by TMA
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        mbar_arrive_expect_tx(z.bars + 2, np * np * 8);
        bulk_copy(z.T, Tg, np * np * 8, z.bars + 2);
        mbar_arrive_expect_tx(z.bars + 0, (uint32_t)h * np * 8);
        for (int pnl = 0; pnl < np / 16; ++pnl)
          for (int r = 0; r < h; r += box_rows)
            tma_load_2d(z.Y.base + (size_t)pnl * h * 128 + (size_t)r * 128, mapV_p, z.bars + 0, pnl * 16,
                        (int)(row0 + r));
      }
      // ---- M = T C on the FP32 pipe (T upper triangular).  M feeds C -= M, which carries the
      //      chain from leaf to leaf, so it takes FP32 rounding rather than the tensor cores'
      //      accumulation; the rows of Q below do not feed forward.
      {
        const bool ok = wait_all(z, z.bars + 2, t_phase, st.status);
        t_phase ^= 1u;
        if (!ok) {
          alive = false;
          break;
        }
      }
      for (int o = tid; o < np * np; o += kT3) {
        const int a = o >> 6, b = o & 63;
        float v = 0.f;
        for (int p = a; p < n; ++p) v = __fmaf_rn(z.T[a * np + p].hi, z.C[p * kLd + b], v);
        z.M[a * kLd + b] = v;
      }
      __syncthreads();
      for (int i = tid; i < np * np; i += kT3) {
        const int o = (i >> 6) * kLd + (i & 63);
        z.C[o] = __fsub_rn(z.C[o], z.M[o]);
      }
      // ---- Q_rows = -Y M: B = M, A = Y (rows h.. zero)
      write_terms(z.b, kTermB, np, [&](int j, int k) { return z.M[k * kLd + j]; });
      {
        const bool ok = wait_all(z, z.bars + 0, y_phase, st.status);
        y_phase ^= 1u;
        if (!ok) {
          alive = false;
          break;
        }
      }
      write_terms(z.a, kTermA, h, [&](int r, int k) { return yv(z.Y, r, k); });
      if (!mma_terms(z, tmem, mma_phase, st.status)) {
        alive = false;
        break;
      }
      epilogue(tmem, rows_valid, [&](int i, int j, float v) {
        if (j < n) Q[gidx(P, row0 + i, j, ldq)] = -v;
      });
    } else {
      // ---- first leaf on the FP32 pipe: Q_rows = [C; 0] - V (T (V_top^T C))
      float* T = reinterpret_cast<float*>(z.a);  // the A terms are free here
      float* X = T + np * np;
      for (int i = tid; i < np * np; i += kT3) T[i] = Tg[i].hi;
      if (!tile_load(z.Y, mapV_p, z.bars, y_phase, np, row0, h, 0, box_rows, st.status, z.flag)) {
        alive = false;
        break;
      }
      for (int o = tid; o < np * np; o += kT3) {
        const int a = o >> 6, b = o & 63;
        float v = 0.f;
        if (a < n) {
          v = z.C[a * kLd + b];
          for (int r = a + 1; r < n; ++r) v = __fmaf_rn(yv(z.Y, r, a), z.C[r * kLd + b], v);
        }
        X[a * np + b] = v;
      }
      __syncthreads();
      for (int o = tid; o < np * np; o += kT3) {  // M = T X, T upper triangular
        const int a = o >> 6, b = o & 63;
        float v = 0.f;
        for (int p = a; p < n; ++p) v = __fmaf_rn(T[a * np + p], X[p * np + b], v);
        z.M[a * kLd + b] = v;
      }
      __syncthreads();
      constexpr int G = kT3 / 64;
      const int cown = tid & 63, gown = tid >> 6;
      if (cown < n) {
        for (int r = gown; r < rows_valid; r += G) {
          float acc = 0.f;
          const int amax = (r < n) ? r : n;
          for (int a = 0; a < amax; ++a) acc = __fmaf_rn(yv(z.Y, r, a), z.M[a * kLd + cown], acc);
          if (r < n) acc = __fadd_rn(acc, z.M[r * kLd + cown]);
          float v = -acc;
          if (r < n) v = __fadd_rn(v, z.C[r * kLd + cown]);
          Q[gidx(P, row0 + r, cown, ldq)] = v;
        }
      }
      __syncthreads();
    }
  }
  // after a timeout, give the copies and MMAs in flight one more bounded wait before TMEM is freed
  if (!alive && tid == 0) {
    oz::wait_bar(z.bars + 1, mma_phase);
    oz::wait_bar(z.bars + 0, y_phase);
    oz::wait_bar(z.bars + 2, t_phase);
  }
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  if (warp == 0) oz::tmem_dealloc(tmem, kTmemCols3);
}

// split: the chain's other leaves were taken by the recurrence and leaf-product kernels
// (formq_f32_phases.cu), so only its first leaf is left here (a chain that holds a short last
// leaf is taken whole).
__global__ void __launch_bounds__(kT3, 1)
    formq_bf16x3_kernel(const __grid_constant__ CUtensorMap mapV, const Plan P, const Store st, float* __restrict__ Q,
                        int64_t ldq, int box_rows, bool split) {
  extern __shared__ char smem_raw[];
  const int g = blockIdx.x;
  formq_bf16x3_chain(&mapV, P, st, Q, ldq, box_rows, g, smem_raw, split && !formq_chain_short(P, g));
}

__global__ void __launch_bounds__(kT3, 1)
    formq_bf16x3_batched_kernel(const BatchItem* __restrict__ items, const BatchWork* __restrict__ work) {
  extern __shared__ char smem_raw[];
  const BatchWork w = work[blockIdx.x];
  const BatchItem& it = items[w.item];
  formq_bf16x3_chain(&it.mapV, it.plan, it.store, static_cast<float*>(it.Q), it.ldq, it.box_rows, w.chain, smem_raw);
}

}  // namespace

size_t formq_bf16x3_smem_bytes(const Plan& P) {
  const size_t ybytes = ((size_t)P.h * 64 * 8 + 1023) & ~size_t(1023);
  return 1024 + ybytes + 3 * kTermA + 3 * kTermB + 64 * 64 * 8 + 2 * 64 * kLd * 4 + 3 * 8 + 8 + 16;
}

bool bf16x3_form_q_applies(const Plan& P) { return P.precision == kPrecF32 && P.np == 64 && P.h <= 128; }

cudaError_t prepare_formq_bf16x3_batched(size_t smem) {
  return cudaFuncSetAttribute(formq_bf16x3_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_formq_bf16x3_batched(const BatchItem* items, const BatchWork* work, int blocks, size_t smem,
                                        cudaStream_t stream) {
  formq_bf16x3_batched_kernel<<<blocks, kT3, smem, stream>>>(items, work);
  return cudaGetLastError();
}

cudaError_t launch_formq_bf16x3_chains(const CUtensorMap& mapV, const Plan& P, const Store& st, float* Q, int64_t ldq,
                                       int box_rows, cudaStream_t stream) {
  // the chains' recurrences (M = T C of every leaf but the first, into Q; the block entering the
  // first leaf into node_r), then the first leaves, then the other leaves' products -Y M
  cudaError_t e = launch_formq_f32_recur(P, st, Q, ldq, stream);
  if (e != cudaSuccess) return e;
  const size_t smem = formq_bf16x3_smem_bytes(P);
  e = cudaFuncSetAttribute(formq_bf16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  formq_bf16x3_kernel<<<P.chains, kT3, smem, stream>>>(mapV, P, st, Q, ldq, box_rows, true);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_formq_bf16x3_leaves(P, st, Q, ldq, stream);
}

}  // namespace tsqr
