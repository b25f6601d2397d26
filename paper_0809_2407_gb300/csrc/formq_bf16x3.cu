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
#include <cuda_bf16.h>

#include "../../include/tsqr.h"
#include "arith.cuh"
#include "factor_kernels.h"
#include "ozaki.cuh"

namespace tsqr {
namespace {

constexpr int kT3 = 256;
constexpr int kLd = 65;
constexpr uint32_t kTermA = 128 * 64 * 2;  // one A term: 128 rows x 64 k of bf16, 16 KB
constexpr uint32_t kTermB = 64 * 64 * 2;   // one B term: 64 rows x 64 k, 8 KB
constexpr uint32_t kTmemCols3 = 64;

struct Tc3Smem {
  Tile Y;          // h x 64 leaf tile (8-byte slots, the FP32 value in the low half)
  char* a;         // 3 A terms
  char* b;         // 3 B terms
  f32x2* T;        // 64 x 64 slots (bulk copy of the leaf's T)
  float* C;        // 64 x 65
  float* M;        // 64 x 65
  uint64_t* bars;  // 0: Y tile, 1: MMA commit, 2: T
  uint32_t* slot;  // TMEM base address
  int* flag;
};

__device__ inline Tc3Smem carve_tc3(char* raw, int h) {
  Tc3Smem z;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  const size_t ybytes = ((size_t)h * 64 * 8 + 1023) & ~size_t(1023);
  z.Y = Tile{base, h};
  z.a = base + ybytes;
  z.b = z.a + 3 * kTermA;
  z.T = reinterpret_cast<f32x2*>(z.b + 3 * kTermB);
  z.C = reinterpret_cast<float*>(z.T + 64 * 64);
  z.M = z.C + 64 * kLd;
  z.bars = reinterpret_cast<uint64_t*>(z.M + 64 * kLd);  // 8-byte aligned: C and M are 2 * 64 * 65 floats
  z.slot = reinterpret_cast<uint32_t*>(z.bars + 3);
  z.flag = reinterpret_cast<int*>(z.slot + 2);
  return z;
}

// The three bf16 terms of a, as raw 16-bit patterns.
__device__ __forceinline__ void split3(float a, uint32_t t[3]) {
  const __nv_bfloat16 b1 = __float2bfloat16_rn(a);
  const float r1 = __fsub_rn(a, __bfloat162float(b1));
  const __nv_bfloat16 b2 = __float2bfloat16_rn(r1);
  const float r2 = __fsub_rn(r1, __bfloat162float(b2));
  const __nv_bfloat16 b3 = __float2bfloat16_rn(r2);
  t[0] = __bfloat16_as_ushort(b1);
  t[1] = __bfloat16_as_ushort(b2);
  t[2] = __bfloat16_as_ushort(b3);
}

// Writes the three terms of the (rows x 64) operand val(r, k) into the 128-byte swizzled K-major
// buffers base + s * term_bytes (two k per 32-bit store).  All threads call.
template <class Val>
__device__ inline void write_terms(char* base, uint32_t term_bytes, int rows, Val val) {
  for (int idx = threadIdx.x; idx < rows * 32; idx += kT3) {
    const int r = idx >> 5, k = (idx & 31) * 2;
    uint32_t t0[3], t1[3];
    split3(val(r, k), t0);
    split3(val(r, k + 1), t1);
    const uint32_t off = oz::op_off(r, k);
#pragma unroll
    for (int s = 0; s < 3; ++s) *reinterpret_cast<uint32_t*>(base + s * term_bytes + off) = t0[s] | (t1[s] << 16);
  }
}

// Rows r0..127 of the three A terms set to zero (the MMA reads all 128 rows).
__device__ inline void zero_a_rows(char* a, int r0) {
  const int per = (128 - r0) * 8;  // 16-byte chunks per term
  for (int i = threadIdx.x; i < 3 * per; i += kT3) {
    const int s = i / per, rem = i % per;
    *reinterpret_cast<uint4*>(a + s * kTermA + (size_t)(r0 + rem / 8) * 128 + (rem % 8) * 16) = make_uint4(0, 0, 0, 0);
  }
}

// Thread 0 waits (bounded) for a barrier phase; every thread learns the outcome.
__device__ inline bool wait_all(const Tc3Smem& z, uint64_t* bar, uint32_t parity, int* status) {
  if (threadIdx.x == 0 && !oz::wait_bar(bar, parity)) {
    atomicOr(status, kStatusTimeout);
    *z.flag = 1;
  }
  __syncthreads();
  return *z.flag == 0;
}

// D (128 x 64, TMEM) = sum over the six term pairs of A_s B_t.  The terms must be written; all
// threads call.  False on timeout.
__device__ inline bool mma_terms(const Tc3Smem& z, uint32_t tmem, uint32_t& phase, int* status) {
  fence_proxy_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    oz::fence_after_sync();
    const uint32_t idesc = oz::idesc_bf16(128, 64);
    // smallest terms first: (3,1) (2,2) (1,3) (2,1) (1,2) (1,1)
    const int sa[6] = {2, 1, 0, 1, 0, 0}, sb[6] = {0, 1, 2, 0, 1, 0};
    uint32_t acc = 0;
    for (int p = 0; p < 6; ++p) {
      const uint64_t ad = oz::sw128_desc(smem_u32(z.a + sa[p] * kTermA));
      const uint64_t bd = oz::sw128_desc(smem_u32(z.b + sb[p] * kTermB));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {  // K step of 16 bf16 = 32 bytes = 2 descriptor units
        oz::mma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, idesc, acc);
        acc = 1;
      }
    }
    oz::mma_commit(z.bars + 1);
  }
  const bool ok = wait_all(z, z.bars + 1, phase, status);
  phase ^= 1u;
  oz::fence_after_sync();
  return ok;
}

// Reads the accumulator back: out(i, j, value) for rows i < rows, columns 0..63.  Warp w reads
// TMEM lanes 32 (w & 3).. and columns 32 (w >> 2)..; all threads call.
template <class Out>
__device__ inline void epilogue(uint32_t tmem, int rows, Out out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, c0 = 32 * (warp >> 2);
  if (32 * q < rows) {
    uint32_t v[32];
    oz::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
    oz::tmem_wait_ld();
    const int i = 32 * q + lane;
    if (i < rows) {
#pragma unroll
      for (int c = 0; c < 32; ++c) out(i, c0 + c, __uint_as_float(v[c]));
    }
  }
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ float yv(const Tile& Y, int r, int c) {
  return reinterpret_cast<const f32x2*>(Y.ptr(r, c))->hi;
}

__global__ void __launch_bounds__(kT3, 1)
    formq_bf16x3_kernel(const __grid_constant__ CUtensorMap mapV, const Plan P, const Store st, float* __restrict__ Q,
                        int64_t ldq, int box_rows) {
  extern __shared__ char smem_raw[];
  Tc3Smem z = carve_tc3(smem_raw, P.h);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int np = 64, n = P.n, h = P.h;
  const int g = blockIdx.x;
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
    z.C[a * kLd + b] = (P.depth == 0) ? ((a == b && a < n) ? (float)__ldcg(st.signs + a) : 0.f)
                                      : blocks[(size_t)g * np * np + i].hi;
  }
  __syncthreads();
  // rows h..127 of the A terms stay zero (the MMA reads 128 rows; only the first leaf, which is
  // processed last, reuses the buffers as scratch)
  if (h < 128) zero_a_rows(z.a, h);
  const int64_t l0 = chain_first_leaf(P, g), l1 = chain_end_leaf(P, g);
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
            tma_load_2d(z.Y.base + (size_t)pnl * h * 128 + (size_t)r * 128, &mapV, z.bars + 0, pnl * 16,
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
      if (!tile_load(z.Y, &mapV, z.bars, y_phase, np, row0, h, 0, box_rows, st.status, z.flag)) {
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

}  // namespace

size_t formq_bf16x3_smem_bytes(const Plan& P) {
  const size_t ybytes = ((size_t)P.h * 64 * 8 + 1023) & ~size_t(1023);
  return 1024 + ybytes + 3 * kTermA + 3 * kTermB + 64 * 64 * 8 + 2 * 64 * kLd * 4 + 3 * 8 + 8 + 16;
}

bool bf16x3_form_q_applies(const Plan& P) { return P.precision == kPrecF32 && P.np == 64 && P.h <= 128; }

cudaError_t launch_formq_bf16x3_chains(const CUtensorMap& mapV, const Plan& P, const Store& st, float* Q, int64_t ldq,
                                       int box_rows, cudaStream_t stream) {
  const size_t smem = formq_bf16x3_smem_bytes(P);
  cudaError_t e = cudaFuncSetAttribute(formq_bf16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  formq_bf16x3_kernel<<<P.chains, kT3, smem, stream>>>(mapV, P, st, Q, ldq, box_rows);
  return cudaGetLastError();
}

}  // namespace tsqr
