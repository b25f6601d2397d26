// Shared pieces of the FP32-storage kernels that run compact-WY products on the tensor cores as
// bf16x3 term products: each FP32 operand value a is split into three bf16 terms,
//   a1 = bf16(a),  a2 = bf16(a - a1),  a3 = bf16(a - a1 - a2),
// each difference exact in FP32, and the six term products of weight >= 2^-16 of the leading one
// (s + t <= 4) accumulate in one FP32 TMEM accumulator through tcgen05.mma kind::f16 (bf16 in,
// FP32 accumulation, M = 128, N = 64, K = 16).  The dropped products weigh below 2^-24.
// A 256-thread block, one accumulator of 64 TMEM columns.  Used by the thin Q
// (formq_bf16x3.cu) and by Q^T B / Q B (apply_bf16x3.cu).
#pragma once

#include <cuda_bf16.h>

#include "arith.cuh"
#include "ozaki.cuh"

namespace tsqr {
namespace bf3 {

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

// D (128 x 64, TMEM) = sum over the six term pairs of A_s B_t (added to D with accumulate).  The
// terms must be written; all threads call.  False on timeout.
__device__ inline bool mma_terms(const Tc3Smem& z, uint32_t tmem, uint32_t& phase, int* status,
                                 bool accumulate = false) {
  fence_proxy_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    oz::fence_after_sync();
    const uint32_t idesc = oz::idesc_bf16(128, 64);
    // smallest terms first: (3,1) (2,2) (1,3) (2,1) (1,2) (1,1)
    const int sa[6] = {2, 1, 0, 1, 0, 0}, sb[6] = {0, 1, 2, 0, 1, 0};
    uint32_t acc = accumulate ? 1u : 0u;
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

}  // namespace bf3
}  // namespace tsqr
