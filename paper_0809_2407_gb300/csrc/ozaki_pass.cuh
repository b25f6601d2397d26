// Shared pieces of the kernels that run compact-WY products on the tensor cores as Ozaki splits
// (ozaki.cuh): the shared-memory layout of a 512-thread block, the digit slices of the operands,
// one product of 34 digit pairs into the eight TMEM group accumulators, and the int64 epilogue.
// Used by the thin-Q kernel (apply.cu) and by the Q^T B / Q B chain kernel (apply_ozaki.cu).
// slice_pair (the 7-bit form) serves the factorization's Gram entries and blocked step.
#pragma once

#include "arith.cuh"
#include "ozaki.cuh"

namespace tsqr {

constexpr int kOzT = 512;
static constexpr int kOzLd = 65;

struct OzSmem {
  Tile Y;           // h x 64 FP64 leaf tile (TMA); converted in place to fixed point
  char* bsl;        // 8 B slices, 8 KB each; FP64 scratch (T, X) for the first leaf
  char* asl;        // 2 A slice buffers, 16 KB each
  double* C;        // 64 x 65
  double* M;        // 64 x 65; the leaf's T (64 x 64, bulk copy) then its fixed-point form
  int* expA;        // 128
  int* expB;        // 64
  uint64_t* bars;   // 0: Y tile, 1: A buffer 0, 2: A buffer 1, 3: T
  uint32_t* slot;   // TMEM base address
  int* flag;
};

__device__ inline OzSmem carve_ozaki(char* raw, int h) {
  OzSmem z;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  const size_t ybytes = ((size_t)h * 64 * 8 + 1023) & ~size_t(1023);
  z.Y = Tile{base, h};
  z.bsl = base + ybytes;
  z.asl = z.bsl + 8 * oz::kBSliceBytes;
  z.C = reinterpret_cast<double*>(z.asl + 2 * oz::kASliceBytes);
  z.M = z.C + 64 * kOzLd;
  z.expA = reinterpret_cast<int*>(z.M + 64 * kOzLd);
  z.expB = z.expA + 128;
  z.bars = reinterpret_cast<uint64_t*>(z.expB + 64);
  z.slot = reinterpret_cast<uint32_t*>(z.bars + 4);
  z.flag = reinterpret_cast<int*>(z.slot + 2);
  return z;
}

// bf16 bits of slices s of two fixed-point values, packed low|high: the 7-bit integer is made an
// exact FP32 by the 2^23 magic add, whose upper 16 bits are its bf16 form.
__device__ __forceinline__ uint32_t slice_pair(uint64_t f0, uint64_t f1, int s) {
  const uint32_t c0 = (uint32_t)(f0 >> (56 - 7 * s)) & 127u;
  const uint32_t c1 = (uint32_t)(f1 >> (56 - 7 * s)) & 127u;
  const float x0 = __fsub_rn(__int_as_float(0x4B000000 | c0), 8388608.f);
  const float x1 = __fsub_rn(__int_as_float(0x4B000000 | c1), 8388608.f);
  const uint32_t sg = ((uint32_t)(f0 >> 48) & 0x8000u) | ((uint32_t)(f1 >> 32) & 0x80000000u);
  return __byte_perm(__float_as_uint(x0), __float_as_uint(x1), 0x7632) | sg;
}

// *dst = max(*dst, e over the warp), for a full warp whose lanes all target dst (the callers'
// index idx >> 6 is the same across 32 consecutive idx): one shared atomic per warp.
__device__ __forceinline__ void warp_max_into(int* dst, int e) {
  const int m = __reduce_max_sync(0xffffffffu, e);
  if ((threadIdx.x & 31) == 0) atomicMax(dst, m);
}

// Waits (thread 0, bounded) for a barrier phase; every thread learns the outcome.
__device__ inline bool oz_wait_all(const OzSmem& z, uint64_t* bar, uint32_t parity, int* status) {
  if (threadIdx.x == 0 && !oz::wait_bar(bar, parity)) {
    atomicOr(status, kStatusTimeout);
    *z.flag = 1;
  }
  __syncthreads();
  return *z.flag == 0;
}

// One Ozaki product D (128 x 64) = A (a_rows x 64) B (64 x 64) in the digit form of the split
// (ozaki.cuh) into the 8 TMEM groups.  The B digit slices (and the eighth, zero) must be in z.bsl
// and rows a_rows..127 of both A buffers zero; afix(r, k) gives the biased fixed-point A entries
// (to_biased54).  kLanesOnRows puts the lanes of a warp on consecutive rows r (for an afix source
// laid out with r contiguous); otherwise on consecutive k.  All threads call.  False on timeout.
template <bool kLanesOnRows = false, class AFix>
__device__ inline bool ozaki_mma_pass(const OzSmem& z, uint32_t tmem, int a_rows, AFix afix, uint32_t ph[2],
                                      int* status) {
  const int tid = threadIdx.x;
  for (int s = 1; s <= oz::kDigits; ++s) {
    const int b = (s - 1) & 1;
    if (s >= 3) {
      const bool ok = oz_wait_all(z, z.bars + 1 + b, ph[b], status);
      ph[b] ^= 1u;
      if (!ok) return false;
    }
    char* abuf = z.asl + b * oz::kASliceBytes;
    for (int idx = tid; idx < a_rows * 32; idx += kOzT) {  // two k per thread: one 32-bit store
      const int r = kLanesOnRows ? idx % a_rows : idx >> 5;
      const int k = kLanesOnRows ? (idx / a_rows) * 2 : (idx & 31) * 2;
      *reinterpret_cast<uint32_t*>(abuf + oz::op_off(r, k)) = oz::digit_pair(afix(r, k), afix(r, k + 1), s);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      oz::fence_after_sync();
      // the B slices t = 1 .. digit_t_max(s) lie one after another, as do their groups s + t - 2
      // in TMEM: one MMA takes up to four of them (N up to 256)
      const uint64_t adesc = oz::sw128_desc(smem_u32(abuf));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)  // K step of 16 bf16 = 32 bytes = 2 descriptor units
        for (int t0 = 1; t0 <= oz::digit_t_max(s); t0 += 4) {
          const int nt = min(4, oz::digit_t_max(s) + 1 - t0);
          const uint32_t d = tmem + (uint32_t)(s + t0 - 2) * 64u;
          const uint64_t bdesc = oz::sw128_desc(smem_u32(z.bsl + (t0 - 1) * oz::kBSliceBytes));
          oz::mma_bf16(d, adesc + 2 * kk, bdesc + 2 * kk, oz::idesc_bf16(oz::kM, 64u * nt),
                       (s > 1 || kk > 0) ? 1u : 0u);
        }
      oz::mma_commit(z.bars + 1 + b);
    }
  }
  bool ok = oz_wait_all(z, z.bars + 1, ph[0], status);
  ph[0] ^= 1u;
  ok = oz_wait_all(z, z.bars + 2, ph[1], status) && ok;
  ph[1] ^= 1u;
  oz::fence_after_sync();
  return ok;
}

// Rows r0..r1-1 of both A buffers set to zero (the MMA reads all 128 rows).
__device__ inline void ozaki_zero_a_rows(const OzSmem& z, int r0, int r1) {
  for (int i = threadIdx.x; i < 2 * (r1 - r0) * 8; i += kOzT) {
    const int b = i / ((r1 - r0) * 8), rem = i % ((r1 - r0) * 8);
    *reinterpret_cast<uint4*>(z.asl + b * oz::kASliceBytes + (size_t)(r0 + rem / 8) * 128 + (rem % 8) * 16) =
        make_uint4(0, 0, 0, 0);
  }
}

// The 7 digit slices of a B operand entry pair and the eighth, zero slice.
__device__ __forceinline__ void put_b_digits(const OzSmem& z, uint32_t off, uint64_t m0, uint64_t m1) {
#pragma unroll
  for (int s = 1; s <= oz::kDigits; ++s)
    *reinterpret_cast<uint32_t*>(z.bsl + (s - 1) * oz::kBSliceBytes + off) = oz::digit_pair(m0, m1, s);
  *reinterpret_cast<uint32_t*>(z.bsl + (oz::kDigitBSlices - 1) * oz::kBSliceBytes + off) = 0u;
}

// B digit slices of the 64 x 64 matrix whose output column j and k-th entry is bval(j, k),
// against the column exponents in z.expB.  All threads call; ends with a barrier.
template <class BVal>
__device__ inline void ozaki_b_fill(const OzSmem& z, BVal bval) {
  const int tid = threadIdx.x;
  for (int idx = tid; idx < 64 * 32; idx += kOzT) {
    const int j = idx >> 5, k = (idx & 31) * 2;
    put_b_digits(z, oz::op_off(j, k), oz::to_biased54(bval(j, k), z.expB[j]), oz::to_biased54(bval(j, k + 1), z.expB[j]));
  }
  fence_proxy_async_smem();
  __syncthreads();
}

// The same with the column exponents computed here from the 64 entries of each column.
template <class BVal>
__device__ inline void ozaki_b_slices(const OzSmem& z, BVal bval) {
  const int tid = threadIdx.x;
  for (int j = tid; j < 64; j += kOzT) z.expB[j] = 0;
  __syncthreads();
  for (int idx = tid; idx < 64 * 64; idx += kOzT) warp_max_into(&z.expB[idx >> 6], oz::bexp(bval(idx >> 6, idx & 63)));
  __syncthreads();
  ozaki_b_fill(z, bval);
}

// The same for a source laid out with j contiguous: the lanes of a warp take consecutive j, so
// the reads of bval do not collide in the shared-memory banks.
template <class BVal>
__device__ inline void ozaki_b_slices_jmajor(const OzSmem& z, BVal bval) {
  const int tid = threadIdx.x;
  for (int j = tid; j < 64; j += kOzT) z.expB[j] = 0;
  __syncthreads();
  {  // column j's maximum over k, k strided by the kOzT / 64 groups
    const int j = tid & 63, kg = tid >> 6;
    int e = 0;
    for (int k = kg; k < 64; k += kOzT / 64) e = max(e, oz::bexp(bval(j, k)));
    atomicMax(&z.expB[j], e);
  }
  __syncthreads();
  for (int idx = tid; idx < 64 * 32; idx += kOzT) {
    const int j = idx & 63, k = (idx >> 6) * 2;
    put_b_digits(z, oz::op_off(j, k), oz::to_biased54(bval(j, k), z.expB[j]), oz::to_biased54(bval(j, k + 1), z.expB[j]));
  }
  fence_proxy_async_smem();
  __syncthreads();
}

// Reads the 8 group accumulators back: out(i, j, value) for rows i < rows and all 64 columns.
// Warp w reads TMEM lanes 32 (w & 3).. and columns 16 (w >> 2)..; warps without valid rows skip.
template <class Out>
__device__ inline void ozaki_epilogue(const OzSmem& z, uint32_t tmem, int rows, Out out) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sp = warp & 3;
  const int i = 32 * sp + lane;
  const int c0 = 16 * (warp >> 2);
  if (32 * sp < rows) {
    const uint32_t tb = tmem + ((uint32_t)(32 * sp) << 16) + (uint32_t)c0;
    const int ea = z.expA[i];
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {  // 8 columns at a time, four groups' loads per wait
      long long acc[8];
      oz::load_digit_groups8(tb + 8u * (uint32_t)hf, 64u, acc);
      if (i < rows) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int j = c0 + 8 * hf + c;
          out(i, j, oz::scale_int(acc[c], ea + z.expB[j] - 2096));
        }
      }
    }
  }
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// The value of an 8-byte workspace slot: a double, or a double-float (hi, lo) pair when the
// factorization ran in double-float arithmetic (the sum is exact in FP64).
template <bool kPairs>
__device__ __forceinline__ double slot_val(double raw) {
  if constexpr (kPairs) {
    const f32x2 p = *reinterpret_cast<const f32x2*>(&raw);
    return (double)p.hi + (double)p.lo;
  } else {
    return raw;
  }
}

// Exponent and fixed-point form of a slot, straight from the pair's FP32 bits when kPairs.
template <bool kPairs>
__device__ __forceinline__ int slot_bexp(double raw) {
  if constexpr (kPairs) return oz::bexp_pair(raw);
  else return oz::bexp(raw);
}
// The biased 54-bit fixed point of a slot, for the digit form of the split (ozaki.cuh).
template <bool kPairs>
__device__ __forceinline__ uint64_t slot_biased54(double raw, int emax) {
  if constexpr (kPairs) return oz::to_biased54_pair(raw, emax);
  else return oz::to_biased54(raw, emax);
}

}  // namespace tsqr
