// The Gram entries that the compact-WY T of a flat-tree step is built from, g_pq = v_p^T v_q
// (p < q, over the leaf's rows; Sec. 3.2: T from the reflectors' inner products), taken on the
// tensor cores as one Ozaki-split product V^T V, for the Ozaki WY form (FP64 storage, FP64-level
// results).  The reflectors themselves, tau, R and the merge that turns the Gram entries into T
// stay on the FP64 path.  The operand conversion also reads double-float pairs, but the
// double-float forms keep the column loop's Gram entries (factor.cu says why).
//
// Reading: building T is native FP64 in the method's precision split, but its Gram entries are a
// dense contraction of the reflectors, the same kind of product as the WY products, so they are
// taken the same way; the merge T = [T1, -T1 G12 T2; 0, T2] that consumes them stays FP64.
//
// Scheme (ozaki.cuh): every column c of the leaf's reflector block V_bot (H x 64) in 56-bit fixed
// point against its largest exponent, cut into 8 slices of 7 bits held exactly in bf16.  The 36
// slice pairs of weight s + t <= 9 accumulate in 8 FP32 TMEM groups; a group sum stays below
// 127^2 * H * 8 < 2^24 for H <= 128, so it is exact, and the int64 recombination gives g_pq to
// about 2^-50 of |v_p|_max |v_q|_max.
//
// Shared memory: the step's T and reduction scratch are free once the column loop ends, so the
// slices are staged there, 16 rows of V_bot at a time (32-byte K-major rows, the 32-byte
// swizzle), all 8 slices at once (16 KB).  TMEM: 8 groups x 32 columns = 256 columns, so a block
// holds half of an SM's TMEM and two blocks run per SM; the 64 x 64 Gram is taken in two column
// passes (q < 32, then q >= 32).  Only 64 of the M = 128 rows of each MMA are real: the other rows
// of the A operand are whatever shared memory follows (always inside the staging area), and their
// TMEM lanes are never read.
#pragma once

#include "arith.cuh"
#include "ozaki.cuh"
#include "ozaki_pass.cuh"

namespace tsqr {
namespace gram {

constexpr uint32_t kTmemCols = 256;    // 8 weight groups x 32 columns
constexpr int kChunk = 16;             // rows of V_bot per staging round (the MMA's K)
constexpr uint32_t kSliceBytes = 2048; // 64 operand rows x 32 bytes
// The 8 slices plus the 64 rows past the last one that an M = 128 MMA reads.
constexpr uint32_t kStageBytes = 9 * kSliceBytes;

// What the tensor-core Gram needs besides the step's own operands.
struct GramTC {
  char* stage;      // kStageBytes of shared memory, 256-byte aligned, free during the call
  int* expc;        // 64 ints of shared memory
  uint64_t* bar;    // MMA completion barrier (count 1)
  uint32_t* phase;  // its parity, tracked by every thread
  uint32_t tmem;    // kTmemCols TMEM columns held by the block
  int* status;      // device status word
  int* flag;        // shared broadcast word
};

// Shared-memory matrix descriptor of a K-major operand in 32-byte swizzled rows of 16 bf16: 8-row
// groups 256 bytes apart (SBO), descriptor version 1, swizzle mode 32B.
__device__ __forceinline__ uint64_t sw32_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(256 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)6 << 61);
}
// Byte offset of element (row c, k) of such an operand: the 16-byte chunk index (k / 8) XOR bit 2
// of the row.
__device__ __forceinline__ uint32_t op32_off(int c, int k) {
  const uint32_t byte = (uint32_t)k * 2u;
  return (uint32_t)c * 32u + ((((byte >> 4) ^ (((uint32_t)c >> 2) & 1u))) << 4) + (byte & 15u);
}

// Biased FP64 exponent bound of a stored entry (2047 for Inf or NaN) and its fixed-point form
// against the column's bound: FP64 entries directly, double-float pairs by their two words.
template <class Ar>
__device__ __forceinline__ int entry_exp(double raw) {
  if constexpr (Ar::kPrecision == 0) {
    return oz::bexp(raw);
  } else {
    const uint32_t hb = (uint32_t)(unsigned long long)__double_as_longlong(raw);
    return (((hb >> 23) & 0xFFu) == 0xFFu) ? 2047 : oz::bexp_pair(raw);
  }
}
template <class Ar>
__device__ __forceinline__ uint64_t entry_fixed(double raw, int emax) {
  if constexpr (Ar::kPrecision == 0)
    return oz::to_fixed(raw, emax);
  else
    return oz::to_fixed_pair(raw, emax);
}

// The 8 slices of bottom rows [kChunk k, kChunk k + kChunk) of columns 0..C-1 into the stage:
// slice s (1-based) at (s - 1) * kSliceBytes, operand row c = column c, K = the chunk's rows.
// Lanes run along K first, so a warp writes whole 32-byte rows.
template <class Ar, int NP, int C>
__device__ __forceinline__ void stage_chunk(const Tile& S, const GramTC& g, int k) {
  constexpr int RPT = C * kChunk / kThreads;  // rows per thread: 4 (C = 64) or 2 (C = 32)
  constexpr int KQ = kChunk / RPT;            // threads along K per column
  static_assert(RPT == 2 || RPT == 4, "two or four rows per thread");
  const int tid = threadIdx.x;
  const int c = tid / KQ;
  const int k0 = (tid % KQ) * RPT;
  const int e = g.expc[c];
  uint64_t fx[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) fx[i] = entry_fixed<Ar>(*S.ptr(NP + kChunk * k + k0 + i, c), e);
  const uint32_t off = op32_off(c, k0);
#pragma unroll
  for (int s = 1; s <= oz::kSlices; ++s) {
    char* buf = g.stage + (s - 1) * kSliceBytes;
    if constexpr (RPT == 4) {
      uint2 w;
      w.x = slice_pair(fx[0], fx[1], s);
      w.y = slice_pair(fx[2], fx[3], s);
      *reinterpret_cast<uint2*>(buf + off) = w;
    } else {
      *reinterpret_cast<uint32_t*>(buf + off) = slice_pair(fx[0], fx[1], s);
    }
  }
}

// Thread 0 waits (bounded) for the MMAs committed last; every thread learns the outcome.
__device__ __forceinline__ bool wait_mma(const GramTC& g) {
  if (threadIdx.x == 0) {
    const bool ok = oz::wait_bar(g.bar, *g.phase);
    *g.flag = ok ? 0 : 1;
    if (!ok) atomicOr(g.status, kStatusTimeout);
  }
  *g.phase ^= 1u;
  __syncthreads();
  oz::fence_after_sync();
  return *g.flag == 0;
}

// One column pass: the group sums of D = V_bot^T V_bot(:, q0..q0+31) over all H rows, with C
// operand rows staged (32 for q0 = 0: only p < q < 32 is wanted; 64 for q0 = 32).
template <class Ar, int NP, int H, int C>
__device__ inline bool gram_pass(const Tile& S, const GramTC& g, int q0) {
  const uint32_t idesc = oz::idesc_bf16(oz::kM, 32);
  for (int k = 0; k < H / kChunk; ++k) {
    stage_chunk<Ar, NP, C>(S, g, k);
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      oz::fence_after_sync();
      const uint32_t base = smem_u32(g.stage);
      for (int s = 1; s <= oz::kSlices; ++s) {
        const uint64_t a = sw32_desc(base + (uint32_t)(s - 1) * kSliceBytes);
        for (int t = 1; t <= oz::kSlices + 1 - s; ++t) {
          const uint64_t b = sw32_desc(base + (uint32_t)(t - 1) * kSliceBytes + (uint32_t)q0 * 32u);
          oz::mma_bf16(g.tmem + (uint32_t)(s + t - 2) * 32u, a, b, idesc, (k > 0 || s > 1) ? 1u : 0u);
        }
      }
      oz::mma_commit(g.bar);
    }
    if (!wait_mma(g)) return false;  // the stage is rewritten next round
  }
  return true;
}

// Reads the pass's 8 groups (warps whose TMEM lane quarter holds rows p < rows), recombines them
// and hands g_pq (p < q < n) to put(p, q, value).
template <class Put>
__device__ inline void gram_read(const GramTC& g, int rows, int q0, int n, Put put) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, half = warp >> 2;  // lanes 32 quarter.., columns 16 half..
  if (quarter * 32 >= rows) return;
  const int p = quarter * 32 + lane;
  const int ep = g.expc[p];
#pragma unroll 1
  for (int part = 0; part < 2; ++part) {
    const int c0 = 16 * half + 8 * part;
    long long acc[8];
    oz::load_groups<8>(g.tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, 32, acc);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int q = q0 + c0 + c;
      if (p < q && q < n) {
        const int eq = g.expc[q];
        const double v = (ep == 2047 || eq == 2047) ? __longlong_as_double(0x7FF8000000000000LL)
                                                    : oz::int_to_f64_scaled(acc[c], ep + eq - 2100);
        put(p, q, v);
      }
    }
  }
}

// The Gram entries of the step's reflectors (rows NP..NP+H-1 of the tile, columns 0..n-1, scaled
// v = x / (alpha - beta) with the unit top parts left implicit: e_p^T e_q = 0) into T_s above the
// diagonal, and tau_s on its diagonal, ready for the blocked merge.  X (32 x 32 entries) holds
// the first pass's results while T_s is the stage.  All threads call; false on a timed-out wait.
template <class Ar, int NP, int H>
__device__ inline bool gram_ozaki(const Tile& S, int n, typename Ar::E* T_s, const typename Ar::E* tau_s,
                                  typename Ar::E* X, const GramTC& g) {
  static_assert(NP == 64, "the Gram passes cover 64 columns");
  static_assert(H % kChunk == 0 && H <= 128, "group sums are exact for at most 128 rows");
  using E = typename Ar::E;
  const int tid = threadIdx.x;
  // the largest exponent of every column
  for (int c = tid; c < NP; c += kThreads) g.expc[c] = 0;
  __syncthreads();
  {
    const int c = tid & (NP - 1);
    int e = 0;
    for (int r = tid / NP; r < H; r += kThreads / NP) e = max(e, entry_exp<Ar>(*S.ptr(NP + r, c)));
    atomicMax(&g.expc[c], e);
  }
  __syncthreads();
  // pass 0: q < 32 (rows p < 32), kept in X
  if (!gram_pass<Ar, NP, H, 32>(S, g, 0)) return false;
  gram_read(g, 32, 0, n, [&](int p, int q, double v) { X[p * 32 + q] = Ar::from_f64(v); });
  oz::fence_before_sync();
  __syncthreads();
  // pass 1: q >= 32 (all rows p), straight into T_s now that the stage is done with
  if (!gram_pass<Ar, NP, H, 64>(S, g, 32)) return false;
  gram_read(g, 64, 32, n, [&](int p, int q, double v) { T_s[tri_off(p, NP) + (q - p)] = Ar::from_f64(v); });
  oz::fence_before_sync();
  __syncthreads();
  for (int i = tid; i < 32 * 32; i += kThreads) {
    const int p = i >> 5, q = i & 31;
    if (p < q && q < n) T_s[tri_off(p, NP) + (q - p)] = X[i];
  }
  for (int j = tid; j < n; j += kThreads) T_s[tri_off(j, NP)] = tau_s[j];
  __syncthreads();
  return true;
}

}  // namespace gram
}  // namespace tsqr
