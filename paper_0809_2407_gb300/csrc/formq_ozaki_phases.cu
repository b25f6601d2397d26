// Thin Q with Ozaki products (precision modes 2 and 3, np = 64, h <= 128), in three kernels.
//
// In a flat chain the thin Q flows from the chain's last leaf to its first: with C_k the n x n
// block carried into leaf k's step (Sec. 3.2, Q_k = I - Y_k T_k Y_k^T with Y_k = [I; V_k]),
//   M_k = T_k C_k,   C_{k-1} = C_k - M_k,   Q rows of leaf k = -V_k M_k.
// Only the n x n recurrence carries the chain's dependence, so the work is taken apart:
//   1. formq_ozaki_recur_kernel: per chain, the recurrence alone.  C stays in the registers of
//      half of the block's warps, which build its slices, wait for the product and update C;
//      the other half splits the next leaf's T (which does not depend on C) into a second
//      buffer while the tensor cores work, so each leaf costs one commit.  M_k goes into the
//      first n rows of leaf k's own rows of Q; the block entering the first leaf into node_r[g].
//   2. formq_ozaki_kernel (apply.cu), split mode: each chain's first leaf (V unit lower
//      trapezoidal; three products), from that block.
//   3. formq_ozaki_leaves_kernel: the h x n products -V_k M_k of all other leaves, independent
//      of one another, written over M_k.
// A chain that holds a short last leaf (fewer than n rows) is taken whole by kernel 2.
//
// Ozaki products (ozaki.cuh): every operand row (A) or column (B) in 56-bit fixed point against
// its largest exponent, cut into 8 slices of 7 bits held exactly in bf16; the 36 slice pairs of
// weight <= 9 accumulate in 8 exact FP32 TMEM groups (K = 64), recombined in int64.  Every wait
// is bounded; a block that gives up sets the status word, waits once more for its MMAs in flight
// and frees its TMEM.
#include "factor_kernels.h"
#include "ozaki_pass.cuh"

namespace tsqr {
namespace {

// ---- 1. the recurrences --------------------------------------------------------------------
// One block of 512 threads per SM, persistent over chains.  M = T C is taken as two products of
// 32 columns whose real rows land in different TMEM lane halves: the first with T's slices as the
// A operand (rows 0..63 -> lanes 0..63), the second with the A descriptor started 64 rows
// (8 KB) earlier, so T's rows arrive in lanes 64..127.  Half hh's weight group g sits at TMEM
// column 256 hh + 32 g.  Every warp can then read a part of M back
// (a warp reads only its own lane quarter): thread (warp, lane) owns row i = 32 (warp & 1) + lane
// of columns j0 .. j0 + 7, j0 = 32 ((warp >> 1) & 1) + 8 (warp >> 2), and keeps C's entries there
// in registers.  While the tensor cores work, every warp splits the next leaf's T (4 rows each)
// into the other slice buffer, so a leaf costs one commit and T's splitting is off its path.
constexpr uint32_t kTSliceBytes = 64 * 128;               // 64 operand rows of 128 bytes
constexpr uint32_t kTBufBytes = oz::kDigits * kTSliceBytes;  // one leaf's 7 digit slices of T
// C's slices as two halves of 32 output columns, the 8 slices of a half (the last one zero)
// one after another
constexpr uint32_t kCSliceBytes = 32 * 128;
constexpr uint32_t kCHalfBytes = oz::kDigitBSlices * kCSliceBytes;

size_t recur_smem_bytes() {
  // 64 rows read before the first buffer, two T buffers, 64 rows read past the second, C's
  // slices, T row exponents (2 x 64), C column maxima of the two lane halves (2 x 64), barrier,
  // slot, flag
  return 1024 + kTSliceBytes + 2 * (size_t)kTBufBytes + kTSliceBytes + 2 * (size_t)kCHalfBytes + 4 * 64 * 4 + 8 +
         8 + 8;
}

template <bool kPairs>
__global__ void __launch_bounds__(kOzT, 1)
    formq_ozaki_recur_kernel(const Plan P, const Store st, double* __restrict__ Q, int64_t ldq) {
  extern __shared__ char smem_raw[];
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  char* tbuf = base + kTSliceBytes;                       // 2 x kTBufBytes, 64 rows before and after
  char* bsl = tbuf + 2 * kTBufBytes + kTSliceBytes;       // C's 8 slices
  int* expT = reinterpret_cast<int*>(bsl + 2 * kCHalfBytes);  // [2][64]
  int* expC2 = expT + 2 * 64;                                       // [2][64]
  uint64_t* bar = reinterpret_cast<uint64_t*>(expC2 + 2 * 64);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  int* flag = reinterpret_cast<int*>(slot + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q4 = warp & 3;                     // TMEM lane quarter
  const int half = q4 >> 1;                    // which 32-column product this warp reads
  const int i = 32 * (q4 & 1) + lane;          // row of C and M
  const int j0 = 32 * half + 8 * (warp >> 2);  // first of its 8 columns
  const int np = 64, n = P.n, h = P.h;
  const bool odd = (lane & 1) != 0;

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    *flag = 0;
  }
  for (int i2 = tid; i2 < 2 * (int)kCSliceBytes / 16; i2 += kOzT)  // the zero eighth slice of each half
    *reinterpret_cast<uint4*>(bsl + (i2 / (kCSliceBytes / 16)) * kCHalfBytes + (oz::kDigitBSlices - 1) * kCSliceBytes +
                              (i2 % (kCSliceBytes / 16)) * 16) = make_uint4(0, 0, 0, 0);
  fence_proxy_async_smem();
  if (warp == 0) oz::tmem_alloc(slot, oz::kTmemCols);
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  const uint32_t tmem = *slot;
  uint32_t phase = 0;
  bool alive = true;

  // T rows warp + 16 u (u < 4) of a leaf in registers, then their exponents and slices into buffer bb
  double2 traw[4];
  auto t_load = [&](int64_t leaf) {
    const double* Tk = st.t_leaf + leaf * np * np;
#pragma unroll
    for (int u = 0; u < 4; ++u) traw[u] = __ldcg(reinterpret_cast<const double2*>(Tk + (warp + 16 * u) * np) + lane);
  };
  auto t_slices = [&](int bb) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = warp + 16 * u;
      const int e = __reduce_max_sync(0xffffffffu, max(slot_bexp<kPairs>(traw[u].x), slot_bexp<kPairs>(traw[u].y)));
      if (lane == 0) expT[bb * 64 + r] = e;
      const uint64_t f0 = slot_biased54<kPairs>(traw[u].x, e), f1 = slot_biased54<kPairs>(traw[u].y, e);
      char* dst = tbuf + bb * kTBufBytes + oz::op_off(r, 2 * lane);
#pragma unroll
      for (int s = 1; s <= oz::kDigits; ++s)
        *reinterpret_cast<uint32_t*>(dst + (s - 1) * kTSliceBytes) = oz::digit_pair(f0, f1, s);
    }
  };
  // C's column exponent: the two lane halves of a column meet in shared memory
  auto col_exp = [&](int q) { return max(expC2[j0 + q], expC2[64 + j0 + q]); };

  for (int g = blockIdx.x; g < P.chains && alive; g += gridDim.x) {
    if (formq_chain_short(P, g)) continue;  // taken whole by formq_ozaki_kernel
    const int64_t l0 = chain_first_leaf(P, g), l1 = chain_end_leaf(P, g);
    double* Cg = st.node_r + (size_t)g * np * np;
    double c[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      c[q] = (P.depth == 0) ? ((i == j0 + q && i < n) ? __ldcg(st.signs + i) : 0.0)
                            : slot_val<kPairs>(__ldcg(Cg + i * np + j0 + q));
    if (l1 - 1 > l0) {
      t_load(l1 - 1);
      t_slices(0);
      if (l1 - 2 > l0) t_load(l1 - 2);
    }
    int b = 0;
    for (int64_t k = l1 - 1; k > l0; --k, b ^= 1) {
      const int64_t row0 = k * h;
      // ---- C's column exponents
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int e = __reduce_max_sync(0xffffffffu, oz::bexp(c[q]));
        if (lane == 0) expC2[(q4 & 1) * 64 + j0 + q] = e;
      }
      __syncthreads();
      // ---- C's slices (B operand: output column j, K = C's row): rows i, i + 1 pair up; the
      //      even lane takes columns j0 .. j0 + 3, the odd lane j0 + 4 .. j0 + 7
      {
        double recv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) recv[q] = __shfl_xor_sync(0xffffffffu, odd ? c[q] : c[4 + q], 1);
        const int k0 = i & ~1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int cq = odd ? 4 + q : q;
          const int ec = col_exp(cq);
          const uint64_t f0 = oz::to_biased54(odd ? recv[q] : c[q], ec);
          const uint64_t f1 = oz::to_biased54(odd ? c[4 + q] : recv[q], ec);
          char* dst = bsl + half * kCHalfBytes + oz::op_off(j0 - 32 * half + cq, k0);
#pragma unroll
          for (int s = 1; s <= oz::kDigits; ++s)
            *reinterpret_cast<uint32_t*>(dst + (s - 1) * kCSliceBytes) = oz::digit_pair(f0, f1, s);
        }
      }
      fence_proxy_async_smem();
      __syncthreads();
      // ---- M = T C: two 32-column products of 36 slice pairs each, one commit
      if (tid == 0) {
        oz::fence_after_sync();
        // digit slice s of T meets C's digit slices t = 1 .. digit_t_max(s) of a half, which lie
        // one after another in shared memory, as do their groups s + t - 2 in TMEM: one MMA each
        for (int kk = 0; kk < 4; ++kk)  // K step of 16 bf16 = 32 bytes = 2 descriptor units
          for (int hh = 0; hh < 2; ++hh)
            for (int s = 1; s <= oz::kDigits; ++s) {
              const uint64_t adesc = oz::sw128_desc(
                  smem_u32(tbuf + b * kTBufBytes + (s - 1) * kTSliceBytes - (uint32_t)hh * kTSliceBytes));
              const uint32_t d = tmem + 256u * (uint32_t)hh + (uint32_t)(s - 1) * 32u;
              const uint64_t bdesc = oz::sw128_desc(smem_u32(bsl + (uint32_t)hh * kCHalfBytes));
              oz::mma_bf16(d, adesc + 2 * kk, bdesc + 2 * kk, oz::idesc_bf16(oz::kM, 32u * oz::digit_t_max(s)),
                           (s > 1 || kk > 0) ? 1u : 0u);
            }
        oz::mma_commit(bar);
      }
      // ---- while they run: the next leaf's T slices into the other buffer, the one after loaded
      if (k - 1 > l0) {
        t_slices(b ^ 1);
        if (k - 2 > l0) t_load(k - 2);
      }
      if (tid == 0) {
        const bool ok = oz::wait_bar(bar, phase);
        *flag = ok ? 0 : 1;
        if (!ok) atomicOr(st.status, kStatusTimeout);
      }
      phase ^= 1u;
      __syncthreads();
      oz::fence_after_sync();
      if (*flag != 0) {
        alive = false;
        break;
      }
      // ---- M back from TMEM (row i, columns j0..j0+7), C -= M, M into Q
      {
        long long acc[8];
        oz::load_digit_groups8(tmem + ((uint32_t)(32 * q4) << 16) + 256u * (uint32_t)half + (uint32_t)(j0 - 32 * half),
                               32u, acc);
        const int ea = expT[b * 64 + i];
        double* dst = Q + gidx(P, row0 + i, 0, ldq);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const double mq = oz::int_to_f64_scaled(acc[q], ea + col_exp(q) - 2096);
          c[q] -= mq;
          if (i < n && j0 + q < n) dst[P.col_major ? (int64_t)(j0 + q) * ldq : j0 + q] = mq;
        }
      }
      oz::fence_before_sync();
      __syncthreads();
    }
    // the block entering the chain's first leaf, for formq_ozaki_kernel (plain FP64)
    if (alive) {
#pragma unroll
      for (int q = 0; q < 8; ++q) Cg[i * np + j0 + q] = c[q];
    }
  }
  if (!alive && tid == 0) oz::wait_bar(bar, phase ^ 1u);  // the MMAs in flight, once more
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  if (warp == 0) oz::tmem_dealloc(tmem, oz::kTmemCols);
}

// ---- 3. the leaf products -------------------------------------------------------------------
// Persistent grid, one block of 512 threads per SM, leaves by grid stride.  Per leaf: the
// reflector rows straight from HBM (one warp per row, two entries per lane, a 16-byte load), their
// exponent by a warp reduction, their 8 slices into shared memory as the A operand (128 operand
// rows, zero past the leaf); M (zero past n) as the B operand; the 36 slice products in one
// commit; while they run, the next leaf's reflector rows and M are loaded into registers; then
// the int64 epilogue writes -V M over M.
constexpr int kWarps = kOzT / 32;          // 16
constexpr int kRowsPerWarp = oz::kM / kWarps;  // 8: the 128 operand rows over the warps
constexpr int kMPerThread = 64 * 32 / kOzT;    // 4 pairs (k, k + 1) of M entries per thread

size_t leaves_smem_bytes() {
  return 1024 + oz::kDigits * (size_t)oz::kASliceBytes + oz::kDigitBSlices * (size_t)oz::kBSliceBytes + 128 * 4 +
         64 * 4 + 8 + 8 + 8;
}

__device__ __forceinline__ int64_t next_deferred(const Plan& P, int64_t leaf) {
  while (leaf < P.leaves && !formq_leaf_deferred(P, leaf)) leaf += gridDim.x;
  return leaf;
}

template <bool kPairs>
__global__ void __launch_bounds__(kOzT, 1)
    formq_ozaki_leaves_kernel(const Plan P, const Store st, double* __restrict__ Q, int64_t ldq) {
  extern __shared__ char smem_raw[];
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  char* asl = base;
  char* bsl = asl + oz::kDigits * oz::kASliceBytes;
  int* expA = reinterpret_cast<int*>(bsl + oz::kDigitBSlices * oz::kBSliceBytes);
  int* expB = expA + 128;
  uint64_t* bar = reinterpret_cast<uint64_t*>(expB + 64);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  int* flag = reinterpret_cast<int*>(slot + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = P.n, h = P.h;
  const double* V = st.v;
  const int64_t ldv = st.ldv;

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    *flag = 0;
  }
  for (int i2 = tid; i2 < (int)oz::kBSliceBytes / 16; i2 += kOzT)  // the zero eighth B slice
    *reinterpret_cast<uint4*>(bsl + (oz::kDigitBSlices - 1) * oz::kBSliceBytes + i2 * 16) = make_uint4(0, 0, 0, 0);
  fence_proxy_async_smem();
  if (warp == 0) oz::tmem_alloc(slot, oz::kTmemCols);
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  const uint32_t tmem = *slot;
  uint32_t phase = 0;

  // one leaf's operands in registers: rows warp + kWarps u of V (columns 2 lane, 2 lane + 1), and
  // M entries (k, j), (k + 1, j) with j = tid % 64, k = 2 (tid / 64 + 8 u)
  double2 vr[kRowsPerWarp], mr[kMPerThread];
  const int j_own = tid & 63;
  auto load = [&](int64_t leaf) {
    const int64_t row0 = leaf * h;
    const int rv = (int)((P.m - row0 < h) ? (P.m - row0) : h);
    const int c = 2 * lane;
#pragma unroll
    for (int u = 0; u < kRowsPerWarp; ++u) {
      const int r = warp + kWarps * u;
      double2 v = make_double2(0.0, 0.0);
      if (r < rv && c < n) {
        v = __ldcg(reinterpret_cast<const double2*>(V + (row0 + r) * ldv + c));
        if (c + 1 >= n) v.y = 0.0;
      }
      vr[u] = v;
    }
#pragma unroll
    for (int u = 0; u < kMPerThread; ++u) {
      const int k = 2 * ((tid >> 6) + 8 * u);
      mr[u].x = (k < n && j_own < n) ? __ldcg(Q + gidx(P, row0 + k, j_own, ldq)) : 0.0;
      mr[u].y = (k + 1 < n && j_own < n) ? __ldcg(Q + gidx(P, row0 + k + 1, j_own, ldq)) : 0.0;
    }
  };

  int64_t leaf = next_deferred(P, blockIdx.x);
  if (leaf < P.leaves) load(leaf);
  bool alive = true;
  while (leaf < P.leaves) {
    const int64_t row0 = leaf * h;
    const int rv = (int)((P.m - row0 < h) ? (P.m - row0) : h);
    // ---- A: the reflector rows, exponent per row, fixed point, 8 slices
    if (tid < 64) expB[tid] = 0;
#pragma unroll
    for (int u = 0; u < kRowsPerWarp; ++u) {
      const int r = warp + kWarps * u;
      const int e = __reduce_max_sync(0xffffffffu, max(slot_bexp<kPairs>(vr[u].x), slot_bexp<kPairs>(vr[u].y)));
      if (lane == 0) expA[r] = e;
      const uint64_t f0 = slot_biased54<kPairs>(vr[u].x, e), f1 = slot_biased54<kPairs>(vr[u].y, e);
      const uint32_t off = oz::op_off(r, 2 * lane);
#pragma unroll
      for (int s = 1; s <= oz::kDigits; ++s)
        *reinterpret_cast<uint32_t*>(asl + (s - 1) * oz::kASliceBytes + off) = oz::digit_pair(f0, f1, s);
    }
    __syncthreads();
    // ---- B: M's column exponents, then its slices (output column j, K = M's rows)
    {
      int e = 0;
#pragma unroll
      for (int u = 0; u < kMPerThread; ++u) e = max(e, max(oz::bexp(mr[u].x), oz::bexp(mr[u].y)));
      atomicMax(&expB[j_own], e);
    }
    __syncthreads();
    {
      const int e = expB[j_own];
#pragma unroll
      for (int u = 0; u < kMPerThread; ++u) {
        const int k = 2 * ((tid >> 6) + 8 * u);
        const uint64_t f0 = oz::to_biased54(mr[u].x, e), f1 = oz::to_biased54(mr[u].y, e);
        const uint32_t off = oz::op_off(j_own, k);
#pragma unroll
        for (int s = 1; s <= oz::kDigits; ++s)
          *reinterpret_cast<uint32_t*>(bsl + (s - 1) * oz::kBSliceBytes + off) = oz::digit_pair(f0, f1, s);
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    // ---- the 36 slice products, one commit
    if (tid == 0) {
      oz::fence_after_sync();
      // digit slice s of A meets B's slices t = 1 .. digit_t_max(s), which lie one after another
      // in shared memory and whose groups s + t - 2 lie one after another in TMEM: one MMA takes up
      // to four of them (N up to 256), so a product is 11 MMAs per K step instead of 34
      for (int kk = 0; kk < 4; ++kk)  // K step of 16 bf16 = 32 bytes = 2 descriptor units
        for (int s = 1; s <= oz::kDigits; ++s) {
          const uint64_t adesc = oz::sw128_desc(smem_u32(asl + (s - 1) * oz::kASliceBytes));
          for (int t0 = 1; t0 <= oz::digit_t_max(s); t0 += 4) {
            const int nt = min(4, oz::digit_t_max(s) + 1 - t0);
            const uint32_t d = tmem + (uint32_t)(s + t0 - 2) * 64u;
            const uint64_t bdesc = oz::sw128_desc(smem_u32(bsl + (t0 - 1) * oz::kBSliceBytes));
            oz::mma_bf16(d, adesc + 2 * kk, bdesc + 2 * kk, oz::idesc_bf16(oz::kM, 64u * nt),
                         (s > 1 || kk > 0) ? 1u : 0u);
          }
        }
      oz::mma_commit(bar);
    }
    // ---- the next leaf's operands load while the products run (this leaf's are in shared memory)
    const int64_t next = next_deferred(P, leaf + gridDim.x);
    if (next < P.leaves) load(next);
    if (tid == 0) {
      const bool ok = oz::wait_bar(bar, phase);
      *flag = ok ? 0 : 1;
      if (!ok) atomicOr(st.status, kStatusTimeout);
    }
    phase ^= 1u;
    __syncthreads();
    oz::fence_after_sync();
    if (*flag != 0) {
      alive = false;
      break;
    }
    // ---- -V M over the leaf's rows (M was read into registers before this leaf started)
    {
      // warp w reads TMEM lanes 32 (w & 3).. (rows) and columns 16 (w >> 2).., 8 at a time, into
      // a 128 x 64 FP64 tile over the A slices (dead until the next leaf), in 16-byte units whose
      // index within a row is XORed with (row & 7); then every warp writes whole rows to Q
      double* tile = reinterpret_cast<double*>(asl);
      const int sp = warp & 3, i = 32 * sp + lane, c0 = 16 * (warp >> 2);
      if (32 * sp < rv) {
        const uint32_t tb = tmem + ((uint32_t)(32 * sp) << 16) + (uint32_t)c0;
        const int ea = expA[i];
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          long long X[8];
          oz::load_digit_groups8(tb + 8u * (uint32_t)hf, 64u, X);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = c0 + 8 * hf + 2 * u;
            const int unit = (j >> 1) ^ (i & 7);
            *reinterpret_cast<double2*>(tile + i * 64 + 2 * unit) =
                make_double2(-oz::int_to_f64_scaled(X[2 * u], ea + expB[j] - 2096),
                             -oz::int_to_f64_scaled(X[2 * u + 1], ea + expB[j + 1] - 2096));
          }
        }
      }
      oz::fence_before_sync();
      __syncthreads();
      oz::fence_after_sync();
      const int j = 2 * lane;
      for (int r = warp; r < rv; r += kWarps) {
        const double2 v = *reinterpret_cast<const double2*>(tile + r * 64 + 2 * (lane ^ (r & 7)));
        if (j < n) {
          double* q = Q + gidx(P, row0 + r, j, ldq);
          if (!P.col_major && j + 1 < n && (reinterpret_cast<uintptr_t>(q) & 15) == 0) {
            *reinterpret_cast<double2*>(q) = v;
          } else {
            q[0] = v.x;
            if (j + 1 < n) Q[gidx(P, row0 + r, j + 1, ldq)] = v.y;
          }
        }
      }
      __syncthreads();  // the tile is read before the next leaf's A slices go over it
    }
    leaf = next;
  }
  // a block that gave up: one more bounded wait for the MMAs in flight before TMEM is freed
  if (!alive && tid == 0) oz::wait_bar(bar, phase ^ 1u);
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  if (warp == 0) oz::tmem_dealloc(tmem, oz::kTmemCols);
}

}  // namespace

cudaError_t launch_formq_ozaki_recur(const Plan& P, const Store& st, double* Q, int64_t ldq, cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = P.chains < sms ? P.chains : sms;
  const size_t smem = recur_smem_bytes();
  auto kernel = prec_df(P.precision) ? formq_ozaki_recur_kernel<true> : formq_ozaki_recur_kernel<false>;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kernel<<<blocks, kOzT, smem, stream>>>(P, st, Q, ldq);
  return cudaGetLastError();
}

cudaError_t launch_formq_ozaki_leaves(const Plan& P, const Store& st, double* Q, int64_t ldq, cudaStream_t stream) {
  if (P.leaves <= P.chains) return cudaSuccess;  // every leaf is the first of its chain
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t deferred = P.leaves - P.chains;
  const int blocks = (int)(deferred < sms ? deferred : sms);
  const size_t smem = leaves_smem_bytes();
  const bool pairs = prec_df(P.precision);
  auto kernel = pairs ? formq_ozaki_leaves_kernel<true> : formq_ozaki_leaves_kernel<false>;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kernel<<<blocks, kOzT, smem, stream>>>(P, st, Q, ldq);
  return cudaGetLastError();
}

}  // namespace tsqr
