// Blocked flat-tree step with the WY products on the tensor cores (precision mode 2: FP64 storage,
// FP64-level results).
//
// The step QR([R; A_k]) (Algorithm 2; Sec. 3.1: triangle atop a full block) is taken in panels of
// NB = 16 columns, the right-looking blocked Householder QR whose trailing update is the compact-WY
// form of the panel (Sec. 3.1-3.2: Q_p = I - V_p T_p V_p^T):
//   1. the panel's reflectors by the FP64 pipe, column by column (norms, beta and tau native FP64);
//   2. one Ozaki product over the leaf's h rows, D = S_bot^T V_p (64 x 16): its rows for the
//      columns right of the panel give W = C_top + V_bot^T C_bot, its other rows the Gram entries
//      v_c^T v_j (c < j) that T is built from;
//   3. T_p from the panel's Gram entries and tau by the blocked merge T = [T1, -T1 G12 T2; 0, T2]
//      in FP64, then W' = T_p^T W in FP64 and C_top -= W' on the pivot rows;
//   4. one Ozaki product C_bot -= V_bot W' over the trailing columns.
// After the last panel the leaf's T is completed by the same merge over the panels' blocks, with
// the cross-panel Gram entries from step 2.  Reading: the Gram entries feeding T are a contraction
// (V^T V), so they are taken on the tensor cores with the W product; the merge itself, the
// reflectors and the tree nodes stay native FP64.
//
// Ozaki products (ozaki.cuh): every operand row (A) or column (B) in 56-bit fixed point against
// its largest exponent, cut into 8 slices of 7 bits held exactly in bf16; the 36 slice pairs of
// weight <= 9 accumulate in 8 FP32 TMEM groups, exact because every group sum stays below 2^23
// (K <= 64); an int64 epilogue recombines them.  Only 64 of the M = 128 rows of each MMA are real:
// the other 64 rows of the A operand are whatever shared memory follows it (always inside this
// block's allocation), and the matching TMEM lanes are never read.
//
// Shared memory fits two blocks per SM (about 113 KB each), so one block's FP64 panel work
// overlaps the other's tensor-core products; each block holds 256 TMEM columns.
#include "factor_kernels.h"
#include "factor_chain.cuh"
#include "ozaki_pass.cuh"
#include "bf16x3_pass.cuh"

namespace tsqr {
namespace blk {

constexpr int NP = 64;           // padded column count
constexpr int H = 64;            // leaf height (bottom rows of the tile)
constexpr int NB = 16;           // panel width
constexpr uint32_t kTmemCols = 256;

// Stage area (byte offsets; every operand buffer 1024-byte aligned for the 128-byte swizzle).
//   W product : A slice buffer [0, 8K) (rows 64..127 of the MMA read the B slices after it),
//               B slices [8K, 24K) (8 x 2 KB); afterwards W (16 x 48 FP64) at [0, 6K).
//   update    : A buffers [0, 8K) and [8K, 16K) (4 slices per 128-byte row, 32 bytes each),
//               B buffers [16K, 22K) and [22K, 28K) (likewise).
//   FP64 work between products: X (merge scratch) [8K, 16K), red [16K, 18K), dvec, wvec, invs.
constexpr uint32_t kStA = 0;
constexpr uint32_t kStWB = 8192;
constexpr uint32_t kStW = 0;
constexpr uint32_t kStUA0 = 0;
constexpr uint32_t kStUA1 = 8192;
constexpr uint32_t kStUB0 = 16384;
constexpr uint32_t kStUB1 = 22528;
constexpr uint32_t kStX = 8192;
constexpr uint32_t kStRed = 16384;
constexpr uint32_t kStDvec = 18432;
constexpr uint32_t kStWvec = 18944;
constexpr uint32_t kStInvs = 19456;
constexpr uint32_t kStageBytes = 28672;

constexpr uint32_t kTileBytes = (NP + H) * NP * 8;              // 64 KB
constexpr uint32_t kOffTile = kStageBytes;
constexpr uint32_t kOffT = kOffTile + kTileBytes;                // packed T (tri_size(64) doubles)
constexpr uint32_t kOffTau = kOffT + 2080 * 8;
constexpr uint32_t kOffSc = kOffTau + NP * 8;
constexpr uint32_t kOffExpA = kOffSc + 8 * 8;                     // 64 ints: tile column exponents
constexpr uint32_t kOffExpU = kOffExpA + NP * 4;                  // 64 ints: V_bot row exponents
constexpr uint32_t kOffExpW = kOffExpU + NP * 4;                  // 64 ints: W' column exponents
constexpr uint32_t kOffBar = kOffExpW + NP * 4;                   // 1 mbarrier + TMA barrier
constexpr uint32_t kOffSlot = kOffBar + 16;
constexpr uint32_t kOffFlag = kOffSlot + 4;
constexpr uint32_t kSmemBytes = 1024 + kOffFlag + 8;

struct Smem {
  char* stage;
  uint64_t* mma_bar;
  uint32_t* slot;
  int *expA, *expU, *expW;
};

// Fixed-point bf16 slice s (1-based) of a value already in fixed-point form: the 16-bit pattern.
__device__ __forceinline__ uint32_t slice16(uint64_t fx, int s) { return slice_pair(fx, 0ull, s) & 0xFFFFu; }

// Bounded wait of every thread on the MMA barrier (thread 0 waits, the block learns the outcome).
__device__ inline bool mma_wait(const Smem& z, uint32_t& phase, int* status, int* flag) {
  if (threadIdx.x == 0) {
    const bool ok = oz::wait_bar(z.mma_bar, phase);
    *flag = ok ? 0 : 1;
    if (!ok) atomicOr(status, kStatusTimeout);
  }
  phase ^= 1u;
  __syncthreads();
  oz::fence_after_sync();
  return *flag == 0;
}




// T of the compact-WY form over columns [c0, c1), in place in the packed T_s, by blocked merges
// T = [T1, -T1 G12 T2; 0, T2] at block sizes b = bmin, 2 bmin, ... < bmax: T_s holds tau on the
// diagonal, the merged blocks of size bmin on the diagonal and the Gram entries v_c^T v_j above
// them.  X holds (c1 - c0) * bmax / 2 entries.  All threads call.
template <class Ar>
__device__ inline void merge_t(typename Ar::E* T_s, typename Ar::E* X, int c0, int c1, int bmin, int bmax) {
  using E = typename Ar::E;
  const int tid = threadIdx.x;
  const int w = c1 - c0;
  for (int b = bmin, lb = __ffs(bmin) - 1; b < bmax && b < w; b <<= 1, ++lb) {
    const int pairs = (w + 2 * b - 1) >> (lb + 1);
    // X = G12 T2 for every pair; the row i varies fastest so a warp's loop lengths agree
    for (int o = tid; o < (pairs << (2 * lb)); o += kThreads) {
      const int k = o >> (2 * lb), qq = (o >> lb) & (b - 1), i = o & (b - 1);
      const int r1 = c0 + 2 * b * k + i, c2 = c0 + 2 * b * k + b + qq;
      E v = Ar::zero();
      if (r1 < c1 && c2 < c1) {
        for (int p = c0 + 2 * b * k + b; p <= c2; ++p)
          Ar::fma_acc(v, T_s[tri_off(r1, NP) + (p - r1)], T_s[tri_off(p, NP) + (c2 - p)]);
      }
      X[(k * b + i) * b + qq] = Ar::fin(v);
    }
    __syncthreads();
    // T12 = -T1 X
    for (int o = tid; o < (pairs << (2 * lb)); o += kThreads) {
      const int k = o >> (2 * lb), i = (o >> lb) & (b - 1), qq = o & (b - 1);
      const int r1 = c0 + 2 * b * k + i, c2 = c0 + 2 * b * k + b + qq;
      if (r1 < c1 && c2 < c1) {
        E v = Ar::zero();
        for (int p = r1; p < c0 + 2 * b * k + b; ++p)
          Ar::fma_acc(v, T_s[tri_off(r1, NP) + (p - r1)], X[(k * b + (p - c0 - 2 * b * k)) * b + qq]);
        T_s[tri_off(r1, NP) + (c2 - r1)] = Ar::neg(Ar::fin(v));
      }
    }
    __syncthreads();
  }
}

// merge_t for one panel (c1 - c0 <= 16, bmax <= 16) by the 32 lanes of one warp, with warp
// barriers only.  X holds 64 entries.  Only the calling warp takes part.
template <class Ar>
__device__ inline void merge_t_warp(typename Ar::E* T_s, typename Ar::E* X, int c0, int c1, int bmax) {
  using E = typename Ar::E;
  const int lane = threadIdx.x & 31;
  const int w = c1 - c0;
  for (int b = 1, lb = 0; b < bmax && b < w; b <<= 1, ++lb) {
    const int pairs = (w + 2 * b - 1) >> (lb + 1);
    for (int o = lane; o < (pairs << (2 * lb)); o += 32) {
      const int k = o >> (2 * lb), qq = (o >> lb) & (b - 1), i = o & (b - 1);
      const int r1 = c0 + 2 * b * k + i, c2 = c0 + 2 * b * k + b + qq;
      E v = Ar::zero();
      if (r1 < c1 && c2 < c1) {
        for (int p = c0 + 2 * b * k + b; p <= c2; ++p)
          Ar::fma_acc(v, T_s[tri_off(r1, NP) + (p - r1)], T_s[tri_off(p, NP) + (c2 - p)]);
      }
      X[(k * b + i) * b + qq] = Ar::fin(v);
    }
    __syncwarp();
    for (int o = lane; o < (pairs << (2 * lb)); o += 32) {
      const int k = o >> (2 * lb), i = (o >> lb) & (b - 1), qq = o & (b - 1);
      const int r1 = c0 + 2 * b * k + i, c2 = c0 + 2 * b * k + b + qq;
      if (r1 < c1 && c2 < c1) {
        E v = Ar::zero();
        for (int p = r1; p < c0 + 2 * b * k + b; ++p)
          Ar::fma_acc(v, T_s[tri_off(r1, NP) + (p - r1)], X[(k * b + (p - c0 - 2 * b * k)) * b + qq]);
        T_s[tri_off(r1, NP) + (c2 - r1)] = Ar::neg(Ar::fin(v));
      }
    }
    __syncwarp();
  }
}

// Reduce-scatter of W partial sums across the 32 lanes of a warp (W = 16 or 8): on return lane l
// holds in x[0] the warp-wide sum of entry (l >> 1) (W = 16) or (l >> 2) (W = 8).  Each round
// halves the entries a lane keeps, so the W sums cost W native FP64 adds in all.
template <int W>
__device__ __forceinline__ void reduce_scatter(double (&x)[16], int lane) {
  int len = W;
#pragma unroll
  for (int o = 16; o >= 2 && len > 1; o >>= 1) {
    const bool hi = (lane & o) != 0;
    len >>= 1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i < len) {
        const double send = hi ? x[i] : x[i + len];
        const double keep = hi ? x[i + len] : x[i];
        x[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
  }
  // the lanes that share an entry add their halves
#pragma unroll
  for (int o = (W == 16 ? 1 : 2); o >= 1; o >>= 1) x[0] += __shfl_xor_sync(0xffffffffu, x[0], o);
}

// Column JJ of panel_qr_warp (below): its reflector, then the dot products with the panel's
// columns (all 16 while JJ is in the first half, the second half's 8 after that), the pivot-row
// update and the column update.  Compile-time JJ keeps every register index static.
template <int JJ>
__device__ __forceinline__ void panel_column(const Tile& S, int c0, int jn, double (&a0)[16], double (&a1)[16],
                                             double* tau_s, double* T_s, int lane) {
  if (JJ >= jn) return;
  const int j = c0 + JJ;
  const double x0 = a0[JJ], x1 = a1[JJ];
  const double alpha = *S.ptr(j, j);
  double ss = fma(x1, x1, x0 * x0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  ss = __shfl_sync(0xffffffffu, ss, 0);  // one value for every lane
  const bool nz = __any_sync(0xffffffffu, ((((unsigned long long)__double_as_longlong(x0)) << 1) |
                                           (((unsigned long long)__double_as_longlong(x1)) << 1)) != 0ull);
  double beta = alpha, tau = 0.0, inv = 0.0;
  if (nz) {
    const double full = fma(alpha, alpha, ss);
    const bool normal = full >= 0x1p-900 && full <= 0x1p+900;
    double nrm;
    if (normal) {
      nrm = sqrt(full);
    } else {  // rescale by the largest magnitude (keeps NaN)
      // NaN-propagating max, the same on every lane, so the branch below stays warp-uniform
      double mx = max_nan(fabs(alpha), max_nan(fabs(x0), fabs(x1)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max_nan(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (mx == 0.0 || !(mx <= 1.7976931348623157e308)) {
        nrm = mx;
      } else {
        const double t0 = alpha / mx, u0 = x0 / mx, u1 = x1 / mx;
        double s2 = fma(u1, u1, u0 * u0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s2 = __shfl_sync(0xffffffffu, s2, 0);
        nrm = mx * sqrt(fma(t0, t0, s2));
      }
    }
    beta = (alpha >= 0.0) ? -nrm : nrm;
    const double d = alpha - beta;  // |d| = |alpha| + |beta|
    if (normal) {
      const double qd = 1.0 / (beta * d);  // one division; |beta d| in [full, 2 full]
      inv = beta * qd;
      tau = -(d * d) * qd;
    } else {
      tau = (beta - alpha) / beta;
      inv = 1.0 / d;
    }
  }
  if (lane == 0) {
    if (nz) *S.ptr(j, j) = beta;
    tau_s[j] = tau;
    T_s[tri_off(j, NP)] = tau;
  }
  if (!nz) return;  // H_j = I: no update, and its Gram entries stay zero
  const double v0 = x0 * inv, v1 = x1 * inv;
  a0[JJ] = v0;
  a1[JJ] = v1;
  constexpr int kW = (JJ < 8) ? 16 : 8;
  constexpr int kB = 16 - kW;
  double x[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = (i < kW) ? fma(v1, a1[kB + i], v0 * a0[kB + i]) : 0.0;
  reduce_scatter<kW>(x, lane);
  const int cl = kB + ((kW == 16) ? (lane >> 1) : (lane >> 2));  // this lane's panel column
  const bool leader = (lane & (kW == 16 ? 1 : 3)) == 0;
  double w = 0.0;
  if (cl > JJ && cl < jn) {
    double& pr = *S.ptr(j, c0 + cl);
    const double dd = pr + x[0];
    w = tau * dd;
    if (leader) pr = fma(-tau, dd, pr);
  } else if (cl < JJ && leader) {
    T_s[tri_off(c0 + cl, NP) + (JJ - cl)] = x[0];  // Gram entry v_cl^T v_JJ
  }
#pragma unroll
  for (int c = JJ + 1; c < 16; ++c) {
    const double wc = __shfl_sync(0xffffffffu, w, (kW == 16) ? 2 * c : 4 * (c - kB));
    a0[c] = fma(-wc, v0, a0[c]);
    a1[c] = fma(-wc, v1, a1[c]);
  }
}

template <int JJ>
struct PanelColumns {
  __device__ __forceinline__ static void run(const Tile& S, int c0, int jn, double (&a0)[16], double (&a1)[16],
                                             double* tau_s, double* T_s, int lane) {
    panel_column<JJ>(S, c0, jn, a0, a1, tau_s, T_s, lane);
    PanelColumns<JJ + 1>::run(S, c0, jn, a0, a1, tau_s, T_s, lane);
  }
};
template <>
struct PanelColumns<16> {
  __device__ __forceinline__ static void run(const Tile&, int, int, double (&)[16], double (&)[16], double*, double*,
                                             int) {}
};

// The reflectors of the panel's columns [c0, c0 + jn) of [R; A_k] (R in tile rows 0..63, A_k in
// rows 64..127), taken by warp 0 alone with the panel's 64 x 16 bottom block in registers (lane l
// holds rows l and l + 32): for each column j the reflector (beta = -sign(alpha) ||x||,
// tau = (beta - alpha) / beta, v = x / (alpha - beta), as the other steps take it), the dot
// products d_c = S(j, c) + v^T S_bot(:, c) of the panel columns right of j, the pivot-row update
// S(j, c) -= tau d_c and the column update S_bot(:, c) -= tau d_c v.  The same dot products with
// the columns left of j are the Gram entries v_c^T v_j that T is built from; for j in the panel's
// second half only its second half is visited (the W product supplies the rest).  Native FP64;
// no block barrier.  Only warp 0 calls.
__device__ inline void panel_qr_warp(const Tile& S, int c0, int jn, double* tau_s, double* T_s) {
  const int lane = threadIdx.x & 31;
  double a0[16], a1[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    a0[c] = *S.ptr(NP + lane, c0 + c);
    a1[c] = *S.ptr(NP + 32 + lane, c0 + c);
  }
  PanelColumns<0>::run(S, c0, jn, a0, a1, tau_s, T_s, lane);
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    if (c < jn) {
      *S.ptr(NP + lane, c0 + c) = a0[c];
      *S.ptr(NP + 32 + lane, c0 + c) = a1[c];
    }
  }
}

// Fixed-point value of tile entry (r, c) of the bottom block against exponent e.
__device__ __forceinline__ uint64_t bot_fixed(const Tile& S, int r, int c, int e) {
  return oz::to_fixed(*S.ptr(NP + r, c), e);
}

// Value of a recombined accumulator: X * 2^(ea + eb - 2100), NaN if either operand row/column held
// an Inf or NaN (exponent field 2047), which fixed point cannot carry.
__device__ __forceinline__ double ozaki_value(long long X, int ea, int eb) {
  if (ea == 2047 || eb == 2047) return __longlong_as_double(0x7FF8000000000000LL);
  return oz::int_to_f64_scaled(X, ea + eb - 2100);
}

// Step 2: D = S_bot^T V_q (64 x 16, K = the 64 bottom rows) as one Ozaki product.  Rows c of D:
// c < 16q + j gives the Gram entry v_c^T v_{16q+j} (into T_s); c >= 16(q+1) gives
// W[j][c - 16(q+1)] = S(16q + j, c) + D[c][j] (into the stage at kStW).  False on timeout.
__device__ inline bool w_product(const Tile& S, const Smem& z, int q, double* T_s, uint32_t tmem, uint32_t& phase,
                                 int* status, int* flag) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  char* abuf = z.stage + kStA;
  char* bsl = z.stage + kStWB;
  // column exponents over the 64 bottom rows (one shared atomic per warp: 64 consecutive idx share c)
  for (int c = tid; c < NP; c += kThreads) z.expA[c] = 0;
  __syncthreads();
  for (int idx = tid; idx < NP * H; idx += kThreads) warp_max_into(&z.expA[idx >> 6], oz::bexp(*S.ptr(NP + (idx & 63), idx >> 6)));
  __syncthreads();
  // B: V_q as 16 rows (its columns) x K = 64 rows, all 8 slices
  for (int idx = tid; idx < NB * 32; idx += kThreads) {
    const int j = idx >> 5, r = (idx & 31) * 2;
    const int c = NB * q + j, e = z.expA[c];
    const uint64_t f0 = bot_fixed(S, r, c, e), f1 = bot_fixed(S, r + 1, c, e);
#pragma unroll
    for (int t = 1; t <= oz::kSlices; ++t)
      *reinterpret_cast<uint32_t*>(bsl + (t - 1) * 2048 + oz::op_off(j, r)) = slice_pair(f0, f1, t);
  }
  // A = S_bot^T (64 rows = tile columns, K = 64 bottom rows): each thread's 8 entry pairs in fixed
  // point once, kept in registers for the 8 slices
  constexpr int kItems = NP * 32 / kThreads;
  uint64_t fx[kItems][2];
#pragma unroll
  for (int u = 0; u < kItems; ++u) {
    const int idx = tid + u * kThreads;
    const int c = idx >> 5, r = (idx & 31) * 2;
    const int e = z.expA[c];
    fx[u][0] = bot_fixed(S, r, c, e);
    fx[u][1] = bot_fixed(S, r + 1, c, e);
  }
  for (int s = 1; s <= oz::kSlices; ++s) {
    if (s > 1 && !mma_wait(z, phase, status, flag)) return false;
#pragma unroll
    for (int u = 0; u < kItems; ++u) {
      const int idx = tid + u * kThreads;
      *reinterpret_cast<uint32_t*>(abuf + oz::op_off(idx >> 5, (idx & 31) * 2)) = slice_pair(fx[u][0], fx[u][1], s);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      oz::fence_after_sync();
      // the B slices t = 1 .. 9 - s lie one after another, as do their groups s + t - 2 in TMEM:
      // one MMA of N = 16 (9 - s) per K step
      const uint64_t adesc = oz::sw128_desc(smem_u32(abuf));
      const uint32_t d = tmem + (uint32_t)(s - 1) * NB;
      const uint64_t bdesc = oz::sw128_desc(smem_u32(bsl));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        oz::mma_bf16(d, adesc + 2 * kk, bdesc + 2 * kk, oz::idesc_bf16(128, (uint32_t)(NB * (oz::kSlices + 1 - s))),
                     (s > 1 || kk > 0) ? 1u : 0u);
      oz::mma_commit(z.mma_bar);
    }
  }
  if (!mma_wait(z, phase, status, flag)) return false;
  // epilogue: warps 0, 1, 4, 5 hold TMEM lanes 0..63 (rows c); warp >> 2 picks 8 of the 16 columns
  double* W = reinterpret_cast<double*>(z.stage + kStW);
  if ((warp & 3) < 2) {
    const int c = 32 * (warp & 3) + lane;
    const int j0 = 8 * (warp >> 2);
    long long acc[8];
    oz::load_groups<8>(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)j0, NB, acc);
    const int c1 = NB * (q + 1);
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int col = NB * q + j0 + jj;
      const double v = ozaki_value(acc[jj], z.expA[c], z.expA[col]);
      // Gram entries the panel's own dot products did not visit: earlier panels' columns, and
      // the panel's first half against its second half
      if (c < col && (c < NB * q || (c < NB * q + 8 && col >= NB * q + 8)))
        T_s[tri_off(c, NP) + (col - c)] = v;
      else if (c >= c1)
        W[(j0 + jj) * 48 + (c - c1)] = v + *S.ptr(col, c);
    }
  }
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  return true;
}

// Step 3: W' = T_q^T W (16 x nc) in place in the stage, and C_top -= W' on the panel's pivot rows.
__device__ inline void w_prime(const Tile& S, const Smem& z, int q, const double* T_s) {
  const int tid = threadIdx.x;
  const int c1 = NB * (q + 1), nc = NP - c1;
  double* W = reinterpret_cast<double*>(z.stage + kStW);
  double out[3];
  const int total = NB * nc;  // <= 768 = 3 per thread
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int o = tid + u * kThreads;
    double v = 0.0;
    if (o < total) {
      const int i = o / nc, c = o - i * nc;
      const int ri = NB * q + i;
      for (int k = 0; k <= i; ++k) v = fma(T_s[tri_off(NB * q + k, NP) + (ri - NB * q - k)], W[k * 48 + c], v);
    }
    out[u] = v;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int o = tid + u * kThreads;
    if (o < total) {
      const int i = o / nc, c = o - i * nc;
      W[i * 48 + c] = out[u];
      double& top = *S.ptr(NB * q + i, c1 + c);
      top -= out[u];
    }
  }
  __syncthreads();
}

// Step 4: C_bot(:, 16(q+1):) -= V_bot W' as one Ozaki product per chunk of <= 32 columns
// (K = the 16 panel columns; 4 slices side by side in each 128-byte operand row).  False on timeout.
__device__ inline bool update_product(const Tile& S, const Smem& z, int q, uint32_t tmem, uint32_t& phase,
                                      int* status, int* flag) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c1 = NB * (q + 1), nc = NP - c1;
  const double* W = reinterpret_cast<const double*>(z.stage + kStW);
  // exponents: W' columns over its 16 rows, V_bot rows over the 16 panel columns
  for (int c = tid; c < NP; c += kThreads) {
    z.expW[c] = 0;
    z.expU[c] = 0;
  }
  __syncthreads();
  for (int idx = tid; idx < NB * nc; idx += kThreads) {
    const int c = idx % nc, i = idx / nc;
    atomicMax(&z.expW[c], oz::bexp(W[i * 48 + c]));
  }
  for (int idx = tid; idx < H * NB; idx += kThreads) {
    const int r = idx >> 4, i = idx & 15;
    atomicMax(&z.expU[r], oz::bexp(*S.ptr(NP + r, NB * q + i)));
  }
  __syncthreads();
  // B: W'^T, nc rows x K = 16, slice t at K offset 16 ((t - 1) & 3) of buffer (t - 1) >> 2
  for (int idx = tid; idx < nc * 8; idx += kThreads) {
    const int c = idx >> 3, i = (idx & 7) * 2;
    const int e = z.expW[c];
    const uint64_t f0 = oz::to_fixed(W[i * 48 + c], e), f1 = oz::to_fixed(W[(i + 1) * 48 + c], e);
#pragma unroll
    for (int t = 1; t <= oz::kSlices; ++t)
      *reinterpret_cast<uint32_t*>(z.stage + (t <= 4 ? kStUB0 : kStUB1) + oz::op_off(c, 16 * ((t - 1) & 3) + i)) =
          slice_pair(f0, f1, t);
  }
  __syncthreads();  // W' (over the A buffers) is read; the A slices may be written
  // A: V_bot, 64 rows x K = 16
  for (int idx = tid; idx < H * 8; idx += kThreads) {
    const int r = idx >> 3, i = (idx & 7) * 2;
    const int e = z.expU[r];
    const uint64_t f0 = bot_fixed(S, r, NB * q + i, e), f1 = bot_fixed(S, r, NB * q + i + 1, e);
#pragma unroll
    for (int s = 1; s <= oz::kSlices; ++s)
      *reinterpret_cast<uint32_t*>(z.stage + (s <= 4 ? kStUA0 : kStUA1) + oz::op_off(r, 16 * ((s - 1) & 3) + i)) =
          slice_pair(f0, f1, s);
  }
  fence_proxy_async_smem();
  __syncthreads();
  for (int c0 = 0; c0 < nc; c0 += 32) {
    const int N = (nc - c0 < 32) ? nc - c0 : 32;
    if (tid == 0) {
      oz::fence_after_sync();
      const uint32_t idesc = oz::idesc_bf16(128, (uint32_t)N);
      for (int s = 1; s <= oz::kSlices; ++s) {
        const uint64_t adesc = oz::sw128_desc(smem_u32(z.stage + (s <= 4 ? kStUA0 : kStUA1))) + 2 * ((s - 1) & 3);
        for (int t = 1; t <= oz::kSlices + 1 - s; ++t) {
          const uint64_t bdesc =
              oz::sw128_desc(smem_u32(z.stage + (t <= 4 ? kStUB0 : kStUB1) + c0 * 128)) + 2 * ((t - 1) & 3);
          oz::mma_bf16(tmem + (uint32_t)(s + t - 2) * 32u, adesc, bdesc, idesc, s > 1 ? 1u : 0u);
        }
      }
      oz::mma_commit(z.mma_bar);
    }
    if (!mma_wait(z, phase, status, flag)) return false;
    // epilogue: warps 0, 1, 4, 5 hold rows r = 0..63; warp >> 2 picks half of the N columns
    if ((warp & 3) < 2) {
      const int r = 32 * (warp & 3) + lane;
      const int er = z.expU[r];
      for (int o = (warp >> 2) * (N / 2); o < (warp >> 2) * (N / 2) + N / 2; o += 8) {
        long long acc[8];
        oz::load_groups<8>(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)o, 32, acc);
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int c = c0 + o + jj;
          double& a = *S.ptr(NP + r, c1 + c);
          a -= ozaki_value(acc[jj], er, z.expW[c]);
        }
      }
    }
    oz::fence_before_sync();
    __syncthreads();
    oz::fence_after_sync();
  }
  return true;
}


// The blocked step QR([R; A_k]) on the tile: panels of 16 columns (steps 1-4 above), then the
// merge of the panels' T blocks into the leaf's T.  False on a timed-out wait.
__device__ inline bool blocked_step(const FactorSmem<double>& f, const Plan& P, const Smem& z, uint32_t tmem,
                                    uint32_t& phase, int* status) {
  const int tid = threadIdx.x;
  const int n = P.n;
  // T starts at zero so that columns past n contribute nothing to W' and T stays zero there
  for (int i = tid; i < tri_size(NP); i += kThreads) f.T_s[i] = 0.0;
  for (int j = n + tid; j < NP; j += kThreads) f.tau_s[j] = 0.0;
  __syncthreads();
  for (int q = 0; q < NP / NB && NB * q < n; ++q) {
    const int j0 = NB * q, j1 = min(j0 + NB, n);
    if (tid < 32) panel_qr_warp(f.S, j0, j1 - j0, f.tau_s, f.T_s);
    __syncthreads();
    if (!w_product(f.S, z, q, f.T_s, tmem, phase, status, f.flag)) return false;
    if (tid < 32) merge_t_warp<ArithF64>(f.T_s, f.X, j0, j1, NB);
    __syncthreads();
    if (NB * (q + 1) < n) {
      w_prime(f.S, z, q, f.T_s);
      if (!update_product(f.S, z, q, tmem, phase, status, f.flag)) return false;
    }
  }
  if (!P.r_only) merge_t<ArithF64>(f.T_s, f.X, 0, n, NB, NP);  // R alone needs only the panels' T blocks
  return true;
}

// ---------------------------------------------------------------------------------------------
// FP32 storage: the same blocked step with the FP32 arithmetic policy (every value the hi half of
// an 8-byte slot) and the WY products as bf16x3 term products (bf16x3_pass.cuh): each FP32 value
// split into three bf16 terms, the six term products of weight >= 2^-16 accumulated in one FP32
// TMEM accumulator.  The panel's reflectors run on the FP32 pipe (fast on GB300), so here the
// blocking removes most of the per-column barriers and issue work of the FP32 chain step.
namespace b32 {

// Stage (bytes; operand buffers 1024-byte aligned):
//   W product: A terms [0, 24K) (3 x 8K; the MMA's rows 64..127 of the last term read on into
//              the B terms and the tile), B terms [24K, 30K) (3 x 2K); then W (16 x 48 floats) at
//              [24K, 27K).
//   update   : A terms side by side (K offsets 0, 16, 32) in [0, 8K), B terms likewise [16K, 22K).
//   FP32 work between products: X [8K, 16K), red [16K, 18K), dvec, wvec, invs.
constexpr uint32_t kStA = 0, kStB = 24576, kStW = 24576, kStUA = 0, kStUB = 16384;
constexpr uint32_t kStX = 8192, kStRed = 16384, kStDvec = 18432, kStWvec = 18944, kStInvs = 19456;
constexpr uint32_t kStageBytes = 30720;
constexpr uint32_t kOffTile = kStageBytes;
constexpr uint32_t kOffT = kOffTile + kTileBytes;
constexpr uint32_t kOffTau = kOffT + 2080 * 8;
constexpr uint32_t kOffSc = kOffTau + NP * 8;
constexpr uint32_t kOffBar = kOffSc + 8 * 8;
constexpr uint32_t kOffSlot = kOffBar + 16;
constexpr uint32_t kOffFlag = kOffSlot + 4;
constexpr uint32_t kSmemBytes = 1024 + kOffFlag + 8;
constexpr uint32_t kTmemCols = 64;

__device__ __forceinline__ float& atf(const Tile& S, int r, int c) { return reinterpret_cast<f32x2*>(S.ptr(r, c))->hi; }

// Reduce-scatter of W float partial sums across a warp (as reduce_scatter for doubles).
template <int W>
__device__ __forceinline__ void reduce_scatter_f(float (&x)[16], int lane) {
  int len = W;
#pragma unroll
  for (int o = 16; o >= 2 && len > 1; o >>= 1) {
    const bool hi = (lane & o) != 0;
    len >>= 1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i < len) {
        const float send = hi ? x[i] : x[i + len];
        const float keep = hi ? x[i + len] : x[i];
        x[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, o));
      }
    }
  }
#pragma unroll
  for (int o = (W == 16 ? 1 : 2); o >= 1; o >>= 1) x[0] = __fadd_rn(x[0], __shfl_xor_sync(0xffffffffu, x[0], o));
}

// Column JJ of the FP32 warp panel: the reflector (the squares summed as they are while their sum
// stays in [2^-100, 2^100], else after rescaling the column by a power of two from its largest
// magnitude), then the dot products, the pivot-row update and the column update as in the FP64
// panel.
template <int JJ>
__device__ __forceinline__ void panel_column(const Tile& S, int c0, int jn, float (&a0)[16], float (&a1)[16],
                                             f32x2* tau_s, f32x2* T_s, int lane) {
  if (JJ >= jn) return;
  const int j = c0 + JJ;
  const float x0 = a0[JJ], x1 = a1[JJ];
  const float alpha = atf(S, j, j);
  float ss = __fmaf_rn(x1, x1, __fmul_rn(x0, x0));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss = __fadd_rn(ss, __shfl_xor_sync(0xffffffffu, ss, o));
  ss = __shfl_sync(0xffffffffu, ss, 0);  // one value for every lane
  const bool active = __any_sync(0xffffffffu, ((__float_as_uint(x0) | __float_as_uint(x1)) << 1) != 0u);
  float beta = alpha, tau = 0.f, inv = 0.f;
  if (active) {
    const float full = __fmaf_rn(alpha, alpha, ss);
    float nrm;
    if (full >= 0x1p-100f && full <= 0x1p+100f) {
      nrm = __fsqrt_rn(full);
    } else {  // rescale by a power of two from the largest magnitude before squaring
      float tmx = fmaxf(fabsf(x0), fabsf(x1));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tmx = fmaxf(tmx, __shfl_xor_sync(0xffffffffu, tmx, o));
      const float mx = fmaxf(tmx, fabsf(alpha));
      const int bexp = (__float_as_int(mx) >> 23) & 0xff;
      int k = 126 - bexp;  // mx * 2^k in [0.5, 1)
      k = k < -126 ? -126 : (k > 126 ? 126 : k);
      const float up = __int_as_float((127 + k) << 23);
      const float y0 = __fmul_rn(x0, up), y1 = __fmul_rn(x1, up);
      float s2 = __fmaf_rn(y1, y1, __fmul_rn(y0, y0));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s2 = __fadd_rn(s2, __shfl_xor_sync(0xffffffffu, s2, o));
      s2 = __shfl_sync(0xffffffffu, s2, 0);
      const float as = __fmul_rn(alpha, up);
      s2 = __fmaf_rn(as, as, s2);
      nrm = __fmul_rn(__fsqrt_rn(s2), __int_as_float((127 - k) << 23));
    }
    beta = alpha < 0.f ? nrm : -nrm;
    tau = __fdiv_rn(__fsub_rn(beta, alpha), beta);
    inv = __fdiv_rn(1.f, __fsub_rn(alpha, beta));
  }
  if (lane == 0) {
    if (active) atf(S, j, j) = beta;
    tau_s[j] = f32x2{tau, 0.f};
    T_s[tri_off(j, NP)] = f32x2{tau, 0.f};
  }
  if (!active) return;
  const float v0 = __fmul_rn(x0, inv), v1 = __fmul_rn(x1, inv);
  a0[JJ] = v0;
  a1[JJ] = v1;
  constexpr int kW = (JJ < 8) ? 16 : 8;
  constexpr int kB = 16 - kW;
  float x[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = (i < kW) ? __fmaf_rn(v1, a1[kB + i], __fmul_rn(v0, a0[kB + i])) : 0.f;
  reduce_scatter_f<kW>(x, lane);
  const int cl = kB + ((kW == 16) ? (lane >> 1) : (lane >> 2));
  const bool leader = (lane & (kW == 16 ? 1 : 3)) == 0;
  float w = 0.f;
  if (cl > JJ && cl < jn) {
    float& pr = atf(S, j, c0 + cl);
    const float dd = __fadd_rn(pr, x[0]);
    w = __fmul_rn(tau, dd);
    if (leader) pr = __fmaf_rn(-tau, dd, pr);
  } else if (cl < JJ && leader) {
    T_s[tri_off(c0 + cl, NP) + (JJ - cl)] = f32x2{x[0], 0.f};
  }
#pragma unroll
  for (int c = JJ + 1; c < 16; ++c) {
    const float wc = __shfl_sync(0xffffffffu, w, (kW == 16) ? 2 * c : 4 * (c - kB));
    a0[c] = __fmaf_rn(-wc, v0, a0[c]);
    a1[c] = __fmaf_rn(-wc, v1, a1[c]);
  }
}

template <int JJ>
struct PanelColumns {
  __device__ __forceinline__ static void run(const Tile& S, int c0, int jn, float (&a0)[16], float (&a1)[16],
                                             f32x2* tau_s, f32x2* T_s, int lane) {
    panel_column<JJ>(S, c0, jn, a0, a1, tau_s, T_s, lane);
    PanelColumns<JJ + 1>::run(S, c0, jn, a0, a1, tau_s, T_s, lane);
  }
};
template <>
struct PanelColumns<16> {
  __device__ __forceinline__ static void run(const Tile&, int, int, float (&)[16], float (&)[16], f32x2*, f32x2*,
                                             int) {}
};

__device__ inline void panel_qr_warp(const Tile& S, int c0, int jn, f32x2* tau_s, f32x2* T_s) {
  const int lane = threadIdx.x & 31;
  float a0[16], a1[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    a0[c] = atf(S, NP + lane, c0 + c);
    a1[c] = atf(S, NP + 32 + lane, c0 + c);
  }
  PanelColumns<0>::run(S, c0, jn, a0, a1, tau_s, T_s, lane);
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    if (c < jn) {
      atf(S, NP + lane, c0 + c) = a0[c];
      atf(S, NP + 32 + lane, c0 + c) = a1[c];
    }
  }
}

// The bf16 term bits of two FP32 values packed low | high, term s (0..2).
__device__ __forceinline__ void split_pair(float a, float b, uint32_t out[3]) {
  uint32_t ta[3], tb[3];
  bf3::split3(a, ta);
  bf3::split3(b, tb);
#pragma unroll
  for (int s = 0; s < 3; ++s) out[s] = ta[s] | (tb[s] << 16);
}

// Issues the six term products (s + t <= 2, smallest weights first) of one K-step set into the
// accumulator at tmem; thread 0 only.  adesc/bdesc give term s's descriptor; ksteps K-steps each.
template <class AD, class BD>
__device__ __forceinline__ void issue_terms(uint32_t tmem, uint32_t idesc, AD adesc, BD bdesc, int ksteps) {
  const int sa[6] = {2, 1, 0, 1, 0, 0}, sb[6] = {0, 1, 2, 0, 1, 0};
  uint32_t acc = 0;
  for (int p = 0; p < 6; ++p)
    for (int kk = 0; kk < ksteps; ++kk) {
      oz::mma_bf16(tmem, adesc(sa[p]) + 2 * kk, bdesc(sb[p]) + 2 * kk, idesc, acc);
      acc = 1;
    }
}

// Step 2 (FP32): D = S_bot^T V_q (64 x 16, K = 64) as bf16x3 term products: Gram entries into T_s,
// W[j][c - 16(q+1)] = S(16q + j, c) + D[c][j] into the stage.  False on timeout.
__device__ inline bool w_product(const Tile& S, const Smem& z, int q, f32x2* T_s, uint32_t tmem, uint32_t& phase,
                                 int* status, int* flag) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  char* const st = z.stage;
  for (int idx = tid; idx < NP * 32; idx += kThreads) {  // A: tile columns x 64 bottom rows
    const int c = idx >> 5, r = (idx & 31) * 2;
    uint32_t t[3];
    split_pair(atf(S, NP + r, c), atf(S, NP + r + 1, c), t);
#pragma unroll
    for (int s = 0; s < 3; ++s) *reinterpret_cast<uint32_t*>(st + kStA + s * 8192 + oz::op_off(c, r)) = t[s];
  }
  for (int idx = tid; idx < NB * 32; idx += kThreads) {  // B: V_q, its 16 columns x 64 bottom rows
    const int j = idx >> 5, r = (idx & 31) * 2;
    uint32_t t[3];
    split_pair(atf(S, NP + r, NB * q + j), atf(S, NP + r + 1, NB * q + j), t);
#pragma unroll
    for (int s = 0; s < 3; ++s) *reinterpret_cast<uint32_t*>(st + kStB + s * 2048 + oz::op_off(j, r)) = t[s];
  }
  fence_proxy_async_smem();
  __syncthreads();
  if (tid == 0) {
    oz::fence_after_sync();
    issue_terms(
        tmem, oz::idesc_bf16(128, NB), [&](int s) { return oz::sw128_desc(smem_u32(st + kStA + s * 8192)); },
        [&](int s) { return oz::sw128_desc(smem_u32(st + kStB + s * 2048)); }, 4);
    oz::mma_commit(z.mma_bar);
  }
  if (!mma_wait(z, phase, status, flag)) return false;
  float* W = reinterpret_cast<float*>(st + kStW);
  if ((warp & 3) < 2) {
    const int c = 32 * (warp & 3) + lane;
    const int j0 = 8 * (warp >> 2);
    uint32_t v[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)j0));
    oz::tmem_wait_ld();
    const int c1 = NB * (q + 1);
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int col = NB * q + j0 + jj;
      const float d = __uint_as_float(v[jj]);
      if (c < col && (c < NB * q || (c < NB * q + 8 && col >= NB * q + 8)))
        T_s[tri_off(c, NP) + (col - c)] = f32x2{d, 0.f};
      else if (c >= c1)
        W[(j0 + jj) * 48 + (c - c1)] = __fadd_rn(d, atf(S, col, c));
    }
  }
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  return true;
}

// Step 3 (FP32): W' = T_q^T W in place, C_top -= W'.
__device__ inline void w_prime(const Tile& S, const Smem& z, int q, const f32x2* T_s) {
  const int tid = threadIdx.x;
  const int c1 = NB * (q + 1), nc = NP - c1;
  float* W = reinterpret_cast<float*>(z.stage + kStW);
  float out[3];
  const int total = NB * nc;
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int o = tid + u * kThreads;
    float v = 0.f;
    if (o < total) {
      const int i = o / nc, c = o - i * nc;
      for (int k = 0; k <= i; ++k) v = __fmaf_rn(T_s[tri_off(NB * q + k, NP) + (i - k)].hi, W[k * 48 + c], v);
    }
    out[u] = v;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int o = tid + u * kThreads;
    if (o < total) {
      const int i = o / nc, c = o - i * nc;
      W[i * 48 + c] = out[u];
      float& top = atf(S, NB * q + i, c1 + c);
      top = __fsub_rn(top, out[u]);
    }
  }
  __syncthreads();
}

// Step 4 (FP32): C_bot(:, 16(q+1):) -= V_bot W' as bf16x3 term products (K = 16, the three terms
// side by side in each 128-byte operand row).  False on timeout.
__device__ inline bool update_product(const Tile& S, const Smem& z, int q, uint32_t tmem, uint32_t& phase,
                                      int* status, int* flag) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c1 = NB * (q + 1), nc = NP - c1;
  char* const st = z.stage;
  const float* W = reinterpret_cast<const float*>(st + kStW);
  for (int idx = tid; idx < nc * 8; idx += kThreads) {  // B: W'^T, nc rows x K = 16
    const int c = idx >> 3, i = (idx & 7) * 2;
    uint32_t t[3];
    split_pair(W[i * 48 + c], W[(i + 1) * 48 + c], t);
#pragma unroll
    for (int s = 0; s < 3; ++s) *reinterpret_cast<uint32_t*>(st + kStUB + oz::op_off(c, 16 * s + i)) = t[s];
  }
  for (int idx = tid; idx < H * 8; idx += kThreads) {  // A: V_bot, 64 rows x K = 16
    const int r = idx >> 3, i = (idx & 7) * 2;
    uint32_t t[3];
    split_pair(atf(S, NP + r, NB * q + i), atf(S, NP + r, NB * q + i + 1), t);
#pragma unroll
    for (int s = 0; s < 3; ++s) *reinterpret_cast<uint32_t*>(st + kStUA + oz::op_off(r, 16 * s + i)) = t[s];
  }
  fence_proxy_async_smem();
  __syncthreads();
  if (tid == 0) {
    oz::fence_after_sync();
    const uint64_t ad = oz::sw128_desc(smem_u32(st + kStUA)), bd = oz::sw128_desc(smem_u32(st + kStUB));
    issue_terms(
        tmem, oz::idesc_bf16(128, (uint32_t)nc), [&](int s) { return ad + 2 * s; }, [&](int s) { return bd + 2 * s; },
        1);
    oz::mma_commit(z.mma_bar);
  }
  if (!mma_wait(z, phase, status, flag)) return false;
  if ((warp & 3) < 2) {
    const int r = 32 * (warp & 3) + lane;
    const int half = nc / 2;
    for (int o = (warp >> 2) * half; o < (warp >> 2) * half + half; o += 8) {
      uint32_t v[8];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                   : "r"(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)o));
      oz::tmem_wait_ld();
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        float& a = atf(S, NP + r, c1 + o + jj);
        a = __fsub_rn(a, __uint_as_float(v[jj]));
      }
    }
  }
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  return true;
}

__device__ inline bool blocked_step(const FactorSmem<f32x2>& f, const Plan& P, const Smem& z, uint32_t tmem,
                                    uint32_t& phase, int* status) {
  const int tid = threadIdx.x;
  const int n = P.n;
  for (int i = tid; i < tri_size(NP); i += kThreads) f.T_s[i] = f32x2{0.f, 0.f};
  for (int j = n + tid; j < NP; j += kThreads) f.tau_s[j] = f32x2{0.f, 0.f};
  __syncthreads();
  for (int q = 0; q < NP / NB && NB * q < n; ++q) {
    const int j0 = NB * q, j1 = min(j0 + NB, n);
    if (tid < 32) b32::panel_qr_warp(f.S, j0, j1 - j0, f.tau_s, f.T_s);
    __syncthreads();
    if (!b32::w_product(f.S, z, q, f.T_s, tmem, phase, status, f.flag)) return false;
    if (tid < 32) merge_t_warp<ArithF32>(f.T_s, f.X, j0, j1, NB);
    __syncthreads();
    if (NB * (q + 1) < n) {
      b32::w_prime(f.S, z, q, f.T_s);
      if (!b32::update_product(f.S, z, q, tmem, phase, status, f.flag)) return false;
    }
  }
  if (!P.r_only) merge_t<ArithF32>(f.T_s, f.X, 0, n, NB, NP);
  return true;
}

}  // namespace b32

}  // namespace blk

__global__ void __launch_bounds__(kThreads, 2)
    factor_blocked_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapV,
                          const Plan P, const Store st, double* __restrict__ R_out, int64_t ldr, int box_rows) {
  using namespace blk;
  extern __shared__ char smem_raw[];
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  char* stage = base;
  FactorSmem<double> f;
  f.S = Tile{base + kOffTile, NP + H};
  f.T_s = reinterpret_cast<double*>(base + kOffT);
  f.red = reinterpret_cast<double*>(stage + kStRed);
  f.dvec = reinterpret_cast<double*>(stage + kStDvec);
  f.wvec = reinterpret_cast<double*>(stage + kStWvec);
  f.invs = reinterpret_cast<double*>(stage + kStInvs);
  f.X = reinterpret_cast<double*>(stage + kStX);
  f.sc = reinterpret_cast<double*>(base + kOffSc);
  f.tau_s = reinterpret_cast<double*>(base + kOffTau);
  f.bar = reinterpret_cast<uint64_t*>(base + kOffBar + 8);
  f.flag = reinterpret_cast<int*>(base + kOffFlag);
  Smem z;
  z.stage = stage;
  z.mma_bar = reinterpret_cast<uint64_t*>(base + kOffBar);
  z.slot = reinterpret_cast<uint32_t*>(base + kOffSlot);
  z.expA = reinterpret_cast<int*>(base + kOffExpA);
  z.expU = reinterpret_cast<int*>(base + kOffExpU);
  z.expW = reinterpret_cast<int*>(base + kOffExpW);
  if (threadIdx.x == 0) {
    mbar_init(z.mma_bar, 1);
    fence_mbar_init();
  }
  if ((threadIdx.x >> 5) == 0) oz::tmem_alloc(z.slot, kTmemCols);
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  const uint32_t tmem = *z.slot;
  uint32_t phase = 0;
  int* status = st.status;
  factor_chain<ArithF64>(&mapA, &mapV, P, st, R_out, ldr, box_rows, blockIdx.x, f,
                         [&](const FactorSmem<double>& ff, const Plan& p) {
                           return blocked_step(ff, p, z, tmem, phase, status);
                         });
  oz::fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) oz::tmem_dealloc(tmem, kTmemCols);
}

// FP32 storage: the blocked step with bf16x3 tensor-core products.
__global__ void __launch_bounds__(kThreads, 2)
    factor_blocked_f32_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapV,
                              const Plan P, const Store st, float* __restrict__ R_out, int64_t ldr, int box_rows) {
  using namespace blk;
  extern __shared__ char smem_raw[];
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  char* stage = base;
  FactorSmem<f32x2> f;
  f.S = Tile{base + b32::kOffTile, NP + H};
  f.T_s = reinterpret_cast<f32x2*>(base + b32::kOffT);
  f.red = reinterpret_cast<f32x2*>(stage + b32::kStRed);
  f.dvec = reinterpret_cast<f32x2*>(stage + b32::kStDvec);
  f.wvec = reinterpret_cast<f32x2*>(stage + b32::kStWvec);
  f.invs = reinterpret_cast<f32x2*>(stage + b32::kStInvs);
  f.X = reinterpret_cast<f32x2*>(stage + b32::kStX);
  f.sc = reinterpret_cast<f32x2*>(base + b32::kOffSc);
  f.tau_s = reinterpret_cast<f32x2*>(base + b32::kOffTau);
  f.bar = reinterpret_cast<uint64_t*>(base + b32::kOffBar + 8);
  f.flag = reinterpret_cast<int*>(base + b32::kOffFlag);
  Smem z;
  z.stage = stage;
  z.mma_bar = reinterpret_cast<uint64_t*>(base + b32::kOffBar);
  z.slot = reinterpret_cast<uint32_t*>(base + b32::kOffSlot);
  z.expA = z.expU = z.expW = nullptr;
  if (threadIdx.x == 0) {
    mbar_init(z.mma_bar, 1);
    fence_mbar_init();
  }
  if ((threadIdx.x >> 5) == 0) oz::tmem_alloc(z.slot, b32::kTmemCols);
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  const uint32_t tmem = *z.slot;
  uint32_t phase = 0;
  int* status = st.status;
  factor_chain<ArithF32>(&mapA, &mapV, P, st, R_out, ldr, box_rows, blockIdx.x, f,
                         [&](const FactorSmem<f32x2>& ff, const Plan& p) {
                           return b32::blocked_step(ff, p, z, tmem, phase, status);
                         });
  oz::fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) oz::tmem_dealloc(tmem, b32::kTmemCols);
}

bool blocked_factor_applies(const Plan& P) {
  return (P.precision == kPrecOzaki || P.precision == kPrecF32) && P.np == blk::NP && P.h == blk::H &&
         P.arity == 2 && P.rows_cap == blk::NP + blk::H;
}

cudaError_t launch_factor_blocked(const CUtensorMap& mapA, const CUtensorMap& mapV, const Plan& P, const Store& st,
                                  void* R_out, int64_t ldr, int box_rows, cudaStream_t stream) {
  const bool f32 = P.precision == kPrecF32;
  const size_t smem = f32 ? blk::b32::kSmemBytes : blk::kSmemBytes;
  cudaError_t e = f32 ? cudaFuncSetAttribute(factor_blocked_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem)
                      : cudaFuncSetAttribute(factor_blocked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(st.counters, 0, sizeof(int) * (size_t)(P.tree_nodes > 0 ? P.tree_nodes : 1), stream);
  if (e != cudaSuccess) return e;
  if (f32)
    factor_blocked_f32_kernel<<<P.chains, kThreads, smem, stream>>>(mapA, mapV, P, st, static_cast<float*>(R_out), ldr,
                                                                     box_rows);
  else
    factor_blocked_kernel<<<P.chains, kThreads, smem, stream>>>(mapA, mapV, P, st, static_cast<double*>(R_out), ldr,
                                                                 box_rows);
  return cudaGetLastError();
}

}  // namespace tsqr
