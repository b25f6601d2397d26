// The flat-tree step QR([R; A_k]) (Algorithm 2, loop body; Sec. 3.1: triangle atop a full
// block) for the default leaf shapes, scheduled for GB300.
//
// Same mathematics as stacked_qr(CHAIN): for each column j the reflector of the pivot R_jj and
// the h rows of A_k, applied to the columns right of j, with the compact-WY T.  The schedule
// differs in four ways, all aimed at the issue slots and barriers that bound this step:
//   * shapes are compile-time and the h bottom rows are walked in blocks of 8 whose swizzled
//     shared-memory offsets are precomputed per column, so inner loops do no address math;
//   * look-ahead: while warps 1..7 apply reflector j to columns j+2.., warp 0 applies it to
//     column j+1 and builds reflector j+1, so the serial norm/sqrt/division work overlaps the
//     trailing update (three barriers per column instead of five);
//   * warp 0 scales the new reflector column to v = x/(alpha-beta) right after building it,
//     inside the look-ahead, so the dot products and the Gram entries need no extra factors
//     (and no product of two tiny entries can underflow);
//   * T is assembled after the leaf from the Gram entries g_pj = v_p^T v_j by the blocked
//     Schreiber-Van Loan merge T = [T1, -T1 G12 T2; 0, T2], in parallel, instead of a
//     column recurrence on the critical path of every reflector.
// With kTc the Gram entries are not taken in the column loop at all but after it, as one
// tensor-core product V^T V (gram_tc.cuh), so the loop's dot products cover only the columns
// right of the pivot.
#pragma once

#include "householder.cuh"
#include "gram_tc.cuh"

namespace tsqr {

// Shapes with a specialised chain step: (np, h) of the default plans.
template <int NP>
struct ChainShape;
template <>
struct ChainShape<64> {
  static constexpr int H = 96;
};
template <>
struct ChainShape<32> {
  static constexpr int H = 256;
};
template <>
struct ChainShape<16> {
  static constexpr int H = 512;
};

// Byte offset of element (r, c) in a Tile with rows_cap rows (the layout of Tile::ptr).
__device__ __forceinline__ uint32_t tile_off(int rows_cap, int r, int c) {
  return (uint32_t)(c >> 4) * (uint32_t)rows_cap * 128u + (uint32_t)r * 128u +
         (((((uint32_t)c & 15u) >> 1) ^ ((uint32_t)r & 7u)) << 4) + (((uint32_t)c & 1u) << 3);
}

// Offsets of column c in the 8 rows of a block that starts at a row multiple of 8.
__device__ __forceinline__ void block_offsets(int rows_cap, int c, uint32_t off[8]) {
#pragma unroll
  for (int t = 0; t < 8; ++t) off[t] = tile_off(rows_cap, t, c);
}

// Scratch of chain_qr, in shared memory: red (kThreads), dvec, wvec, invs (NP each),
// sc (4), X (NP/2 * NP/2) for the T merges.
template <class Ar, int NP>
struct ChainScratch {
  typename Ar::E *red, *dvec, *wvec, *invs, *sc, *X;
};

// QR of [R; A_k] held in tile rows 0..NP-1 (R, strict lower part zero) and NP..NP+H-1 (A_k;
// H = the leaf height of the default plan, or the padded height of a binary tree node).
// Leaves R in rows 0..n-1, the scaled reflectors in rows NP.., tau in tau_s and, with want_t,
// T packed by rows in T_s (tri_off); without it the Gram entries and the merge are skipped (R
// alone).  All threads call.
//
// kTri: the bottom block is the upper triangle R_1 of a binary tree node (rows past NP zero), so
// the structure of eq. fact_2rs holds: column j's reflector and every column it updates are
// nonzero in bottom rows 0..j only (reflectors 0..j-1 touched rows below j of no column), and
// the dot products, Gram entries and updates visit only the 8-row blocks 0..j/8.  The skipped
// terms are products with exact zeros (in FP64 the results equal the dense step's bit for bit on
// finite data), and the structural zeros stay exactly zero even when a reflector carries Inf or
// NaN.  Every loop bound depends on j alone, never on data, and no barrier is skipped.
//
// kTc: the Gram entries come from the tensor cores after the loop (tc; its stage is the T_s, red,
// dvec and sc scratch, contiguous and free by then); R, the reflectors and tau are bitwise those
// of the step without it.  False only if a wait on the tensor cores timed out.
template <class Ar, int NP, int H = ChainShape<NP>::H, bool kTri = false, bool kTc = false>
__device__ bool chain_qr(const Tile& S, int n, typename Ar::E* tau_s, typename Ar::E* T_s,
                         const ChainScratch<Ar, NP>& w, bool want_t = true, const gram::GramTC* tc = nullptr) {
  using E = typename Ar::E;
  constexpr int NB = H / 8;            // row blocks of the bottom part
  constexpr int G = kThreads / NP;     // row groups of the dot products
  constexpr int NBG = NB / G;          // blocks per group
  static_assert(NB % G == 0, "row blocks must divide among the groups");
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int rc = S.rows_cap;
  char* const bottom = S.base + (size_t)NP * 128;  // row NP starts block 0
  E* sc = w.sc;
  const bool gram_loop = want_t && !kTc;  // Gram entries taken by the loop's dot products

  // bottom rows that can be nonzero in column c (all of them unless kTri)
  auto rows_of = [](int c) { return kTri ? (c + 1 < H ? c + 1 : H) : H; };
  // warp 0: v_c = x_c inv_c over the bottom rows, once reflector c is built
  auto scale_column = [&](int c) {
    __syncwarp();
    const E s = w.invs[c];
    const int rc_end = NP + rows_of(c);
    for (int r = NP + lane; r < rc_end; r += 32) {
      E& x = at<E>(S, r, c);
      x = Ar::mul(x, s);
    }
  };
  // reflector of column 0 before the loop
  if (warp == 0) {
    chain_reflector<Ar>(S, NP, H, 0, sc, w.invs);
    scale_column(0);
  }
  for (int j = tid + n; j < NP; j += kThreads) tau_s[j] = Ar::zero();
  __syncthreads();

  const int cown = tid & (NP - 1);
  const int gown = tid / NP;
  uint32_t oc[8];
  block_offsets(rc, cown, oc);

  for (int j = 0; j < n; ++j) {
    const E tau = sc[1];
    const bool active = !Ar::is_zero(sc[3]);
    if (tid == j) tau_s[j] = tau;
    if (gram_loop && tid == j) T_s[tri_off(j, NP)] = tau;
    if (active) {
      // ---- A: D_c = sum_r v_r a_rc over the bottom rows, every column c != j (without the
      //      loop's Gram entries only c > j).  Native FP64 without the Gram entries packs those
      //      a = n - 1 - j columns and their G row groups onto the first G a threads, so whole
      //      warps fall idle as j grows and the FP64 pipe, which charges a warp instruction
      //      whatever its active lanes, is spared; each partial sum covers the same rows in the
      //      same order, so the results do not change.  The FP32-pipe arithmetics keep the fixed
      //      mapping (their loop is bound by latency, and the packing measured slower there).
      uint32_t oj[8];
      block_offsets(rc, j, oj);
      int ca = cown, ga = gown;
      uint32_t op[8];
      bool act;
      if (gram_loop || Ar::kPrecision != 0) {
        act = cown < n && cown != j && (gram_loop || cown > j);
#pragma unroll
        for (int t = 0; t < 8; ++t) op[t] = oc[t];
      } else {
        const int a = n - 1 - j;
        act = tid < G * a;
        if (act) {
          ca = j + 1 + tid % a;
          ga = tid / a;
        }
        block_offsets(rc, ca, op);
      }
      if (act) {
        // four independent partial sums so consecutive multiply-adds do not wait on each other
        // on the FP32 pipe; FP64 keeps one: its pipe, not the latency, bounds the dots, and the
        // three adds that join four sums are FP64 instructions too
        constexpr int kAcc = Ar::kPrecision == 0 ? 1 : 4;
        E acc[4] = {Ar::zero(), Ar::zero(), Ar::zero(), Ar::zero()};
#pragma unroll
        for (int bb = 0; bb < NBG; ++bb) {
          if (kTri && ga + bb * G > (j >> 3)) continue;  // rows past j: exact zeros in v_j
          const char* pb = bottom + (size_t)(ga + bb * G) * 1024;
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const E x = *reinterpret_cast<const E*>(pb + oj[t]);
            const E a = *reinterpret_cast<const E*>(pb + op[t]);
            Ar::fma_acc(acc[t % kAcc], x, a);
          }
        }
        if constexpr (kAcc == 1)
          w.red[ga * NP + ca] = Ar::fin(acc[0]);
        else
          w.red[ga * NP + ca] = Ar::add(Ar::add(acc[0], acc[1]), Ar::add(acc[2], acc[3]));
      }
      __syncthreads();
      // ---- B: d_c = S(j,c) + D_c (c > j): pivot-row update and the update weight tau d_c;
      //         g_cj = D_c = v_c^T v_j (c < j): Gram entries for T (the top parts e_c, e_j are
      //         orthogonal)
      if (tid < n && tid != j) {
        E D = w.red[tid];
#pragma unroll
        for (int g = 1; g < G; ++g) D = Ar::add(D, w.red[g * NP + tid]);
        if (tid > j) {
          E& pr = at<E>(S, j, tid);
          const E d = Ar::add(pr, D);
          pr = Ar::axpy(pr, tau, d);
          w.wvec[tid] = Ar::mul(tau, d);
        } else if (gram_loop) {
          T_s[tri_off(tid, NP) + (j - tid)] = D;
        }
      }
      if (tid == 0) at<E>(S, j, j) = sc[0];
      __syncthreads();
      // ---- C: trailing update a_rc -= w_c v_r; warp 0 takes column j+1 and then builds and
      //         scales reflector j+1, warps 1..7 take columns j+2..n-1
      if (warp == 0) {
        if (j + 1 < n) {
          const int c = j + 1;
          const E wc = w.wvec[c];
          const int r_end = NP + rows_of(j);  // v_j is zero below
          for (int r = NP + lane; r < r_end; r += 32) {
            E& a = at<E>(S, r, c);
            a = Ar::axpy(a, wc, at<E>(S, r, j));
          }
          __syncwarp();
          chain_reflector<Ar>(S, NP, H, j + 1, sc, w.invs);
          scale_column(j + 1);
        }
      } else {
        const int ac = n - j - 2;
        if (ac > 0) {
          const int t2 = tid - 32;
          const int Gu = (kThreads - 32) / ac;
          const int gu = t2 / ac;
          if (gu < Gu) {
            const int c = j + 2 + t2 % ac;
            const E wc = w.wvec[c];
            uint32_t oa[8];
            block_offsets(rc, c, oa);
            const int nb_end = kTri ? ((j >> 3) + 1 < NB ? (j >> 3) + 1 : NB) : NB;
            for (int b = gu; b < nb_end; b += Gu) {
              char* pb = bottom + (size_t)b * 1024;
#pragma unroll
              for (int t = 0; t < 8; ++t) {
                E& a = *reinterpret_cast<E*>(pb + oa[t]);
                a = Ar::axpy(a, wc, *reinterpret_cast<const E*>(pb + oj[t]));
              }
            }
          }
        }
      }
      __syncthreads();
    } else {
      // H_j = I: no update; Gram entries with column j are zero; build reflector j+1
      if (gram_loop && tid < j) T_s[tri_off(tid, NP) + (j - tid)] = Ar::zero();
      if (warp == 0 && j + 1 < n) {
        chain_reflector<Ar>(S, NP, H, j + 1, sc, w.invs);
        scale_column(j + 1);
      }
      __syncthreads();
    }
  }

  if constexpr (kTc) {
    if (want_t && !gram::gram_ozaki<Ar, NP, H>(S, n, T_s, tau_s, w.X, *tc)) return false;
  }
  // ---- T from the Gram entries by blocked merges (sizes b = 2^lb = 1, 2, 4, ... NP/2)
  for (int b = 1, lb = 0; want_t && b < n; b <<= 1, ++lb) {
    const int pairs = (n + 2 * b - 1) >> (lb + 1);
    // X = G12 * T2 for every pair (G12 at rows blk1, cols blk2 of T_s; T2 upper).  The row i
    // varies fastest across the lanes so that the loop length (q + 1) is the same in a warp.
    for (int o = tid; o < (pairs << (2 * lb)); o += kThreads) {
      const int k = o >> (2 * lb), q = (o >> lb) & (b - 1), i = o & (b - 1);
      const int r1 = 2 * b * k + i, c2 = 2 * b * k + b + q;
      E v = Ar::zero();
      if (r1 < n && c2 < n) {
        for (int p = 2 * b * k + b; p <= c2; ++p)
          Ar::fma_acc(v, T_s[tri_off(r1, NP) + (p - r1)], T_s[tri_off(p, NP) + (c2 - p)]);
      }
      w.X[(k * b + i) * b + q] = Ar::fin(v);
    }
    __syncthreads();
    // T12 = -T1 * X
    for (int o = tid; o < (pairs << (2 * lb)); o += kThreads) {
      const int k = o >> (2 * lb), i = (o >> lb) & (b - 1), q = o & (b - 1);
      const int r1 = 2 * b * k + i, c2 = 2 * b * k + b + q;
      if (r1 < n && c2 < n) {
        E v = Ar::zero();
        for (int p = r1; p < 2 * b * k + b; ++p)
          Ar::fma_acc(v, T_s[tri_off(r1, NP) + (p - r1)], w.X[(k * b + (p - 2 * b * k)) * b + q]);
        T_s[tri_off(r1, NP) + (c2 - r1)] = Ar::neg(Ar::fin(v));
      }
    }
    __syncthreads();
  }
  return true;
}

}  // namespace tsqr
