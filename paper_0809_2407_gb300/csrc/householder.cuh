// Householder QR of a stacked matrix held in a shared-memory Tile, in FP64, by one thread
// block.  One routine serves the three shapes TSQR factors (Kind in common.cuh):
//   PLAIN  a leaf block A_i                          (Algorithm 1, first step)
//   CHAIN  [R; A_k], triangle atop a full block      (Algorithm 2, loop body; Sec. 3.1)
//   NODE   [R_0; R_1; ...; R_{q-1}], q triangles      (Algorithm 1, tree step; eq. fact_2rs)
// For CHAIN and NODE the reflector of column j touches only row j of the top triangle, which
// is why the top block of V is the identity (eq. fact_2rs); for NODE it also touches only rows
// 0..j of each lower triangle, which keeps those blocks of V upper triangular and brings the
// cost of a pair down to about 2n^3/3 (Sec. 3.1).
//
// Alongside, the upper-triangular T of the compact-WY form Q = H_0 ... H_{n-1} = I - V T V^T
// (Sec. 3.1-3.2) is built column by column: T_jj = tau_j, T_{0:j,j} = -tau_j T_{0:j,0:j} g with
// g_p = v_p^T v_j.  The g_p are the same dot products over the reflector's rows as the trailing
// update's, taken against the earlier columns, so T costs one pass with the update's access
// pattern.
#pragma once

#include "common.cuh"

namespace tsqr {

// Rows of column j's reflector other than the pivot row j start at r_lo; NODE skips rows whose
// position inside their triangle is below the diagonal.
__device__ __forceinline__ int first_row(int kind, int j, int np) { return kind == PLAIN ? j + 1 : np; }
__device__ __forceinline__ bool skip_row(int kind, int r, int j, int np) {
  return kind == NODE && (r & (np - 1)) > j;
}

// Reflector of column j (x = S(j, j) and the column's rows >= r_lo), written to sc[]:
//   sc[0] = beta (new S(j, j)), sc[1] = tau, sc[2] = 1/(alpha - beta), sc[3] = 1 if H != I.
// beta = -sign(alpha) ||x||, sign(0) = +1; tau = (beta - alpha)/beta; tau = 0 when the rows
// below the pivot are all zero.  ||x|| is taken from the plain sum of squares unless that sum
// leaves [2^-900, 2^900], in which case it is recomputed with every entry scaled by the
// largest magnitude.  Warp 0 computes; ends with a block barrier.
__device__ inline void make_reflector(const Tile& S, int kind, int N, int np, int j, double* sc) {
  const int lane = threadIdx.x;
  if (lane < 32) {
    const int r_lo = first_row(kind, j, np);
    double ss = 0.0;
    for (int r = r_lo + lane; r < N; r += 32) {
      if (skip_row(kind, r, j, np)) continue;
      const double x = S(r, j);
      ss = fma(x, x, ss);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const double alpha = S(j, j);
    double beta = alpha, tau = 0.0, inv = 0.0;
    const bool active = !(ss == 0.0);
    if (active) {
      const double full = fma(alpha, alpha, ss);
      double nrm;
      if (full >= 0x1p-900 && full <= 0x1p+900) {
        nrm = sqrt(full);
      } else {
        double mx = fabs(alpha);
        for (int r = r_lo + lane; r < N; r += 32) {
          if (skip_row(kind, r, j, np)) continue;
          const double a = fabs(S(r, j));
          if (!(a <= mx)) mx = a;  // keeps NaN
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double y = __shfl_xor_sync(0xffffffffu, mx, o);
          if (!(y <= mx)) mx = y;
        }
        if (mx == 0.0 || !(mx <= 1.7976931348623157e308)) {
          nrm = mx;  // zero cannot happen here; Inf or NaN propagate
        } else {
          const double t0 = alpha / mx;
          double s = 0.0;
          for (int r = r_lo + lane; r < N; r += 32) {
            if (skip_row(kind, r, j, np)) continue;
            const double t = S(r, j) / mx;
            s = fma(t, t, s);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          nrm = mx * sqrt(fma(t0, t0, s));
        }
      }
      beta = (alpha >= 0.0) ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      inv = 1.0 / (alpha - beta);
    }
    if (lane == 0) {
      sc[0] = beta;
      sc[1] = tau;
      sc[2] = inv;
      sc[3] = active ? 1.0 : 0.0;
    }
  }
  __syncthreads();
}

// Packed upper-triangular storage of T: row i holds T[i][i..np-1] starting at tri_off(i, np).
__host__ __device__ __forceinline__ int tri_off(int i, int np) { return i * np - (i * (i - 1)) / 2; }
__host__ __device__ __forceinline__ int tri_size(int np) { return np * (np + 1) / 2; }

// QR of the stacked matrix S (rows 0..N-1, real columns 0..n-1 of np; np a power of two in
// 16..64).  On return rows 0..n-1 hold R in their upper triangle and the reflectors' entries
// below their pivots sit where the zeros were created (for CHAIN/NODE the top block's strict
// lower part stays zero; it must be zero on entry).  tau_s[0..np) receives tau (0 beyond n);
// if T_s != nullptr it receives T packed by rows (tri_off; tri_size(np) doubles, any contents
// on entry).  red needs kThreads doubles, dvec np doubles, sc 4 doubles.  All threads must call.
__device__ inline void stacked_qr(const Tile& S, int kind, int N, int np, int n, double* tau_s, double* T_s,
                                  double* red, double* dvec, double* sc) {
  const int tid = threadIdx.x;
  const int G = kThreads / np;  // row groups of the (column, group) mapping
  const int cown = tid & (np - 1);
  const int gown = tid / np;
  for (int j = tid + n; j < np; j += kThreads) tau_s[j] = 0.0;
  for (int j = 0; j < n; ++j) {
    make_reflector(S, kind, N, np, j, sc);
    const double beta = sc[0], tau = sc[1], inv = sc[2];
    const bool active = sc[3] != 0.0;
    const int r_lo = first_row(kind, j, np);
    if (active) {
      // y = x / (alpha - beta) below the pivot
      for (int r = r_lo + tid; r < N; r += kThreads) {
        if (skip_row(kind, r, j, np)) continue;
        S(r, j) *= inv;
      }
      __syncthreads();
      // d_c = S(j, c) + sum_r y_r S(r, c) for every other column: c > j gives the update's
      // inner product, c < j the Gram entry v_c^T v_j for T.
      if (cown < n && cown != j) {
        double acc = 0.0;
        for (int r = r_lo + gown; r < N; r += G) {
          if (skip_row(kind, r, j, np)) continue;
          acc = fma(S(r, j), S(r, cown), acc);
        }
        red[gown * np + cown] = acc;
      }
      __syncthreads();
      if (tid < n && tid != j) {
        double d = S(j, tid);
        for (int g = 0; g < G; ++g) d += red[g * np + tid];
        dvec[tid] = d;
        if (tid > j) S(j, tid) = fma(-tau, d, S(j, tid));
      }
      if (tid == 0) S(j, j) = beta;
      __syncthreads();
      if (T_s != nullptr && tid < j) {
        const double* Ti = T_s + tri_off(tid, np) - tid;  // Ti[p] = T[tid][p]
        double s = 0.0;
        for (int p = tid; p < j; ++p) s = fma(Ti[p], dvec[p], s);
        T_s[tri_off(tid, np) + (j - tid)] = -tau * s;
      }
      // trailing update S(r, c) -= tau d_c y_r.  Only the ac = n-1-j columns right of j take
      // part, so they are spread over all threads afresh for every j: an FP64 instruction costs
      // the same whatever its active-lane count, and a fixed column-per-lane map would leave
      // the lanes of finished columns idle.
      const int ac = n - 1 - j;
      if (ac > 0) {
        const int Gu = kThreads / ac;
        if (tid < Gu * ac) {
          const int c = j + 1 + tid % ac;
          const int gu = tid / ac;
          const double w = tau * dvec[c];
          for (int r = r_lo + gu; r < N; r += Gu) {
            if (skip_row(kind, r, j, np)) continue;
            S(r, c) = fma(-w, S(r, j), S(r, c));
          }
        }
      }
    }
    if (!active && T_s != nullptr && tid < j) T_s[tri_off(tid, np) + (j - tid)] = 0.0;
    if (tid == j) {
      if (T_s != nullptr) T_s[tri_off(j, np)] = tau;
      tau_s[j] = tau;
    }
    __syncthreads();
  }
}

}  // namespace tsqr
