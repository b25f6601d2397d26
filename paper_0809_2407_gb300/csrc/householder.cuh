// Householder QR of a stacked matrix held in a shared-memory Tile, by one thread block, in the
// arithmetic of policy Ar (arith.cuh).  One routine serves the three shapes TSQR factors
// (Kind in common.cuh):
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

#include "arith.cuh"
#include "common.cuh"

namespace tsqr {

template <class E>
__device__ __forceinline__ E& at(const Tile& S, int r, int c) {
  return *reinterpret_cast<E*>(S.ptr(r, c));
}

// Rows of column j's reflector other than the pivot row j start at r_lo; NODE skips rows whose
// position inside their triangle is below the diagonal.
__device__ __forceinline__ int first_row(int kind, int j, int np) { return kind == PLAIN ? j + 1 : np; }
__device__ __forceinline__ bool skip_row(int kind, int r, int j, int np) {
  return kind == NODE && (r & (np - 1)) > j;
}

// Reflector of column j (x = S(j, j) and the column's rows >= r_lo), written to sc[] by lane 0:
//   sc[0] = beta (new S(j, j)), sc[1] = tau, sc[2] = 1/(alpha - beta), sc[3] != 0 if H != I.
// beta = -sign(alpha) ||x||, sign(0) = +1; tau = (beta - alpha)/beta; tau = 0 when the rows
// below the pivot are all zero.  Called by all 32 lanes of one warp; no block barrier.
template <class Ar>
__device__ inline void reflector_warp(const Tile& S, int kind, int N, int np, int j, typename Ar::E* sc);

// max(a, b), NaN when either is NaN: unlike a comparison-and-select, the result does not depend
// on the order of the operands, so every lane of a warp reduction ends with the same value and
// the branches taken on it (which hold full-warp shuffles) stay warp-uniform.
__device__ __forceinline__ double max_nan(double a, double b) { return (a != a || b != b) ? a + b : fmax(a, b); }

// Native FP64: ||x|| from the plain sum of squares unless that sum leaves [2^-900, 2^900], in
// which case every entry is rescaled by the largest magnitude first.  Whether H = I is decided
// from the entries themselves, not from their sum of squares, which underflows to zero for
// entries below about 2^-537.
template <>
__device__ inline void reflector_warp<ArithF64>(const Tile& S, int kind, int N, int np, int j, double* sc) {
  const int lane = threadIdx.x & 31;
  {
    const int r_lo = first_row(kind, j, np);
    double ss = 0.0;
    bool nz = false;  // some entry below the pivot is nonzero (its square may underflow)
    for (int r = r_lo + lane; r < N; r += 32) {
      if (skip_row(kind, r, j, np)) continue;
      const double x = at<double>(S, r, j);
      ss = fma(x, x, ss);
      nz = nz || ((unsigned long long)__double_as_longlong(x) << 1) != 0ull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const double alpha = at<double>(S, j, j);
    double beta = alpha, tau = 0.0, inv = 0.0;
    const bool active = __any_sync(0xffffffffu, nz);
    if (active) {
      const double full = fma(alpha, alpha, ss);
      double nrm;
      if (full >= 0x1p-900 && full <= 0x1p+900) {
        nrm = sqrt(full);
      } else {
        double mx = fabs(alpha);
        for (int r = r_lo + lane; r < N; r += 32) {
          if (skip_row(kind, r, j, np)) continue;
          mx = max_nan(mx, fabs(at<double>(S, r, j)));  // keeps NaN
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          mx = max_nan(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (mx == 0.0 || !(mx <= 1.7976931348623157e308)) {
          nrm = mx;  // zero cannot happen here; Inf or NaN propagate
        } else {
          const double t0 = alpha / mx;
          double s = 0.0;
          for (int r = r_lo + lane; r < N; r += 32) {
            if (skip_row(kind, r, j, np)) continue;
            const double t = at<double>(S, r, j) / mx;
            s = fma(t, t, s);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          nrm = mx * sqrt(fma(t0, t0, s));
        }
      }
      beta = (alpha >= 0.0) ? -nrm : nrm;
      const double d = alpha - beta;  // |d| = |alpha| + |beta|, in [|beta|, 2 |beta|]
      if (full >= 0x1p-900 && full <= 0x1p+900) {
        // one division: q = 1/(beta d), with |beta d| in [full, 2 full] (no over- or underflow);
        // then 1/d = beta q and tau = (beta - alpha)/beta = -d^2 q
        const double q = 1.0 / (beta * d);
        inv = beta * q;
        tau = -(d * d) * q;
      } else {
        tau = (beta - alpha) / beta;
        inv = 1.0 / d;
      }
    }
    if (lane == 0) {
      sc[0] = beta;
      sc[1] = tau;
      sc[2] = inv;
      sc[3] = active ? 1.0 : 0.0;
    }
  }
}

// Double-float: the column is rescaled by 2^k, with k set from its largest |hi|, before the
// squares are summed, so the sum stays inside the FP32 exponent range; the square root and the
// two divisions are double-float operations.
template <>
__device__ inline void reflector_warp<ArithDF>(const Tile& S, int kind, int N, int np, int j, f32x2* sc) {
  using E = f32x2;
  const int lane = threadIdx.x & 31;
  {
    const int r_lo = first_row(kind, j, np);
    float tmx = 0.f;
    for (int r = r_lo + lane; r < N; r += 32) {
      if (skip_row(kind, r, j, np)) continue;
      tmx = fmaxf(tmx, fabsf(at<E>(S, r, j).hi));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tmx = fmaxf(tmx, __shfl_xor_sync(0xffffffffu, tmx, o));
    const E alpha = at<E>(S, j, j);
    E beta = alpha, tau = ArithDF::zero(), inv = ArithDF::zero();
    const bool active = tmx != 0.f;
    if (active) {
      const float mx = fmaxf(tmx, fabsf(alpha.hi));
      int bexp = (__float_as_int(mx) >> 23) & 0xff;  // biased exponent of the largest |hi|
      int k = 126 - bexp;                             // mx * 2^k in [0.5, 1)
      k = k < -126 ? -126 : (k > 126 ? 126 : k);
      E ss = ArithDF::zero();
      for (int r = r_lo + lane; r < N; r += 32) {
        if (skip_row(kind, r, j, np)) continue;
        const E x = ArithDF::ldexp(at<E>(S, r, j), k);
        ArithDF::fma_acc(ss, x, x);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss = ArithDF::add(ss, ArithDF::shfl_xor(ss, o));
      const E as = ArithDF::ldexp(alpha, k);
      ArithDF::fma_acc(ss, as, as);
      const E nrm = ArithDF::ldexp(ArithDF::sqrt_df(ArithDF::norm(ss)), -k);
      beta = ArithDF::is_neg(alpha) ? nrm : ArithDF::neg(nrm);
      tau = ArithDF::div_df(ArithDF::sub(beta, alpha), beta);
      inv = ArithDF::div_df(ArithDF::from_int(1), ArithDF::sub(alpha, beta));
    }
    if (lane == 0) {
      sc[0] = beta;
      sc[1] = tau;
      sc[2] = inv;
      sc[3] = active ? ArithDF::from_int(1) : ArithDF::zero();
    }
  }
}

// FP32: the column is rescaled by 2^k from its largest magnitude before the squares are summed,
// so the sum of squares cannot overflow or lose the column to underflow.
template <>
__device__ inline void reflector_warp<ArithF32>(const Tile& S, int kind, int N, int np, int j, f32x2* sc) {
  using E = f32x2;
  const int lane = threadIdx.x & 31;
  const int r_lo = first_row(kind, j, np);
  float tmx = 0.f;
  for (int r = r_lo + lane; r < N; r += 32) {
    if (skip_row(kind, r, j, np)) continue;
    tmx = fmaxf(tmx, fabsf(at<E>(S, r, j).hi));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tmx = fmaxf(tmx, __shfl_xor_sync(0xffffffffu, tmx, o));
  const float alpha = at<E>(S, j, j).hi;
  float beta = alpha, tau = 0.f, inv = 0.f;
  const bool active = tmx != 0.f;
  if (active) {
    const float mx = fmaxf(tmx, fabsf(alpha));
    const int bexp = (__float_as_int(mx) >> 23) & 0xff;
    int k = 126 - bexp;  // mx * 2^k in [0.5, 1)
    k = k < -126 ? -126 : (k > 126 ? 126 : k);
    const float up = __int_as_float((127 + k) << 23);
    float ss = 0.f;
    for (int r = r_lo + lane; r < N; r += 32) {
      if (skip_row(kind, r, j, np)) continue;
      const float x = __fmul_rn(at<E>(S, r, j).hi, up);
      ss = __fmaf_rn(x, x, ss);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss = __fadd_rn(ss, __shfl_xor_sync(0xffffffffu, ss, o));
    const float as = __fmul_rn(alpha, up);
    ss = __fmaf_rn(as, as, ss);
    const float nrm = __fmul_rn(__fsqrt_rn(ss), __int_as_float((127 - k) << 23));
    beta = alpha < 0.f ? nrm : -nrm;
    tau = __fdiv_rn(__fsub_rn(beta, alpha), beta);
    inv = __fdiv_rn(1.f, __fsub_rn(alpha, beta));
  }
  if (lane == 0) {
    sc[0] = E{beta, 0.f};
    sc[1] = E{tau, 0.f};
    sc[2] = E{inv, 0.f};
    sc[3] = E{active ? 1.f : 0.f, 0.f};
  }
}

// Warp 0 builds the reflector of column j, then the block synchronises.
template <class Ar>
__device__ inline void make_reflector(const Tile& S, int kind, int N, int np, int j, typename Ar::E* sc) {
  if (threadIdx.x < 32) reflector_warp<Ar>(S, kind, N, np, j, sc);
  __syncthreads();
}

// The reflector of column j of the stacked [R; A_k] held in rows 0..np-1 and np..np+h-1
// (one warp), also recording inv = 1/(alpha - beta) in invs[j] (zero when H = I).
template <class Ar>
__device__ inline void chain_reflector(const Tile& S, int np, int h, int j, typename Ar::E* sc,
                                       typename Ar::E* invs) {
  reflector_warp<Ar>(S, CHAIN, np + h, np, j, sc);
  __syncwarp();
  if ((threadIdx.x & 31) == 0) invs[j] = Ar::is_zero(sc[3]) ? Ar::zero() : sc[2];
}

// Packed upper-triangular storage of T: row i holds T[i][i..np-1] starting at tri_off(i, np).
__host__ __device__ __forceinline__ int tri_off(int i, int np) { return i * np - (i * (i - 1)) / 2; }
__host__ __device__ __forceinline__ int tri_size(int np) { return np * (np + 1) / 2; }

// QR of the stacked matrix S (rows 0..N-1, real columns 0..n-1 of np; np a power of two in
// 16..64).  On return rows 0..n-1 hold R in their upper triangle and the reflectors' entries
// below their pivots sit where the zeros were created (for CHAIN/NODE the top block's strict
// lower part stays zero; it must be zero on entry).  tau_s[0..np) receives tau (0 beyond n);
// if T_s != nullptr it receives T packed by rows (tri_off; tri_size(np) elements, any contents
// on entry).  red needs kThreads elements, dvec np, sc 4.  All threads must call.
template <class Ar>
__device__ inline void stacked_qr(const Tile& S, int kind, int N, int np, int n, typename Ar::E* tau_s,
                                  typename Ar::E* T_s, typename Ar::E* red, typename Ar::E* dvec,
                                  typename Ar::E* sc) {
  using E = typename Ar::E;
  const int tid = threadIdx.x;
  const int G = kThreads / np;  // row groups of the (column, group) mapping of the dot products
  const int cown = tid & (np - 1);
  const int gown = tid / np;
  for (int j = tid + n; j < np; j += kThreads) tau_s[j] = Ar::zero();
  for (int j = 0; j < n; ++j) {
    make_reflector<Ar>(S, kind, N, np, j, sc);
    const E beta = sc[0], tau = sc[1], inv = sc[2];
    const bool active = !Ar::is_zero(sc[3]);
    const int r_lo = first_row(kind, j, np);
    if (active) {
      // y = x / (alpha - beta) below the pivot
      for (int r = r_lo + tid; r < N; r += kThreads) {
        if (skip_row(kind, r, j, np)) continue;
        E& x = at<E>(S, r, j);
        x = Ar::mul(x, inv);
      }
      __syncthreads();
      // d_c = S(j, c) + sum_r y_r S(r, c) for every other column: c > j gives the update's
      // inner product, c < j the Gram entry v_c^T v_j for T.
      if (cown < n && cown != j) {
        E acc = Ar::zero();
        for (int r = r_lo + gown; r < N; r += G) {
          if (skip_row(kind, r, j, np)) continue;
          Ar::fma_acc(acc, at<E>(S, r, j), at<E>(S, r, cown));
        }
        red[gown * np + cown] = acc;
      }
      __syncthreads();
      if (tid < n && tid != j) {
        E d = at<E>(S, j, tid);
        for (int g = 0; g < G; ++g) d = Ar::add(d, red[g * np + tid]);
        dvec[tid] = d;
        if (tid > j) at<E>(S, j, tid) = Ar::axpy(at<E>(S, j, tid), tau, d);
      }
      if (tid == 0) at<E>(S, j, j) = beta;
      __syncthreads();
      if (T_s != nullptr && tid < j) {
        const E* Ti = T_s + tri_off(tid, np) - tid;  // Ti[p] = T[tid][p]
        E s = Ar::zero();
        for (int p = tid; p < j; ++p) Ar::fma_acc(s, Ti[p], dvec[p]);
        T_s[tri_off(tid, np) + (j - tid)] = Ar::neg(Ar::mul(tau, Ar::fin(s)));
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
          const E w = Ar::mul(tau, dvec[c]);
          for (int r = r_lo + gu; r < N; r += Gu) {
            if (skip_row(kind, r, j, np)) continue;
            E& a = at<E>(S, r, c);
            a = Ar::axpy(a, w, at<E>(S, r, j));
          }
        }
      }
    }
    if (!active && T_s != nullptr && tid < j) T_s[tri_off(tid, np) + (j - tid)] = Ar::zero();
    if (tid == j) {
      if (T_s != nullptr) T_s[tri_off(j, np)] = tau;
      tau_s[j] = tau;
    }
    __syncthreads();
  }
}

}  // namespace tsqr
