// Applying the implicit Q of a TSQR factorization: explicit thin Q, Q^T B and Q B.
//
// The full Q is the product, from the leaves up, of block-diagonal factors: the chains' local
// Q's (first leaf, then the flat-tree steps) and one factor per tree level (Sec. 2, eq.
// par4:final and seq4:final).  Q^T B runs leaves -> root (a reduction); Q B and the thin Q run
// root -> leaves (a broadcast) (Sec. 4.1).  Every local factor is applied in compact-WY form
// (Sec. 3.2): with V = [I; Y] the node update is D = C0 + Y^T C1, C0 -= T^T D, C1 -= Y T^T D
// for Q^T, and the same with T in place of T^T for Q.
#include "factor_kernels.h"

namespace tsqr {

// ------------------------------------------------------------------------------------------
// small dense helpers on row-major shared matrices (leading dimension given)

// M (np x kb) = T * C (trans = false) or T^T * C (trans = true), T upper triangular n x n.
__device__ inline void tri_mul(const double* T, int ldt, const double* C, int ldc, double* M, int ldm, int n, int np,
                               int kb, bool trans) {
  for (int o = threadIdx.x; o < np * kb; o += kThreads) {
    const int a = o / kb, b = o % kb;
    double s = 0.0;
    if (a < n) {
      if (!trans) {
        for (int p = a; p < n; ++p) s = fma(T[a * ldt + p], C[p * ldc + b], s);
      } else {
        for (int p = 0; p <= a; ++p) s = fma(T[p * ldt + a], C[p * ldc + b], s);
      }
    }
    M[o / kb * ldm + b] = s;
  }
}

// Copies an np x np row-major global matrix into shared memory with leading dimension ld.
__device__ inline void load_square(const double* __restrict__ g, double* s, int np, int ld) {
  for (int i = threadIdx.x; i < np * np; i += kThreads) s[(i / np) * ld + (i % np)] = __ldcg(g + i);
}

// ------------------------------------------------------------------------------------------
// explicit thin Q

struct FormQSmem {
  Tile S;
  double *C, *M, *T, *X;
  uint64_t* bar;
  int* flag;
  int ld;
};

__device__ inline FormQSmem carve_formq(char* raw, const Plan& P) {
  FormQSmem f;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  f.S = Tile{base, P.h};
  f.ld = P.np + 1;
  f.C = reinterpret_cast<double*>(base + (size_t)P.h * P.np * 8);
  f.M = f.C + P.np * f.ld;
  f.T = f.M + P.np * f.ld;
  f.X = f.T + P.np * f.ld;
  f.bar = reinterpret_cast<uint64_t*>(f.X + P.np * f.ld);
  f.flag = reinterpret_cast<int*>(f.bar + 1);
  return f;
}

size_t formq_smem_bytes(const Plan& P) {
  return 1024 + (size_t)P.h * P.np * 8 + 4 * (size_t)P.np * (P.np + 1) * 8 + 8 + 16;
}

// Q rows of one leaf.  chain step (V = [I; Y]):  Q_rows = -Y M with M = T C, then C -= M.
// first leaf (V unit lower trapezoidal): Q_rows = [C; 0] - V (T (V_top^T C)).
__global__ void __launch_bounds__(kThreads, 1)
    formq_kernel(const __grid_constant__ CUtensorMap mapV, const Plan P, const Store st, double* __restrict__ Q,
                 int64_t ldq, int box_rows) {
  extern __shared__ char smem_raw[];
  FormQSmem f = carve_formq(smem_raw, P);
  const Tile& S = f.S;
  const int tid = threadIdx.x;
  const int np = P.np, n = P.n, h = P.h, ld = f.ld;
  const int g = blockIdx.x;
  if (tid == 0) {
    mbar_init(f.bar, 1);
    fence_mbar_init();
  }
  // C = D (signs of the root)
  for (int i = tid; i < np * np; i += kThreads) {
    const int a = i / np, b = i % np;
    f.C[a * ld + b] = (a == b && a < n) ? __ldcg(st.signs + a) : 0.0;
  }
  __syncthreads();
  uint32_t phase = 0;

  // ---- walk the tree from the root down to chain g, keeping only this chain's block
  for (int lev = P.depth; lev >= 1; --lev) {
    int idx = g;
    for (int l = 0; l < lev - 1; ++l) idx /= P.arity;
    const int s = idx % P.arity;  // position of the level-(lev-1) ancestor among its siblings
    const int node = idx / P.arity;
    const int tn = P.level_offset[lev] + node - P.chains;
    load_square(st.node_t + (size_t)tn * np * np, f.T, np, ld);
    __syncthreads();
    tri_mul(f.T, ld, f.C, ld, f.M, ld, n, np, np, false);
    __syncthreads();
    if (s == 0) {
      for (int i = tid; i < np * np; i += kThreads) f.C[(i / np) * ld + i % np] -= f.M[(i / np) * ld + i % np];
    } else {
      load_square(st.node_y + ((size_t)tn * (P.arity - 1) + (s - 1)) * np * np, f.X, np, ld);
      __syncthreads();
      // C = -Y_s M, Y_s upper triangular
      for (int o = tid; o < np * np; o += kThreads) {
        const int a = o / np, b = o % np;
        double v = 0.0;
        for (int p = a; p < n; ++p) v = fma(f.X[a * ld + p], f.M[p * ld + b], v);
        f.C[a * ld + b] = -v;
      }
    }
    __syncthreads();
  }

  // ---- unwind the chain from its last leaf to its first
  const int64_t l0 = chain_first_leaf(P, g), l1 = chain_end_leaf(P, g);
  const int G = kThreads / np;
  const int cown = tid & (np - 1), gown = tid / np;
  for (int64_t leaf = l1 - 1; leaf >= l0; --leaf) {
    const bool plain = (leaf == l0);
    const int64_t row0 = leaf * h;
    load_square(st.t_leaf + leaf * np * np, f.T, np, ld);
    if (!tile_load(S, &mapV, f.bar, phase, np, row0, h, 0, box_rows, st.status, f.flag)) return;
    const int64_t rows_valid = (P.m - row0 < h) ? (P.m - row0) : h;
    if (!plain) {
      tri_mul(f.T, ld, f.C, ld, f.M, ld, n, np, np, false);
      __syncthreads();
      if (cown < n) {
        for (int r = gown; r < rows_valid; r += G) {
          double v = 0.0;
          for (int a = 0; a < n; ++a) v = fma(S(r, a), f.M[a * ld + cown], v);
          Q[(row0 + r) * ldq + cown] = -v;
        }
      }
      for (int i = tid; i < np * np; i += kThreads) f.C[(i / np) * ld + i % np] -= f.M[(i / np) * ld + i % np];
      __syncthreads();
    } else {
      // X = V_top^T C, V_top unit lower triangular (rows 0..n-1 of the leaf)
      for (int o = tid; o < np * np; o += kThreads) {
        const int a = o / np, b = o % np;
        double v = 0.0;
        if (a < n) {
          v = f.C[a * ld + b];
          for (int r = a + 1; r < n; ++r) v = fma(S(r, a), f.C[r * ld + b], v);
        }
        f.X[a * ld + b] = v;
      }
      __syncthreads();
      tri_mul(f.T, ld, f.X, ld, f.M, ld, n, np, np, false);
      __syncthreads();
      if (cown < n) {
        for (int r = gown; r < rows_valid; r += G) {
          double v = (r < n) ? f.C[r * ld + cown] : 0.0;
          const int amax = (r < n) ? r : n;
          for (int a = 0; a < amax; ++a) v = fma(-S(r, a), f.M[a * ld + cown], v);
          if (r < n) v -= f.M[r * ld + cown];  // unit diagonal of V
          Q[(row0 + r) * ldq + cown] = v;
        }
      }
      __syncthreads();
    }
  }
}

cudaError_t launch_form_q(const CUtensorMap& mapV, const Plan& P, const Store& st, double* Q, int64_t ldq,
                          int box_rows, cudaStream_t stream) {
  const size_t smem = formq_smem_bytes(P);
  cudaError_t e = cudaFuncSetAttribute(formq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  formq_kernel<<<P.chains, kThreads, smem, stream>>>(mapV, P, st, Q, ldq, box_rows);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Q^T B and Q B on column blocks of kb columns (kb a power of two <= 32)

struct ApplySmem {
  Tile S;      // leaf reflectors, h rows
  double* B;   // max(h, arity*np) x kb
  double* C;   // np x kb: the chain's top block
  double* W;   // np x kb
  double* W2;  // np x kb
  double* T;   // np x (np+1)
  double* Y;   // np x (np+1): one tree-node block
  double* red; // kThreads
  uint64_t* bar;
  int* flag;
  int ldt, brows;
};

__device__ inline ApplySmem carve_apply(char* raw, const Plan& P, int kb) {
  ApplySmem f;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  f.S = Tile{base, P.h};
  f.brows = max(P.h, P.arity * P.np);
  f.ldt = P.np + 1;
  f.B = reinterpret_cast<double*>(base + (size_t)P.h * P.np * 8);
  f.C = f.B + (size_t)f.brows * kb;
  f.W = f.C + P.np * kb;
  f.W2 = f.W + P.np * kb;
  f.T = f.W2 + P.np * kb;
  f.Y = f.T + P.np * f.ldt;
  f.red = f.Y + P.np * f.ldt;
  f.bar = reinterpret_cast<uint64_t*>(f.red + kThreads);
  f.flag = reinterpret_cast<int*>(f.bar + 1);
  return f;
}

size_t apply_smem_bytes(const Plan& P, int kb) {
  const size_t brows = (size_t)(P.h > P.arity * P.np ? P.h : P.arity * P.np);
  return 1024 + (size_t)P.h * P.np * 8 + brows * kb * 8 + 3 * (size_t)P.np * kb * 8 + 2 * (size_t)P.np * (P.np + 1) * 8 +
         kThreads * 8 + 8 + 16;
}

// W (np x kb) = Vsum, with the row sum split over thread groups when there are few outputs:
//   plain : W[a][b] = B[a][b] + sum_{r=a+1}^{h-1} V[r][a] B[r][b]       (V unit lower trapezoidal)
//   chain : W[a][b] = C[a][b] + sum_{r=0}^{h-1}   Y[r][a] B[r][b]
__device__ inline void wy_inner(const Tile& S, bool plain, int h, int n, int np, const double* B, const double* C,
                                double* W, int kb, double* red) {
  const int OUT = np * kb;
  const int G = OUT >= kThreads ? 1 : kThreads / OUT;
  const int tid = threadIdx.x;
  for (int o0 = 0; o0 < OUT; o0 += kThreads / G) {
    const int o = o0 + tid % (kThreads / G);
    const int gg = tid / (kThreads / G);
    double acc = 0.0;
    if (o < OUT) {
      const int a = o / kb, b = o % kb;
      if (a < n) {
        const int r0 = plain ? a + 1 : 0;
        for (int r = r0 + gg; r < h; r += G) acc = fma(S(r, a), B[r * kb + b], acc);
      }
    }
    if (G == 1) {
      if (o < OUT) {
        const int a = o / kb, b = o % kb;
        W[o] = (a < n) ? acc + (plain ? B[a * kb + b] : C[a * kb + b]) : 0.0;
      }
    } else {
      red[tid] = acc;
      __syncthreads();
      if (gg == 0 && o < OUT) {
        double s = 0.0;
        for (int q = 0; q < G; ++q) s += red[q * (kThreads / G) + tid];
        const int a = o / kb, b = o % kb;
        W[o] = (a < n) ? s + (plain ? B[a * kb + b] : C[a * kb + b]) : 0.0;
      }
      __syncthreads();
    }
  }
}

// B -= V W2 (rows 0..h-1); plain: V unit lower trapezoidal; chain: V = [I; Y] so C -= W2 too.
__device__ inline void wy_update(const Tile& S, bool plain, int h, int n, int np, double* B, double* C,
                                 const double* W2, int kb) {
  for (int o = threadIdx.x; o < h * kb; o += kThreads) {
    const int r = o / kb, b = o % kb;
    double v = B[o];
    const int amax = plain ? (r < n ? r : n) : n;
    for (int a = 0; a < amax; ++a) v = fma(-S(r, a), W2[a * kb + b], v);
    if (plain && r < n) v -= W2[r * kb + b];
    B[o] = v;
  }
  if (!plain)
    for (int o = threadIdx.x; o < np * kb; o += kThreads) C[o] -= W2[o];
}

__device__ inline void load_b(const double* __restrict__ Bg, int64_t ldb, int64_t m, int64_t k, int64_t row0,
                              int rows, int64_t col0, int kb, double* Bs) {
  for (int o = threadIdx.x; o < rows * kb; o += kThreads) {
    const int r = o / kb, b = o % kb;
    const int64_t gr = row0 + r, gc = col0 + b;
    Bs[o] = (gr < m && gc < k) ? __ldcg(Bg + gr * ldb + gc) : 0.0;
  }
}
__device__ inline void store_b(double* __restrict__ Bg, int64_t ldb, int64_t m, int64_t k, int64_t row0, int r_begin,
                               int rows, int64_t col0, int kb, const double* Bs) {
  for (int o = threadIdx.x; o < (rows - r_begin) * kb; o += kThreads) {
    const int r = r_begin + o / kb, b = o % kb;
    const int64_t gr = row0 + r, gc = col0 + b;
    if (gr < m && gc < k) Bg[gr * ldb + gc] = Bs[r * kb + b];
  }
}

// Tree-node step on the stacked top blocks of the q children (child s's block at Bs rows
// s*np..s*np+n-1): D = C0 + sum_s Y_s^T C_s; W2 = T^T D (trans) or T D; C0 -= W2; C_s -= Y_s W2.
__device__ inline void node_apply(ApplySmem& f, const Plan& P, const Store& st, int tn, int q, int kb, bool trans) {
  const int np = P.np, n = P.n, ld = f.ldt, tid = threadIdx.x;
  load_square(st.node_t + (size_t)tn * np * np, f.T, np, ld);
  for (int o = tid; o < np * kb; o += kThreads) f.W[o] = f.B[o];
  __syncthreads();
  for (int s = 1; s < q; ++s) {
    load_square(st.node_y + ((size_t)tn * (P.arity - 1) + (s - 1)) * np * np, f.Y, np, ld);
    __syncthreads();
    const double* Cs = f.B + (size_t)s * np * kb;
    for (int o = tid; o < np * kb; o += kThreads) {
      const int a = o / kb, b = o % kb;
      double v = f.W[o];
      for (int r = 0; r <= a && r < n; ++r) v = fma(f.Y[r * ld + a], Cs[r * kb + b], v);
      f.W[o] = v;
    }
    __syncthreads();
  }
  tri_mul(f.T, ld, f.W, kb, f.W2, kb, n, np, kb, trans);
  __syncthreads();
  for (int o = tid; o < np * kb; o += kThreads) f.B[o] -= f.W2[o];
  for (int s = 1; s < q; ++s) {
    load_square(st.node_y + ((size_t)tn * (P.arity - 1) + (s - 1)) * np * np, f.Y, np, ld);
    __syncthreads();
    double* Cs = f.B + (size_t)s * np * kb;
    for (int o = tid; o < np * kb; o += kThreads) {
      const int a = o / kb, b = o % kb;
      double v = Cs[o];
      for (int p = a; p < n; ++p) v = fma(-f.Y[a * ld + p], f.W2[p * kb + b], v);
      Cs[o] = v;
    }
    __syncthreads();
  }
}

__device__ inline int64_t chain_top_row(const Plan& P, int g) { return chain_first_leaf(P, g) * P.h; }

// Top row of tree node (level, idx): the top row of its first chain.
__device__ inline int64_t node_top_row(const Plan& P, int level, int idx) {
  int64_t c = idx;
  for (int l = 0; l < level; ++l) c *= P.arity;
  return chain_top_row(P, (int)c);
}

// ---- Q^T B: chains leaves-first, then the tree bottom-up by last arrival, then D on the top.
__global__ void __launch_bounds__(kThreads, 1)
    apply_qt_kernel(const __grid_constant__ CUtensorMap mapV, const Plan P, const Store st, int64_t k,
                    double* __restrict__ Bg, int64_t ldb, int kb, int box_rows) {
  extern __shared__ char smem_raw[];
  ApplySmem f = carve_apply(smem_raw, P, kb);
  const int tid = threadIdx.x;
  const int np = P.np, n = P.n, h = P.h;
  const int g = blockIdx.x, cb = blockIdx.y;
  const int64_t col0 = (int64_t)cb * kb;
  if (tid == 0) {
    mbar_init(f.bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  const int64_t l0 = chain_first_leaf(P, g), l1 = chain_end_leaf(P, g);
  for (int64_t leaf = l0; leaf < l1; ++leaf) {
    const bool plain = (leaf == l0);
    const int64_t row0 = leaf * h;
    load_square(st.t_leaf + leaf * np * np, f.T, np, f.ldt);
    load_b(Bg, ldb, P.m, k, row0, h, col0, kb, f.B);
    if (!tile_load(f.S, &mapV, f.bar, phase, np, row0, h, 0, box_rows, st.status, f.flag)) return;
    wy_inner(f.S, plain, h, n, np, f.B, f.C, f.W, kb, f.red);
    __syncthreads();
    tri_mul(f.T, f.ldt, f.W, kb, f.W2, kb, n, np, kb, true);
    __syncthreads();
    wy_update(f.S, plain, h, n, np, f.B, f.C, f.W2, kb);
    __syncthreads();
    if (plain) {  // rows 0..n-1 become the chain's top block
      for (int o = tid; o < np * kb; o += kThreads) f.C[o] = (o / kb < n) ? f.B[o] : 0.0;
      store_b(Bg, ldb, P.m, k, row0, n, h, col0, kb, f.B);
    } else {
      store_b(Bg, ldb, P.m, k, row0, 0, h, col0, kb, f.B);
    }
    __syncthreads();
  }
  // publish the chain's top block
  store_b(Bg, ldb, P.m, k, chain_top_row(P, g), 0, n, col0, kb, f.C);
  int idx = g;
  for (int level = 0; level < P.depth; ++level) {
    const int parent = idx / P.arity;
    const int first = parent * P.arity;
    const int q = min(P.arity, P.level_count[level] - first);
    const int tn = P.level_offset[level + 1] + parent - P.chains;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const int prev = atomicAdd(&st.counters[(size_t)tn * kMaxColBlocks + cb], 1);
      __threadfence();
      *f.flag = (prev == q - 1) ? 1 : 0;
    }
    __syncthreads();
    if (*f.flag == 0) return;
    for (int s = 0; s < q; ++s) {
      const int64_t top = node_top_row(P, level, first + s);
      for (int o = tid; o < np * kb; o += kThreads) {
        const int a = o / kb, b = o % kb;
        const int64_t gc = col0 + b;
        f.B[(size_t)s * np * kb + o] = (a < n && gc < k) ? __ldcg(Bg + (top + a) * ldb + gc) : 0.0;
      }
    }
    __syncthreads();
    node_apply(f, P, st, tn, q, kb, true);
    __syncthreads();
    for (int s = 0; s < q; ++s)
      store_b(Bg, ldb, P.m, k, node_top_row(P, level, first + s), 0, n, col0, kb, f.B + (size_t)s * np * kb);
    idx = parent;
  }
  // root: the thin part gets the signs (the top block is C without a tree, else child 0's)
  __syncthreads();
  const double* topblk = (P.depth == 0) ? f.C : f.B;
  for (int o = tid; o < n * kb; o += kThreads) {
    const int a = o / kb, b = o % kb;
    if (col0 + b < k) Bg[(int64_t)a * ldb + col0 + b] = __ldcg(st.signs + a) * topblk[o];
  }
}

// ---- Q B, tree part: one launch per level, top-down; the root level first applies D.
__global__ void __launch_bounds__(kThreads, 1)
    apply_q_tree_kernel(const Plan P, const Store st, int level, int64_t k, double* __restrict__ Bg, int64_t ldb,
                        int kb) {
  extern __shared__ char smem_raw[];
  ApplySmem f = carve_apply(smem_raw, P, kb);
  const int tid = threadIdx.x;
  const int np = P.np, n = P.n;
  const int node = blockIdx.x, cb = blockIdx.y;
  const int64_t col0 = (int64_t)cb * kb;
  const int first = node * P.arity;
  const int q = min(P.arity, P.level_count[level - 1] - first);
  const int tn = P.level_offset[level] + node - P.chains;
  for (int s = 0; s < q; ++s) {
    const int64_t top = node_top_row(P, level - 1, first + s);
    for (int o = tid; o < np * kb; o += kThreads) {
      const int a = o / kb, b = o % kb;
      const int64_t gc = col0 + b;
      double v = (a < n && gc < k) ? Bg[(top + a) * ldb + gc] : 0.0;
      if (level == P.depth && s == 0 && a < n) v *= st.signs[a];
      f.B[(size_t)s * np * kb + o] = v;
    }
  }
  __syncthreads();
  node_apply(f, P, st, tn, q, kb, false);
  __syncthreads();
  for (int s = 0; s < q; ++s)
    store_b(Bg, ldb, P.m, k, node_top_row(P, level - 1, first + s), 0, n, col0, kb, f.B + (size_t)s * np * kb);
}

// ---- Q B, chains: last leaf first, the first leaf last.
__global__ void __launch_bounds__(kThreads, 1)
    apply_q_chain_kernel(const __grid_constant__ CUtensorMap mapV, const Plan P, const Store st, int64_t k,
                         double* __restrict__ Bg, int64_t ldb, int kb, int box_rows) {
  extern __shared__ char smem_raw[];
  ApplySmem f = carve_apply(smem_raw, P, kb);
  const int tid = threadIdx.x;
  const int np = P.np, n = P.n, h = P.h;
  const int g = blockIdx.x, cb = blockIdx.y;
  const int64_t col0 = (int64_t)cb * kb;
  if (tid == 0) {
    mbar_init(f.bar, 1);
    fence_mbar_init();
  }
  const int64_t top = chain_top_row(P, g);
  for (int o = tid; o < np * kb; o += kThreads) {
    const int a = o / kb, b = o % kb;
    const int64_t gc = col0 + b;
    double v = (a < n && gc < k) ? Bg[(top + a) * ldb + gc] : 0.0;
    if (P.depth == 0 && a < n) v *= st.signs[a];
    f.C[o] = v;
  }
  __syncthreads();
  uint32_t phase = 0;
  const int64_t l0 = chain_first_leaf(P, g), l1 = chain_end_leaf(P, g);
  for (int64_t leaf = l1 - 1; leaf >= l0; --leaf) {
    const bool plain = (leaf == l0);
    const int64_t row0 = leaf * h;
    load_square(st.t_leaf + leaf * np * np, f.T, np, f.ldt);
    load_b(Bg, ldb, P.m, k, row0, h, col0, kb, f.B);
    if (!tile_load(f.S, &mapV, f.bar, phase, np, row0, h, 0, box_rows, st.status, f.flag)) return;
    if (plain)
      for (int o = tid; o < n * kb; o += kThreads) f.B[o] = f.C[o];
    __syncthreads();
    wy_inner(f.S, plain, h, n, np, f.B, f.C, f.W, kb, f.red);
    __syncthreads();
    tri_mul(f.T, f.ldt, f.W, kb, f.W2, kb, n, np, kb, false);
    __syncthreads();
    wy_update(f.S, plain, h, n, np, f.B, f.C, f.W2, kb);
    __syncthreads();
    store_b(Bg, ldb, P.m, k, row0, 0, h, col0, kb, f.B);
    __syncthreads();
  }
}

static int pick_kb(int64_t k) {
  int kb = 1;
  while (kb < k && kb < 32) kb <<= 1;
  return kb;
}

cudaError_t launch_apply_qt(const CUtensorMap& mapV, const Plan& P, const Store& st, int64_t k, double* B,
                            int64_t ldb, int box_rows, cudaStream_t stream) {
  const int kb = pick_kb(k);
  const size_t smem = apply_smem_bytes(P, kb);
  cudaError_t e = cudaFuncSetAttribute(apply_qt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  for (int64_t c0 = 0; c0 < k; c0 += (int64_t)kb * kMaxColBlocks) {
    const int64_t kc = (k - c0 < (int64_t)kb * kMaxColBlocks) ? (k - c0) : (int64_t)kb * kMaxColBlocks;
    const int ncb = (int)((kc + kb - 1) / kb);
    e = cudaMemsetAsync(st.counters, 0, sizeof(int) * (size_t)(P.tree_nodes > 0 ? P.tree_nodes : 1) * kMaxColBlocks,
                        stream);
    if (e != cudaSuccess) return e;
    apply_qt_kernel<<<dim3(P.chains, ncb), kThreads, smem, stream>>>(mapV, P, st, kc, B + c0, ldb, kb, box_rows);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_apply_q(const CUtensorMap& mapV, const Plan& P, const Store& st, int64_t k, double* B,
                           int64_t ldb, int box_rows, cudaStream_t stream) {
  const int kb = pick_kb(k);
  const size_t smem = apply_smem_bytes(P, kb);
  cudaError_t e = cudaFuncSetAttribute(apply_q_tree_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(apply_q_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  for (int64_t c0 = 0; c0 < k; c0 += (int64_t)kb * kMaxColBlocks) {
    const int64_t kc = (k - c0 < (int64_t)kb * kMaxColBlocks) ? (k - c0) : (int64_t)kb * kMaxColBlocks;
    const int ncb = (int)((kc + kb - 1) / kb);
    for (int level = P.depth; level >= 1; --level) {
      apply_q_tree_kernel<<<dim3(P.level_count[level], ncb), kThreads, smem, stream>>>(P, st, level, kc, B + c0, ldb,
                                                                                        kb);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    apply_q_chain_kernel<<<dim3(P.chains, ncb), kThreads, smem, stream>>>(mapV, P, st, kc, B + c0, ldb, kb, box_rows);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace tsqr
