// Applying the implicit Q of a TSQR factorization: explicit thin Q, Q^T B and Q B.
//
// The full Q is the product, from the leaves up, of block-diagonal factors: the chains' local
// Q's (first leaf, then the flat-tree steps) and one factor per tree level (Sec. 2, eq.
// par4:final and seq4:final).  Q^T B runs leaves -> root (a reduction); Q B and the thin Q run
// root -> leaves (a broadcast) (Sec. 4.1).  Every local factor is applied in compact-WY form
// (Sec. 3.2): with V = [I; Y] the node update is D = C0 + Y^T C1, C0 -= T^T D, C1 -= Y T^T D
// for Q^T, and the same with T in place of T^T for Q.
//
// Every kernel is a template on the arithmetic policy (arith.cuh); the factors in the
// workspace are in that policy's element format, and B and Q are in the caller's type (FP64,
// or FP32 with FP32 storage) and layout.  The tensor-core chain kernels of Q^T B / Q B live in
// apply_ozaki.cu (precision modes 2 and 3) and apply_bf16x3.cu (FP32 storage); their tree
// levels run here.
#include "arith.cuh"
#include "factor_kernels.h"
#include "ozaki_pass.cuh"

namespace tsqr {

template <class E>
__device__ __forceinline__ E& tat(const Tile& S, int r, int c) {
  return *reinterpret_cast<E*>(S.ptr(r, c));
}

// Lanes per output when there are fewer outputs than threads: the largest power of two up to 8
// with outputs x lanes <= kThreads and a whole number of warps (the lanes of one output are
// adjacent and combine their partial sums with shuffles).
__device__ __forceinline__ int split_lanes(int outputs) {
  int s = 1;
  while (s < 8 && 2 * s * outputs <= kThreads && (2 * s * outputs) % 32 == 0) s *= 2;
  return s;
}

// M (np x kb) = T * C (trans = false) or T^T * C (trans = true), T upper triangular n x n.
template <class Ar>
__device__ inline void tri_mul(const typename Ar::E* T, int ldt, const typename Ar::E* C, int ldc,
                               typename Ar::E* M, int ldm, int n, int np, int kb, bool trans) {
  using E = typename Ar::E;
  const int S = split_lanes(np * kb);
  if (S == 1) {
    for (int o = threadIdx.x; o < np * kb; o += kThreads) {
      const int a = o / kb, b = o % kb;
      E s = Ar::zero();
      if (a < n) {
        if (!trans) {
          for (int p = a; p < n; ++p) Ar::fma_acc(s, T[a * ldt + p], C[p * ldc + b]);
        } else {
          for (int p = 0; p <= a; ++p) Ar::fma_acc(s, T[p * ldt + a], C[p * ldc + b]);
        }
      }
      M[a * ldm + b] = Ar::fin(s);
    }
    return;
  }
  // few outputs: S adjacent lanes per output, each a strided part of the sum (one pass)
  const int lS = __ffs(S) - 1;
  const int o0 = threadIdx.x;
  if (o0 < (np * kb) << lS) {
    const int o = o0 >> lS, part = o0 & (S - 1);
    const int a = o / kb, b = o % kb;
    E s = Ar::zero();
    if (a < n) {
      if (!trans) {
        for (int p = a + part; p < n; p += S) Ar::fma_acc(s, T[a * ldt + p], C[p * ldc + b]);
      } else {
        for (int p = part; p <= a; p += S) Ar::fma_acc(s, T[p * ldt + a], C[p * ldc + b]);
      }
    }
    s = Ar::fin(s);
    for (int off = 1; off < S; off <<= 1) s = Ar::add(s, Ar::shfl_xor(s, off));
    if (part == 0) M[a * ldm + b] = s;
  }
}

// Copies an np x np row-major matrix of 8-byte elements into shared memory (leading dim ld).
// Each thread issues its loads in batches of 8 before storing any of them, so a 64 x 64 block
// costs two memory round trips rather than one per element.
template <class E>
__device__ inline void load_square(const double* __restrict__ g, E* s, int np, int ld) {
  constexpr int kBatch = 8;
  const int total = np * np;
  for (int i0 = threadIdx.x; i0 < total; i0 += kBatch * kThreads) {
    double v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int i = i0 + u * kThreads;
      v[u] = (i < total) ? __ldcg(g + i) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int i = i0 + u * kThreads;
      if (i < total) s[(i / np) * ld + (i % np)] = *reinterpret_cast<const E*>(&v[u]);
    }
  }
}

// ------------------------------------------------------------------------------------------
// explicit thin Q

template <class E>
struct FormQSmem {
  Tile S, S2;  // the leaf tile; with double buffering a second one (the next leaf's), else S2 = S
  E *C, *M, *T;
  E* X;        // without double buffering its own block; with it, the idle tile buffer is used
  uint64_t* bar;  // one barrier per tile buffer
  int* flag;
  int ld;
  bool dbl;
};

// Maximum opt-in shared memory per block on GB300.
constexpr size_t kFormqSmemCap = 232448;

// The chain part double-buffers its leaf tile (the next leaf's tile and T load while the
// current leaf computes) when two tiles and three np x (np + 1) blocks fit, and a tile can hold
// the first leaf's scratch block X (h > np).
__host__ __device__ inline bool formq_double_buffered(const Plan& P) {
  const size_t tile = (size_t)P.h * P.np * 8, sq = (size_t)P.np * (P.np + 1) * 8;
  return P.h > P.np && 1024 + 2 * tile + 3 * sq + 2 * 8 + 16 <= kFormqSmemCap;
}

// allow_dbl: the layout of a chain kernel built with double buffering (the tree steps and the
// other chain kernels use the single-buffer layout).
template <class E>
__device__ inline FormQSmem<E> carve_formq(char* raw, const Plan& P, bool allow_dbl = false) {
  FormQSmem<E> f;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  const size_t tile = (size_t)P.h * P.np * 8;
  f.dbl = allow_dbl && formq_double_buffered(P);
  f.S = Tile{base, P.h};
  f.S2 = f.dbl ? Tile{base + tile, P.h} : f.S;
  f.ld = P.np + 1;
  f.C = reinterpret_cast<E*>(base + (f.dbl ? 2 : 1) * tile);
  f.M = f.C + P.np * f.ld;
  f.T = f.M + P.np * f.ld;
  f.X = f.dbl ? reinterpret_cast<E*>(f.S2.base) : f.T + P.np * f.ld;
  f.bar = reinterpret_cast<uint64_t*>(f.T + (f.dbl ? 1 : 2) * P.np * f.ld);
  f.flag = reinterpret_cast<int*>(f.bar + 2);
  return f;
}

size_t formq_smem_bytes(const Plan& P, bool allow_dbl) {
  const size_t tile = (size_t)P.h * P.np * 8, sq = (size_t)P.np * (P.np + 1) * 8;
  return (allow_dbl && formq_double_buffered(P)) ? 1024 + 2 * tile + 3 * sq + 2 * 8 + 16
                                                 : 1024 + tile + 4 * sq + 2 * 8 + 16;
}

// One level of the thin-Q broadcast (Sec. 4.1): node (level, idx) holds its block C of
// Q_tree [D; 0] (the root's is D) and hands child s the block of Q_node [C; 0; ...; 0]:
// C - T C for s = 0 and -Y_s T C for s >= 1 (V = [I; Y_1; ...], Sec. 3.2).  The blocks live in
// the node_r slots, which the factorization no longer needs.
template <class Ar>
__device__ __forceinline__ void formq_tree_node(const Plan& P, const Store& st, int level, int node, char* smem_raw) {
  using E = typename Ar::E;
  FormQSmem<E> f = carve_formq<E>(smem_raw, P);
  const int tid = threadIdx.x;
  const int np = P.np, n = P.n, ld = f.ld;
  const int tn = P.level_offset[level] + node - P.chains;
  E* blocks = reinterpret_cast<E*>(st.node_r);
  const E* Cn = blocks + (size_t)(P.level_offset[level] + node) * np * np;
  for (int i = tid; i < np * np; i += kThreads) {
    const int a = i / np, b = i % np;
    if (level == P.depth) {
      f.C[a * ld + b] = (a == b && a < n) ? Ar::from_f64(__ldcg(st.signs + a)) : Ar::zero();
    } else {
      const double v = __ldcg(reinterpret_cast<const double*>(Cn) + i);
      f.C[a * ld + b] = *reinterpret_cast<const E*>(&v);
    }
  }
  load_square(st.node_t + (size_t)tn * np * np, f.T, np, ld);
  __syncthreads();
  tri_mul<Ar>(f.T, ld, f.C, ld, f.M, ld, n, np, np, false);
  __syncthreads();
  const int first = node * P.arity;
  const int q = min(P.arity, P.level_count[level - 1] - first);
  for (int s = 0; s < q; ++s) {
    E* out = blocks + (size_t)(P.level_offset[level - 1] + first + s) * np * np;
    if (s == 0) {
      for (int i = tid; i < np * np; i += kThreads) {
        const int o = (i / np) * ld + i % np;
        out[i] = Ar::sub(f.C[o], f.M[o]);
      }
    } else {
      load_square(st.node_y + ((size_t)tn * (P.arity - 1) + (s - 1)) * np * np, f.X, np, ld);
      __syncthreads();
      for (int i = tid; i < np * np; i += kThreads) {
        const int a = i / np, b = i % np;
        E v = Ar::zero();
        for (int p = a; p < n; ++p) Ar::fma_acc(v, f.X[a * ld + p], f.M[p * ld + b]);
        out[i] = Ar::neg(Ar::fin(v));
      }
      __syncthreads();
    }
  }
}

template <class Ar>
__global__ void __launch_bounds__(kThreads, 1) formq_tree_kernel(const Plan P, const Store st, int level) {
  extern __shared__ char smem_raw[];
  formq_tree_node<Ar>(P, st, level, blockIdx.x, smem_raw);
}

// Q rows of chain g, last leaf first.  chain step (V = [I; Y]): Q_rows = -Y M with M = T C,
// then C -= M.  first leaf (V unit lower trapezoidal): Q_rows = [C; 0] - V (T (V_top^T C)).
// With double buffering (kDbl, where two tiles fit), the next leaf's tile (TMA) and T (register
// loads) are in flight while the current leaf computes.  It costs registers and shared memory,
// so it pays where one block per SM is all that fits anyway (np = 64); narrower plans keep the
// single-buffer kernel and two blocks per SM.
template <class Ar, bool kDbl>
__device__ __forceinline__ void formq_chain(const CUtensorMap* mapV_p, const Plan& P, const Store& st,
                                            typename Ar::Out* __restrict__ Q, int64_t ldq, int box_rows, int g,
                                            char* smem_raw) {
  using E = typename Ar::E;
  FormQSmem<E> f = carve_formq<E>(smem_raw, P, kDbl);
  const int tid = threadIdx.x;
  const int np = P.np, n = P.n, h = P.h, ld = f.ld;
  if (tid == 0) {
    mbar_init(f.bar, 1);
    mbar_init(f.bar + 1, 1);
    fence_mbar_init();
  }
  // C = this chain's block of Q_tree [D; 0], left by the tree levels (or D without a tree)
  {
    const double* Cg = st.node_r + (size_t)g * np * np;
    for (int i = tid; i < np * np; i += kThreads) {
      const int a = i / np, b = i % np;
      if (P.depth == 0) {
        f.C[a * ld + b] = (a == b && a < n) ? Ar::from_f64(__ldcg(st.signs + a)) : Ar::zero();
      } else {
        const double v = __ldcg(Cg + i);
        f.C[a * ld + b] = *reinterpret_cast<const E*>(&v);
      }
    }
  }
  __syncthreads();
  uint32_t phase[2] = {0u, 0u};

  // T of the next leaf in registers: np * np / kThreads <= 16 slots per thread
  constexpr int kTReg = 16;
  double treg[kTReg];
  auto t_fetch = [&](int64_t leaf) {
    const double* Tg = st.t_leaf + leaf * np * np;
#pragma unroll
    for (int u = 0; u < kTReg; ++u) {
      const int i = tid + u * kThreads;
      treg[u] = (i < np * np) ? __ldcg(Tg + i) : 0.0;
    }
  };
  auto t_store = [&]() {
#pragma unroll
    for (int u = 0; u < kTReg; ++u) {
      const int i = tid + u * kThreads;
      if (i < np * np) f.T[(i / np) * ld + (i % np)] = *reinterpret_cast<const E*>(&treg[u]);
    }
  };

  // ---- unwind the chain from its last leaf to its first
  const int64_t l0 = chain_first_leaf(P, g), l1 = chain_end_leaf(P, g);
  const int G = kThreads / np;
  const int cown = tid & (np - 1), gown = tid / np;
  int buf = 0;
  if (f.dbl) {
    tile_load_start(f.S, mapV_p, f.bar, np, (l1 - 1) * h, h, 0, box_rows);
    t_fetch(l1 - 1);
  }
  for (int64_t leaf = l1 - 1; leaf >= l0; --leaf) {
    const bool plain = (leaf == l0);
    const int64_t row0 = leaf * h;
    const Tile& S = buf ? f.S2 : f.S;
    E* X = f.X;
    if (f.dbl) {
      if (!tile_load_finish(f.bar + buf, phase[buf], st.status, f.flag)) return;
      t_store();
      if (!plain) {  // the next leaf's loads go into the idle buffer (its barrier orders t_store too)
        tile_load_start(buf ? f.S : f.S2, mapV_p, f.bar + (buf ^ 1), np, (leaf - 1) * h, h, 0, box_rows);
        t_fetch(leaf - 1);
      } else {
        __syncthreads();
        X = reinterpret_cast<E*>(buf ? f.S.base : f.S2.base);  // the idle buffer
      }
    } else {
      tile_load_start(S, mapV_p, f.bar, np, row0, h, 0, box_rows);  // the tile by TMA while T loads
      load_square(st.t_leaf + leaf * np * np, f.T, np, ld);
      if (!tile_load_finish(f.bar, phase[0], st.status, f.flag)) return;
    }
    const int64_t rows_valid = (P.m - row0 < h) ? (P.m - row0) : h;
    if (!plain) {
      tri_mul<Ar>(f.T, ld, f.C, ld, f.M, ld, n, np, np, false);
      __syncthreads();
      if (cown < n) {
        for (int r = gown; r < rows_valid; r += G) {
          E v = Ar::zero();
          for (int a = 0; a < n; ++a) Ar::fma_acc(v, tat<E>(S, r, a), f.M[a * ld + cown]);
          Q[gidx(P, row0 + r, cown, ldq)] = -Ar::to_out(Ar::fin(v));
        }
      }
      for (int i = tid; i < np * np; i += kThreads) {
        const int o = (i / np) * ld + i % np;
        f.C[o] = Ar::sub(f.C[o], f.M[o]);
      }
      __syncthreads();
    } else {
      // X = V_top^T C, V_top unit lower triangular (rows 0..n-1 of the leaf)
      for (int o = tid; o < np * np; o += kThreads) {
        const int a = o / np, b = o % np;
        E v = Ar::zero();
        if (a < n) {
          v = f.C[a * ld + b];
          for (int r = a + 1; r < n; ++r) Ar::fma_acc(v, tat<E>(S, r, a), f.C[r * ld + b]);
          v = Ar::fin(v);
        }
        X[a * ld + b] = v;
      }
      __syncthreads();
      tri_mul<Ar>(f.T, ld, X, ld, f.M, ld, n, np, np, false);
      __syncthreads();
      if (cown < n) {
        for (int r = gown; r < rows_valid; r += G) {
          // v = [C; 0]_r - sum_a V[r][a] M[a] with V's unit diagonal
          E acc = Ar::zero();
          const int amax = (r < n) ? r : n;
          for (int a = 0; a < amax; ++a) Ar::fma_acc(acc, tat<E>(S, r, a), f.M[a * ld + cown]);
          if (r < n) Ar::fma_acc(acc, Ar::from_int(1), f.M[r * ld + cown]);
          E v = Ar::neg(Ar::fin(acc));
          if (r < n) v = Ar::add(v, f.C[r * ld + cown]);
          Q[gidx(P, row0 + r, cown, ldq)] = Ar::to_out(v);
        }
      }
      __syncthreads();
    }
    if (f.dbl) buf ^= 1;
  }
}

template <class Ar, bool kDbl>
__global__ void __launch_bounds__(kThreads, 1)
    formq_kernel(const __grid_constant__ CUtensorMap mapV, const Plan P, const Store st,
                 typename Ar::Out* __restrict__ Q, int64_t ldq, int box_rows) {
  extern __shared__ char smem_raw[];
  formq_chain<Ar, kDbl>(&mapV, P, st, Q, ldq, box_rows, blockIdx.x, smem_raw);
}

// Batched thin Q: one tree step (item, node, level) per block, or one chain per block.
template <class Ar>
__global__ void __launch_bounds__(kThreads, 1)
    formq_tree_batched_kernel(const BatchItem* __restrict__ items, const BatchWork* __restrict__ work) {
  extern __shared__ char smem_raw[];
  const BatchWork w = work[blockIdx.x];
  const BatchItem& it = items[w.item];
  formq_tree_node<Ar>(it.plan, it.store, w.level, w.chain, smem_raw);
}
template <class Ar>
__global__ void __launch_bounds__(kThreads, 1)
    formq_chain_batched_kernel(const BatchItem* __restrict__ items, const BatchWork* __restrict__ work) {
  extern __shared__ char smem_raw[];
  const BatchWork w = work[blockIdx.x];
  const BatchItem& it = items[w.item];
  formq_chain<Ar, true>(&it.mapV, it.plan, it.store, static_cast<typename Ar::Out*>(it.Q), it.ldq, it.box_rows,
                        w.chain, smem_raw);
}

template <class Ar>
static cudaError_t prepare_form_q_batched_t(size_t smem) {
  cudaError_t e =
      cudaFuncSetAttribute(formq_tree_batched_kernel<Ar>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(formq_chain_batched_kernel<Ar>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t prepare_form_q_batched(int precision, size_t smem) {
  if (prec_df(precision)) return prepare_form_q_batched_t<ArithDF>(smem);
  if (precision == kPrecF32) return prepare_form_q_batched_t<ArithF32>(smem);
  return prepare_form_q_batched_t<ArithF64>(smem);
}

template <class Ar>
static cudaError_t launch_form_q_batched_t(const BatchItem* items, const BatchWork* chain_work, int chain_blocks,
                                           const BatchWork* const* level_work, const int* level_blocks, int depth,
                                           size_t smem, cudaStream_t stream) {
  cudaError_t e;
  for (int d = 0; d < depth; ++d) {
    if (level_blocks[d] == 0) continue;
    formq_tree_batched_kernel<Ar><<<level_blocks[d], kThreads, smem, stream>>>(items, level_work[d]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (chain_blocks == 0) return cudaSuccess;  // every chain runs on the tensor-core kernel
  formq_chain_batched_kernel<Ar><<<chain_blocks, kThreads, smem, stream>>>(items, chain_work);
  return cudaGetLastError();
}

cudaError_t launch_form_q_batched(const BatchItem* items, const BatchWork* chain_work, int chain_blocks,
                                  const BatchWork* const* level_work, const int* level_blocks, int depth,
                                  int precision, size_t smem, cudaStream_t stream) {
  if (prec_df(precision))
    return launch_form_q_batched_t<ArithDF>(items, chain_work, chain_blocks, level_work, level_blocks, depth, smem,
                                            stream);
  if (precision == kPrecF32)
    return launch_form_q_batched_t<ArithF32>(items, chain_work, chain_blocks, level_work, level_blocks, depth, smem,
                                             stream);
  return launch_form_q_batched_t<ArithF64>(items, chain_work, chain_blocks, level_work, level_blocks, depth, smem,
                                           stream);
}

// ------------------------------------------------------------------------------------------
// Thin Q with the compact-WY products on the tensor cores (precision modes 2 and 3): the whole
// chain in one block, as the batched thin Q runs it, and, for a single factorization, the chains'
// first leaves after formq_ozaki_phases.cu has taken the rest.
//
// Per chain leaf: M = T C and Q_rows = -Y M, each an Ozaki-split FP64 product (ozaki.cuh, digit
// form) on tcgen05 with exact FP32 accumulators in TMEM; C -= M in FP64.
// The leaf's T arrives by a bulk copy and its reflector tile by TMA, both issued when the leaf
// starts so that they overlap the T C product.  The first leaf of a chain (V unit lower
// trapezoidal) takes three passes: X = V_top^T C, M = T X, Q_rows = [C; 0] - V M.  Needs
// np = 64 (33 <= n <= 64) and h <= 128.
// 512 threads, one block per SM (all 512 TMEM columns).


size_t formq_ozaki_smem_bytes(const Plan& P) {
  const size_t ybytes = ((size_t)P.h * 64 * 8 + 1023) & ~size_t(1023);
  return 1024 + ybytes + 8 * oz::kBSliceBytes + 2 * oz::kASliceBytes + 2 * 64 * kOzLd * 8 + 128 * 4 + 64 * 4 + 4 * 8 +
         16;
}


// Chain g of one factorization (the body of formq_ozaki_kernel and of its batched form).
// first_only: only the chain's first leaf, with the block C entering it read from node_r[g] as
// plain FP64 (written there by formq_ozaki_recur_kernel after the chain's other leaves).
template <bool kPairs>
__device__ __forceinline__ void formq_ozaki_chain(const CUtensorMap* mapV_p, const Plan& P, const Store& st,
                                                  double* __restrict__ Q, int64_t ldq, int box_rows, int g,
                                                  char* smem_raw, bool first_only = false) {
  OzSmem z = carve_ozaki(smem_raw, P.h);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int np = 64, n = P.n, h = P.h;
  if (tid == 0) {
    for (int b = 0; b < 4; ++b) mbar_init(z.bars + b, 1);
    fence_mbar_init();
    *z.flag = 0;
  }
  if (warp == 0) oz::tmem_alloc(z.slot, oz::kTmemCols);
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  const uint32_t tmem = *z.slot;
  uint32_t ph[2] = {0u, 0u};
  uint32_t y_phase = 0, t_phase = 0;
  // C = this chain's block of Q_tree [D; 0] (first_only: the block entering the first leaf)
  for (int i = tid; i < np * np; i += kOzT) {
    const int a = i / np, b = i % np;
    const double* Cg = st.node_r + (size_t)g * np * np;
    z.C[a * kOzLd + b] = first_only ? __ldcg(Cg + i)
                         : (P.depth == 0) ? ((a == b && a < n) ? __ldcg(st.signs + a) : 0.0)
                                          : slot_val<kPairs>(__ldcg(Cg + i));
  }
  __syncthreads();
  const int64_t l0 = chain_first_leaf(P, g), l1 = first_only ? l0 + 1 : chain_end_leaf(P, g);
  bool alive = true;
  for (int64_t leaf = l1 - 1; leaf >= l0 && alive; --leaf) {
    const int64_t row0 = leaf * h;
    const int rows_valid = (int)((P.m - row0 < h) ? (P.m - row0) : h);
    const double* Tg = st.t_leaf + leaf * np * np;
    if (leaf != l0) {
      // ---- both loads of the leaf start now: T into the M buffer, the reflector tile into Y
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        mbar_arrive_expect_tx(z.bars + 3, np * np * 8);
        bulk_load(z.M, Tg, np * np * 8, z.bars + 3);
        mbar_arrive_expect_tx(z.bars + 0, (uint32_t)h * np * 8);
        for (int pnl = 0; pnl < np / 16; ++pnl)
          for (int r = 0; r < h; r += box_rows)
            tma_load_2d(z.Y.base + (size_t)pnl * h * 128 + (size_t)r * 128, mapV_p, z.bars + 0, pnl * 16,
                        (int)(row0 + r));
      }
      // ---- C (B operand): output column j, k-th entry C[k][j]
      ozaki_b_slices(z, [&](int j, int k) { return z.C[k * kOzLd + j]; });
      ozaki_zero_a_rows(z, np, oz::kM);
      // ---- T (A operand): row exponents, then fixed point in place
      {
        const bool ok = oz_wait_all(z, z.bars + 3, t_phase, st.status);
        t_phase ^= 1u;
        if (!ok) {
          alive = false;
          break;
        }
      }
      long long* Tfix = reinterpret_cast<long long*>(z.M);
      for (int r = tid; r < 128; r += kOzT) z.expA[r] = 0;
      __syncthreads();
      for (int idx = tid; idx < np * np; idx += kOzT) warp_max_into(&z.expA[idx >> 6], slot_bexp<kPairs>(z.M[idx]));
      __syncthreads();
      for (int idx = tid; idx < np * np; idx += kOzT)
        Tfix[idx] = (long long)slot_biased54<kPairs>(z.M[idx], z.expA[idx >> 6]);
      __syncthreads();
      if (!ozaki_mma_pass(z, tmem, np, [&](int r, int k) { return (uint64_t)Tfix[r * 64 + k]; }, ph, st.status)) {
        alive = false;
        break;
      }
      // ---- M = T C (M takes the buffer of Tfix; every MMA reading it has completed)
      ozaki_epilogue(z, tmem, np, [&](int i, int j, double v) { z.M[i * kOzLd + j] = v; });
      for (int i = tid; i < np * np; i += kOzT) {
        const int o = (i / np) * kOzLd + i % np;
        z.C[o] -= z.M[o];
      }
      // ---- M (B operand): output column j, k-th entry M[k][j]
      ozaki_b_slices(z, [&](int j, int k) { return z.M[k * kOzLd + j]; });
      if (h < oz::kM) ozaki_zero_a_rows(z, h, oz::kM);
      // ---- Y (A operand): row exponents, fixed point in place
      {
        const bool ok = oz_wait_all(z, z.bars + 0, y_phase, st.status);
        y_phase ^= 1u;
        if (!ok) {
          alive = false;
          break;
        }
      }
      for (int r = tid; r < 128; r += kOzT) z.expA[r] = 0;
      __syncthreads();
      for (int idx = tid; idx < h * np; idx += kOzT)
        warp_max_into(&z.expA[idx >> 6], slot_bexp<kPairs>(*z.Y.ptr(idx >> 6, idx & 63)));
      __syncthreads();
      for (int idx = tid; idx < h * np; idx += kOzT) {
        double* p = z.Y.ptr(idx >> 6, idx & 63);
        *reinterpret_cast<uint64_t*>(p) = slot_biased54<kPairs>(*p, z.expA[idx >> 6]);
      }
      __syncthreads();
      if (!ozaki_mma_pass(z, tmem, h, [&](int r, int k) { return *reinterpret_cast<const uint64_t*>(z.Y.ptr(r, k)); },
                          ph, st.status)) {
        alive = false;
        break;
      }
      ozaki_epilogue(z, tmem, rows_valid, [&](int i, int j, double v) {
        if (j < n) Q[gidx(P, row0 + i, j, ldq)] = -v;
      });
    } else {
      // ---- first leaf (V unit lower trapezoidal; the tile's rows 0..n-1 hold R above the
      //      diagonal): Q_rows = [C; 0] - V (T (V_top^T C)) as three Ozaki passes
      if (!tile_load(z.Y, mapV_p, z.bars, y_phase, np, row0, h, 0, box_rows, st.status, z.flag)) {
        alive = false;
        break;
      }
      if constexpr (kPairs) {
        for (int idx = tid; idx < h * np; idx += kOzT) {
          double* p = z.Y.ptr(idx >> 6, idx & 63);
          *p = slot_val<true>(*p);
        }
        __syncthreads();
      }
      // V's entry (r, a): 1 on the diagonal, the stored reflector below it, 0 above and past n
      auto vval = [&](int r, int a) -> double {
        return (a < n) ? (r > a ? *z.Y.ptr(r, a) : (r == a ? 1.0 : 0.0)) : 0.0;
      };
      long long* Afix = reinterpret_cast<long long*>(z.M);
      // pass 1: X = V_top^T C; A = V_top^T (row a, k = r < n), B = C
      ozaki_b_slices(z, [&](int j, int k) { return z.C[k * kOzLd + j]; });
      ozaki_zero_a_rows(z, np, oz::kM);
      for (int r = tid; r < 128; r += kOzT) z.expA[r] = 0;
      __syncthreads();
      for (int idx = tid; idx < np * np; idx += kOzT) {
        const int a = idx >> 6, r = idx & 63;
        warp_max_into(&z.expA[a], oz::bexp(r < n ? vval(r, a) : 0.0));
      }
      __syncthreads();
      for (int idx = tid; idx < np * np; idx += kOzT) {
        const int a = idx >> 6, r = idx & 63;
        Afix[idx] = (long long)oz::to_biased54(r < n ? vval(r, a) : 0.0, z.expA[a]);
      }
      __syncthreads();
      if (!ozaki_mma_pass(z, tmem, np, [&](int r, int k) { return (uint64_t)Afix[r * 64 + k]; }, ph, st.status)) {
        alive = false;
        break;
      }
      ozaki_epilogue(z, tmem, np, [&](int i, int j, double v) { z.M[i * kOzLd + j] = v; });  // X
      // pass 2: M = T X; B = X, A = T
      ozaki_b_slices(z, [&](int j, int k) { return z.M[k * kOzLd + j]; });
      for (int i = tid; i < np * np; i += kOzT) z.M[i] = slot_val<kPairs>(__ldcg(Tg + i));
      for (int r = tid; r < 128; r += kOzT) z.expA[r] = 0;
      __syncthreads();
      for (int idx = tid; idx < np * np; idx += kOzT) warp_max_into(&z.expA[idx >> 6], oz::bexp(z.M[idx]));
      __syncthreads();
      for (int idx = tid; idx < np * np; idx += kOzT) Afix[idx] = (long long)oz::to_biased54(z.M[idx], z.expA[idx >> 6]);
      __syncthreads();
      if (!ozaki_mma_pass(z, tmem, np, [&](int r, int k) { return (uint64_t)Afix[r * 64 + k]; }, ph, st.status)) {
        alive = false;
        break;
      }
      ozaki_epilogue(z, tmem, np, [&](int i, int j, double v) { z.M[i * kOzLd + j] = v; });  // M
      // pass 3: Q_rows = [C; 0] - V M; B = M, A = V (rows of the leaf), in place in the tile
      ozaki_b_slices(z, [&](int j, int k) { return z.M[k * kOzLd + j]; });
      if (h < oz::kM) ozaki_zero_a_rows(z, h, oz::kM);
      for (int r = tid; r < 128; r += kOzT) z.expA[r] = 0;
      __syncthreads();
      for (int idx = tid; idx < h * np; idx += kOzT) warp_max_into(&z.expA[idx >> 6], oz::bexp(vval(idx >> 6, idx & 63)));
      __syncthreads();
      for (int idx = tid; idx < h * np; idx += kOzT) {
        const int r = idx >> 6, a = idx & 63;
        const double v = vval(r, a);  // reads only element (r, a), which it then replaces
        *reinterpret_cast<uint64_t*>(z.Y.ptr(r, a)) = oz::to_biased54(v, z.expA[r]);
      }
      __syncthreads();
      if (!ozaki_mma_pass(z, tmem, h, [&](int r, int k) { return *reinterpret_cast<const uint64_t*>(z.Y.ptr(r, k)); },
                          ph, st.status)) {
        alive = false;
        break;
      }
      ozaki_epilogue(z, tmem, rows_valid, [&](int i, int j, double v) {
        if (j < n) Q[gidx(P, row0 + i, j, ldq)] = (i < n ? z.C[i * kOzLd + j] : 0.0) - v;
      });
    }
  }
  // every pass waits for its commits; after a timeout, give the copies and MMAs in flight one
  // more bounded wait before TMEM is freed
  if (!alive && tid == 0) {
    oz::wait_bar(z.bars + 1, ph[0]);
    oz::wait_bar(z.bars + 2, ph[1]);
    oz::wait_bar(z.bars + 0, y_phase);
    oz::wait_bar(z.bars + 3, t_phase);
  }
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  if (warp == 0) oz::tmem_dealloc(tmem, oz::kTmemCols);
}

// split: the chain's other leaves were taken by formq_ozaki_recur_kernel and the leaf products
// kernel, so only its first leaf is left here (except a chain that holds a short last leaf,
// which is taken whole, as without split).
template <bool kPairs>
__global__ void __launch_bounds__(kOzT, 1)
    formq_ozaki_kernel(const __grid_constant__ CUtensorMap mapV, const Plan P, const Store st, double* __restrict__ Q,
                       int64_t ldq, int box_rows, bool split) {
  extern __shared__ char smem_raw[];
  const int g = blockIdx.x;
  formq_ozaki_chain<kPairs>(&mapV, P, st, Q, ldq, box_rows, g, smem_raw, split && !formq_chain_short(P, g));
}

// Batched: block b takes chain work[b].chain of item work[b].item (items whose thin Q runs on the
// tensor cores: padded width 64, leaf height <= 128).
template <bool kPairs>
__global__ void __launch_bounds__(kOzT, 1)
    formq_ozaki_batched_kernel(const BatchItem* __restrict__ items, const BatchWork* __restrict__ work) {
  extern __shared__ char smem_raw[];
  const BatchWork w = work[blockIdx.x];
  const BatchItem& it = items[w.item];
  formq_ozaki_chain<kPairs>(&it.mapV, it.plan, it.store, static_cast<double*>(it.Q), it.ldq, it.box_rows, w.chain,
                            smem_raw);
}

cudaError_t prepare_formq_ozaki_batched(bool pairs, size_t smem) {
  return pairs ? cudaFuncSetAttribute(formq_ozaki_batched_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)
               : cudaFuncSetAttribute(formq_ozaki_batched_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem);
}

cudaError_t launch_formq_ozaki_batched(const BatchItem* items, const BatchWork* work, int blocks, bool pairs,
                                       size_t smem, cudaStream_t stream) {
  if (pairs)
    formq_ozaki_batched_kernel<true><<<blocks, kOzT, smem, stream>>>(items, work);
  else
    formq_ozaki_batched_kernel<false><<<blocks, kOzT, smem, stream>>>(items, work);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Q^T B and Q B on column blocks of kb columns (kb a power of two <= 32)

template <class E>
struct ApplySmem {
  Tile S;   // leaf reflectors, h rows
  E* B;     // max(h, arity*np) x kb
  E* C;     // np x kb: the chain's top block
  E* W;     // np x kb
  E* W2;    // np x kb
  E* T;     // np x (np+1)
  E* Y;     // np x (np+1): one tree-node block (shares the tile's region)
  E* red;   // kThreads
  uint64_t* bar;
  int* flag;
  int ldt, brows;
};

// The leaf tile and a tree node's Y block are never live together (the tree steps follow the
// chain's leaves), so they share one region: the smaller footprint lets two blocks share an SM
// when the column blocks are narrow.
__host__ __device__ inline size_t apply_union_bytes(const Plan& P) {
  const size_t s = (size_t)P.h * P.np * 8, y = (size_t)P.np * (P.np + 1) * 8;
  return ((s > y ? s : y) + 15) & ~size_t(15);
}

template <class E>
__device__ inline ApplySmem<E> carve_apply(char* raw, const Plan& P, int kb) {
  ApplySmem<E> f;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  f.S = Tile{base, P.h};
  f.Y = reinterpret_cast<E*>(base);
  f.brows = max(P.h, P.arity * P.np);
  f.ldt = P.np + 1;
  f.B = reinterpret_cast<E*>(base + apply_union_bytes(P));
  f.C = f.B + (size_t)f.brows * kb;
  f.W = f.C + P.np * kb;
  f.W2 = f.W + P.np * kb;
  f.T = f.W2 + P.np * kb;
  f.red = f.T + P.np * f.ldt;
  f.bar = reinterpret_cast<uint64_t*>(f.red + kThreads);
  f.flag = reinterpret_cast<int*>(f.bar + 1);
  return f;
}

size_t apply_smem_bytes(const Plan& P, int kb) {
  const size_t brows = (size_t)(P.h > P.arity * P.np ? P.h : P.arity * P.np);
  return 1024 + apply_union_bytes(P) + brows * kb * 8 + 3 * (size_t)P.np * kb * 8 + (size_t)P.np * (P.np + 1) * 8 +
         kThreads * 8 + 8 + 16;
}

// W (np x kb), with the row sum split over thread groups when there are few outputs:
//   plain : W[a][b] = B[a][b] + sum_{r=a+1}^{h-1} V[r][a] B[r][b]       (V unit lower trapezoidal)
//   chain : W[a][b] = C[a][b] + sum_{r=0}^{h-1}   Y[r][a] B[r][b]
template <class Ar>
__device__ inline void wy_inner(const Tile& S, bool plain, int h, int n, int np, const typename Ar::E* B,
                                const typename Ar::E* C, typename Ar::E* W, int kb, typename Ar::E* red) {
  using E = typename Ar::E;
  const int OUT = np * kb;
  const int G = OUT >= kThreads ? 1 : kThreads / OUT;
  const int tid = threadIdx.x;
  for (int o0 = 0; o0 < OUT; o0 += kThreads / G) {
    const int o = o0 + tid % (kThreads / G);
    const int gg = tid / (kThreads / G);
    E acc = Ar::zero();
    if (o < OUT) {
      const int a = o / kb, b = o % kb;
      if (a < n) {
        const int r0 = plain ? a + 1 : 0;
        for (int r = r0 + gg; r < h; r += G) Ar::fma_acc(acc, tat<E>(S, r, a), B[r * kb + b]);
      }
    }
    if (G == 1) {
      if (o < OUT) {
        const int a = o / kb, b = o % kb;
        W[o] = (a < n) ? Ar::add(acc, plain ? B[a * kb + b] : C[a * kb + b]) : Ar::zero();
      }
    } else {
      red[tid] = acc;
      __syncthreads();
      if (gg == 0 && o < OUT) {
        E s = Ar::zero();
        for (int q = 0; q < G; ++q) s = Ar::add(s, red[q * (kThreads / G) + tid]);
        const int a = o / kb, b = o % kb;
        W[o] = (a < n) ? Ar::add(s, plain ? B[a * kb + b] : C[a * kb + b]) : Ar::zero();
      }
      __syncthreads();
    }
  }
}

// B -= V W2 (rows 0..h-1); plain: V unit lower trapezoidal; chain: V = [I; Y] so C -= W2 too.
template <class Ar>
__device__ inline void wy_update(const Tile& S, bool plain, int h, int n, int np, typename Ar::E* B,
                                 typename Ar::E* C, const typename Ar::E* W2, int kb) {
  using E = typename Ar::E;
  const int L = split_lanes(h * kb);
  if (L == 1) {
    for (int o = threadIdx.x; o < h * kb; o += kThreads) {
      const int r = o / kb, b = o % kb;
      E acc = Ar::zero();
      const int amax = plain ? (r < n ? r : n) : n;
      for (int a = 0; a < amax; ++a) Ar::fma_acc(acc, tat<E>(S, r, a), W2[a * kb + b]);
      if (plain && r < n) Ar::fma_acc(acc, Ar::from_int(1), W2[r * kb + b]);
      B[o] = Ar::sub(B[o], Ar::fin(acc));
    }
  } else {
    // few outputs (narrow B): L adjacent lanes per row, each a strided part of the sum (one pass)
    const int lL = __ffs(L) - 1;
    const int o0 = threadIdx.x;
    if (o0 < (h * kb) << lL) {
      const int o = o0 >> lL, part = o0 & (L - 1);
      const int r = o / kb, b = o % kb;
      E acc = Ar::zero();
      const int amax = plain ? (r < n ? r : n) : n;
      for (int a = part; a < amax; a += L) Ar::fma_acc(acc, tat<E>(S, r, a), W2[a * kb + b]);
      if (plain && r < n && part == 0) Ar::fma_acc(acc, Ar::from_int(1), W2[r * kb + b]);
      acc = Ar::fin(acc);
      for (int off = 1; off < L; off <<= 1) acc = Ar::add(acc, Ar::shfl_xor(acc, off));
      if (part == 0) B[o] = Ar::sub(B[o], acc);
    }
  }
  if (!plain)
    for (int o = threadIdx.x; o < np * kb; o += kThreads) C[o] = Ar::sub(C[o], W2[o]);
}

template <class Ar>
__device__ inline void load_b(const Plan& P, const typename Ar::Out* __restrict__ Bg, int64_t ldb, int64_t m, int64_t k,
                              int64_t row0, int rows, int64_t col0, int kb, typename Ar::E* Bs) {
  for (int o = threadIdx.x; o < rows * kb; o += kThreads) {
    const int r = o / kb, b = o % kb;
    const int64_t gr = row0 + r, gc = col0 + b;
    Bs[o] = (gr < m && gc < k) ? Ar::from_out(__ldcg(Bg + gidx(P, gr, gc, ldb))) : Ar::zero();
  }
}
template <class Ar>
__device__ inline void store_b(const Plan& P, typename Ar::Out* __restrict__ Bg, int64_t ldb, int64_t m, int64_t k, int64_t row0,
                               int r_begin, int rows, int64_t col0, int kb, const typename Ar::E* Bs) {
  for (int o = threadIdx.x; o < (rows - r_begin) * kb; o += kThreads) {
    const int r = r_begin + o / kb, b = o % kb;
    const int64_t gr = row0 + r, gc = col0 + b;
    if (gr < m && gc < k) Bg[gidx(P, gr, gc, ldb)] = Ar::to_out(Bs[r * kb + b]);
  }
}

// Tree-node step on the stacked top blocks of the q children (child s's block at B rows
// s*np..s*np+n-1): D = C0 + sum_s Y_s^T C_s; W2 = T^T D (trans) or T D; C0 -= W2; C_s -= Y_s W2.
template <class Ar>
__device__ inline void node_apply(ApplySmem<typename Ar::E>& f, const Plan& P, const Store& st, int tn, int q, int kb,
                                  bool trans) {
  using E = typename Ar::E;
  const int np = P.np, n = P.n, ld = f.ldt, tid = threadIdx.x;
  load_square(st.node_t + (size_t)tn * np * np, f.T, np, ld);
  for (int o = tid; o < np * kb; o += kThreads) f.W[o] = f.B[o];
  __syncthreads();
  for (int s = 1; s < q; ++s) {
    load_square(st.node_y + ((size_t)tn * (P.arity - 1) + (s - 1)) * np * np, f.Y, np, ld);
    __syncthreads();
    const E* Cs = f.B + (size_t)s * np * kb;
    for (int o = tid; o < np * kb; o += kThreads) {
      const int a = o / kb, b = o % kb;
      E v = f.W[o];
      for (int r = 0; r <= a && r < n; ++r) Ar::fma_acc(v, f.Y[r * ld + a], Cs[r * kb + b]);
      f.W[o] = Ar::fin(v);
    }
    __syncthreads();
  }
  tri_mul<Ar>(f.T, ld, f.W, kb, f.W2, kb, n, np, kb, trans);
  __syncthreads();
  for (int o = tid; o < np * kb; o += kThreads) f.B[o] = Ar::sub(f.B[o], f.W2[o]);
  for (int s = 1; s < q; ++s) {
    load_square(st.node_y + ((size_t)tn * (P.arity - 1) + (s - 1)) * np * np, f.Y, np, ld);
    __syncthreads();
    E* Cs = f.B + (size_t)s * np * kb;
    for (int o = tid; o < np * kb; o += kThreads) {
      const int a = o / kb, b = o % kb;
      E acc = Ar::zero();
      for (int p = a; p < n; ++p) Ar::fma_acc(acc, f.Y[a * ld + p], f.W2[p * kb + b]);
      Cs[o] = Ar::sub(Cs[o], Ar::fin(acc));
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
template <class Ar>
__global__ void __launch_bounds__(kThreads, 2)
    apply_qt_kernel(const __grid_constant__ CUtensorMap mapV, const Plan P, const Store st, int64_t k,
                    typename Ar::Out* __restrict__ Bg, int64_t ldb, int kb, int box_rows) {
  using E = typename Ar::E;
  extern __shared__ char smem_raw[];
  ApplySmem<E> f = carve_apply<E>(smem_raw, P, kb);
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
    tile_load_start(f.S, &mapV, f.bar, np, row0, h, 0, box_rows);  // the reflector tile by TMA,
    load_square(st.t_leaf + leaf * np * np, f.T, np, f.ldt);      // while T and B's rows load
    load_b<Ar>(P, Bg, ldb, P.m, k, row0, h, col0, kb, f.B);
    if (!tile_load_finish(f.bar, phase, st.status, f.flag)) return;
    wy_inner<Ar>(f.S, plain, h, n, np, f.B, f.C, f.W, kb, f.red);
    __syncthreads();
    tri_mul<Ar>(f.T, f.ldt, f.W, kb, f.W2, kb, n, np, kb, true);
    __syncthreads();
    wy_update<Ar>(f.S, plain, h, n, np, f.B, f.C, f.W2, kb);
    __syncthreads();
    if (plain) {  // rows 0..n-1 become the chain's top block
      for (int o = tid; o < np * kb; o += kThreads) f.C[o] = (o / kb < n) ? f.B[o] : Ar::zero();
      store_b<Ar>(P, Bg, ldb, P.m, k, row0, n, h, col0, kb, f.B);
    } else {
      store_b<Ar>(P, Bg, ldb, P.m, k, row0, 0, h, col0, kb, f.B);
    }
    __syncthreads();
  }
  // publish the chain's top block
  store_b<Ar>(P, Bg, ldb, P.m, k, chain_top_row(P, g), 0, n, col0, kb, f.C);
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
        f.B[(size_t)s * np * kb + o] = (a < n && gc < k) ? Ar::from_out(__ldcg(Bg + gidx(P, top + a, gc, ldb))) : Ar::zero();
      }
    }
    __syncthreads();
    node_apply<Ar>(f, P, st, tn, q, kb, true);
    __syncthreads();
    for (int s = 0; s < q; ++s)
      store_b<Ar>(P, Bg, ldb, P.m, k, node_top_row(P, level, first + s), 0, n, col0, kb, f.B + (size_t)s * np * kb);
    idx = parent;
  }
  // root: the thin part gets the signs (the top block is C without a tree, else child 0's)
  __syncthreads();
  const E* topblk = (P.depth == 0) ? f.C : f.B;
  for (int o = tid; o < n * kb; o += kThreads) {
    const int a = o / kb, b = o % kb;
    if (col0 + b < k) Bg[gidx(P, a, col0 + b, ldb)] = (typename Ar::Out)__ldcg(st.signs + a) * Ar::to_out(topblk[o]);
  }
}

// ---- Q B, tree part: one launch per level, top-down; the root level first applies D.
template <class Ar>
__global__ void __launch_bounds__(kThreads, 2)
    apply_q_tree_kernel(const Plan P, const Store st, int level, int64_t k, typename Ar::Out* __restrict__ Bg,
                        int64_t ldb, int kb) {
  using E = typename Ar::E;
  extern __shared__ char smem_raw[];
  ApplySmem<E> f = carve_apply<E>(smem_raw, P, kb);
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
      typename Ar::Out v = (a < n && gc < k) ? Bg[gidx(P, top + a, gc, ldb)] : typename Ar::Out(0);
      if (level == P.depth && s == 0 && a < n) v *= (typename Ar::Out)st.signs[a];
      f.B[(size_t)s * np * kb + o] = Ar::from_out(v);
    }
  }
  __syncthreads();
  node_apply<Ar>(f, P, st, tn, q, kb, false);
  __syncthreads();
  for (int s = 0; s < q; ++s)
    store_b<Ar>(P, Bg, ldb, P.m, k, node_top_row(P, level - 1, first + s), 0, n, col0, kb, f.B + (size_t)s * np * kb);
}

// ---- Q^T B, tree part as separate launches (after a chain kernel that published each chain's
//      top block): one launch per level, bottom-up; the root level then applies the signs.
template <class Ar>
__global__ void __launch_bounds__(kThreads, 2)
    apply_qt_tree_kernel(const Plan P, const Store st, int level, int64_t k, typename Ar::Out* __restrict__ Bg,
                         int64_t ldb, int kb) {
  using E = typename Ar::E;
  extern __shared__ char smem_raw[];
  ApplySmem<E> f = carve_apply<E>(smem_raw, P, kb);
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
      f.B[(size_t)s * np * kb + o] = (a < n && gc < k) ? Ar::from_out(__ldcg(Bg + gidx(P, top + a, gc, ldb))) : Ar::zero();
    }
  }
  __syncthreads();
  node_apply<Ar>(f, P, st, tn, q, kb, true);
  __syncthreads();
  for (int s = (level == P.depth) ? 1 : 0; s < q; ++s)
    store_b<Ar>(P, Bg, ldb, P.m, k, node_top_row(P, level - 1, first + s), 0, n, col0, kb, f.B + (size_t)s * np * kb);
  if (level == P.depth)  // the root: child 0's block is the thin part, with the signs
    for (int o = tid; o < n * kb; o += kThreads) {
      const int a = o / kb, b = o % kb;
      if (col0 + b < k) Bg[gidx(P, a, col0 + b, ldb)] = (typename Ar::Out)__ldcg(st.signs + a) * Ar::to_out(f.B[o]);
    }
}

// ---- Q B, chains: last leaf first, the first leaf last.
template <class Ar>
__global__ void __launch_bounds__(kThreads, 2)
    apply_q_chain_kernel(const __grid_constant__ CUtensorMap mapV, const Plan P, const Store st, int64_t k,
                         typename Ar::Out* __restrict__ Bg, int64_t ldb, int kb, int box_rows) {
  using E = typename Ar::E;
  extern __shared__ char smem_raw[];
  ApplySmem<E> f = carve_apply<E>(smem_raw, P, kb);
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
    typename Ar::Out v = (a < n && gc < k) ? Bg[gidx(P, top + a, gc, ldb)] : typename Ar::Out(0);
    if (P.depth == 0 && a < n) v *= (typename Ar::Out)st.signs[a];
    f.C[o] = Ar::from_out(v);
  }
  __syncthreads();
  uint32_t phase = 0;
  const int64_t l0 = chain_first_leaf(P, g), l1 = chain_end_leaf(P, g);
  for (int64_t leaf = l1 - 1; leaf >= l0; --leaf) {
    const bool plain = (leaf == l0);
    const int64_t row0 = leaf * h;
    tile_load_start(f.S, &mapV, f.bar, np, row0, h, 0, box_rows);
    load_square(st.t_leaf + leaf * np * np, f.T, np, f.ldt);
    load_b<Ar>(P, Bg, ldb, P.m, k, row0, h, col0, kb, f.B);
    if (!tile_load_finish(f.bar, phase, st.status, f.flag)) return;
    if (plain)
      for (int o = tid; o < n * kb; o += kThreads) f.B[o] = f.C[o];
    __syncthreads();
    wy_inner<Ar>(f.S, plain, h, n, np, f.B, f.C, f.W, kb, f.red);
    __syncthreads();
    tri_mul<Ar>(f.T, f.ldt, f.W, kb, f.W2, kb, n, np, kb, false);
    __syncthreads();
    wy_update<Ar>(f.S, plain, h, n, np, f.B, f.C, f.W2, kb);
    __syncthreads();
    store_b<Ar>(P, Bg, ldb, P.m, k, row0, 0, h, col0, kb, f.B);
    __syncthreads();
  }
}

static int pick_kb(int64_t k) {
  int kb = 1;
  while (kb < k && kb < 32) kb <<= 1;
  return kb;
}

template <class Ar>
static cudaError_t launch_form_q_t(const CUtensorMap& mapV, const Plan& P, const Store& st, void* Q_, int64_t ldq,
                                   int box_rows, cudaStream_t stream) {
  typename Ar::Out* Q = static_cast<typename Ar::Out*>(Q_);
  const size_t smem = formq_smem_bytes(P);
  const bool dbl = (P.np == 64);  // the double-buffered chain kernel where it pays
  const size_t smem_chain = formq_smem_bytes(P, dbl);
  auto chain_kernel = dbl ? formq_kernel<Ar, true> : formq_kernel<Ar, false>;
  cudaError_t e = cudaFuncSetAttribute(chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_chain);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(formq_tree_kernel<Ar>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  for (int level = P.depth; level >= 1; --level) {
    formq_tree_kernel<Ar><<<P.level_count[level], kThreads, smem, stream>>>(P, st, level);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  chain_kernel<<<P.chains, kThreads, smem_chain, stream>>>(mapV, P, st, Q, ldq, box_rows);
  return cudaGetLastError();
}

static cudaError_t launch_form_q_ozaki(const CUtensorMap& mapV, const Plan& P, const Store& st, void* Q_,
                                       int64_t ldq, int box_rows, cudaStream_t stream) {
  double* Q = static_cast<double*>(Q_);
  const bool pairs = prec_df(P.precision);  // the factorization ran in double-float arithmetic
  const size_t smem_tree = formq_smem_bytes(P);
  cudaError_t e = pairs ? cudaFuncSetAttribute(formq_tree_kernel<ArithDF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem_tree)
                        : cudaFuncSetAttribute(formq_tree_kernel<ArithF64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem_tree);
  if (e != cudaSuccess) return e;
  for (int level = P.depth; level >= 1; --level) {
    if (pairs)
      formq_tree_kernel<ArithDF><<<P.level_count[level], kThreads, smem_tree, stream>>>(P, st, level);
    else
      formq_tree_kernel<ArithF64><<<P.level_count[level], kThreads, smem_tree, stream>>>(P, st, level);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // the chains' recurrences (M = T C of every leaf but the first, into Q; the block entering the
  // first leaf into node_r), then the first leaves, then the other leaves' products -V M
  e = launch_formq_ozaki_recur(P, st, Q, ldq, stream);
  if (e != cudaSuccess) return e;
  const size_t smem = formq_ozaki_smem_bytes(P);
  if (pairs) {
    e = cudaFuncSetAttribute(formq_ozaki_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    formq_ozaki_kernel<true><<<P.chains, kOzT, smem, stream>>>(mapV, P, st, Q, ldq, box_rows, true);
  } else {
    e = cudaFuncSetAttribute(formq_ozaki_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    formq_ozaki_kernel<false><<<P.chains, kOzT, smem, stream>>>(mapV, P, st, Q, ldq, box_rows, true);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_formq_ozaki_leaves(P, st, Q, ldq, stream);
}

bool ozaki_form_q_applies(const Plan& P) {
  return (P.precision == kPrecOzaki || P.precision == kPrecDFOzaki) && P.np == 64 && P.h <= 128;
}

// FP32 storage: the tree levels on the FP32 pipe, the chains with bf16x3 tensor-core products.
static cudaError_t launch_form_q_bf16x3(const CUtensorMap& mapV, const Plan& P, const Store& st, void* Q, int64_t ldq,
                                        int box_rows, cudaStream_t stream) {
  const size_t smem_tree = formq_smem_bytes(P);
  cudaError_t e =
      cudaFuncSetAttribute(formq_tree_kernel<ArithF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_tree);
  if (e != cudaSuccess) return e;
  for (int level = P.depth; level >= 1; --level) {
    formq_tree_kernel<ArithF32><<<P.level_count[level], kThreads, smem_tree, stream>>>(P, st, level);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_formq_bf16x3_chains(mapV, P, st, static_cast<float*>(Q), ldq, box_rows, stream);
}

cudaError_t launch_form_q(const CUtensorMap& mapV, const Plan& P, const Store& st, void* Q, int64_t ldq,
                          int box_rows, cudaStream_t stream) {
  if (ozaki_form_q_applies(P)) return launch_form_q_ozaki(mapV, P, st, Q, ldq, box_rows, stream);
  if (prec_df(P.precision)) return launch_form_q_t<ArithDF>(mapV, P, st, Q, ldq, box_rows, stream);
  if (bf16x3_form_q_applies(P)) return launch_form_q_bf16x3(mapV, P, st, Q, ldq, box_rows, stream);
  if (P.precision == kPrecF32) return launch_form_q_t<ArithF32>(mapV, P, st, Q, ldq, box_rows, stream);
  return launch_form_q_t<ArithF64>(mapV, P, st, Q, ldq, box_rows, stream);
}

template <class Ar>
static cudaError_t launch_apply_qt_t(const CUtensorMap& mapV, const Plan& P, const Store& st, int64_t k, void* B_,
                                     int64_t ldb, int box_rows, cudaStream_t stream) {
  typename Ar::Out* B = static_cast<typename Ar::Out*>(B_);
  const int kb = pick_kb(k);
  const size_t smem = apply_smem_bytes(P, kb);
  cudaError_t e = cudaFuncSetAttribute(apply_qt_kernel<Ar>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  for (int64_t c0 = 0; c0 < k; c0 += (int64_t)kb * kMaxColBlocks) {
    const int64_t kc = (k - c0 < (int64_t)kb * kMaxColBlocks) ? (k - c0) : (int64_t)kb * kMaxColBlocks;
    const int ncb = (int)((kc + kb - 1) / kb);
    e = cudaMemsetAsync(st.counters, 0, sizeof(int) * (size_t)(P.tree_nodes > 0 ? P.tree_nodes : 1) * kMaxColBlocks,
                        stream);
    if (e != cudaSuccess) return e;
    apply_qt_kernel<Ar><<<dim3(P.chains, ncb), kThreads, smem, stream>>>(mapV, P, st, kc, B + gidx(P, 0, c0, ldb), ldb,
                                                                          kb, box_rows);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Tree levels of Q^T B bottom-up (after launch_apply_ozaki_chains).
template <class Ar>
static cudaError_t launch_apply_qt_tree_t(const Plan& P, const Store& st, int64_t k, void* B_, int64_t ldb,
                                          cudaStream_t stream) {
  typename Ar::Out* B = static_cast<typename Ar::Out*>(B_);
  const int kb = pick_kb(k);
  const size_t smem = apply_smem_bytes(P, kb);
  cudaError_t e =
      cudaFuncSetAttribute(apply_qt_tree_kernel<Ar>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  for (int64_t c0 = 0; c0 < k; c0 += (int64_t)kb * kMaxColBlocks) {
    const int64_t kc = (k - c0 < (int64_t)kb * kMaxColBlocks) ? (k - c0) : (int64_t)kb * kMaxColBlocks;
    const int ncb = (int)((kc + kb - 1) / kb);
    for (int level = 1; level <= P.depth; ++level) {
      apply_qt_tree_kernel<Ar><<<dim3(P.level_count[level], ncb), kThreads, smem, stream>>>(
          P, st, level, kc, B + gidx(P, 0, c0, ldb), ldb, kb);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// Tree levels of Q B top-down (before launch_apply_ozaki_chains).
template <class Ar>
static cudaError_t launch_apply_q_tree_t(const Plan& P, const Store& st, int64_t k, void* B_, int64_t ldb,
                                         cudaStream_t stream) {
  typename Ar::Out* B = static_cast<typename Ar::Out*>(B_);
  const int kb = pick_kb(k);
  const size_t smem = apply_smem_bytes(P, kb);
  cudaError_t e =
      cudaFuncSetAttribute(apply_q_tree_kernel<Ar>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  for (int64_t c0 = 0; c0 < k; c0 += (int64_t)kb * kMaxColBlocks) {
    const int64_t kc = (k - c0 < (int64_t)kb * kMaxColBlocks) ? (k - c0) : (int64_t)kb * kMaxColBlocks;
    const int ncb = (int)((kc + kb - 1) / kb);
    for (int level = P.depth; level >= 1; --level) {
      apply_q_tree_kernel<Ar><<<dim3(P.level_count[level], ncb), kThreads, smem, stream>>>(
          P, st, level, kc, B + gidx(P, 0, c0, ldb), ldb, kb);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_apply_qt(const CUtensorMap& mapV, const Plan& P, const Store& st, int64_t k, void* B,
                            int64_t ldb, int box_rows, cudaStream_t stream) {
  if (ozaki_apply_applies(P, k)) {  // chains on the tensor cores, then the tree levels
    cudaError_t e = launch_apply_ozaki_chains(mapV, P, st, k, static_cast<double*>(B), ldb, box_rows, true, stream);
    if (e != cudaSuccess) return e;
    return prec_df(P.precision) ? launch_apply_qt_tree_t<ArithDF>(P, st, k, B, ldb, stream)
                                : launch_apply_qt_tree_t<ArithF64>(P, st, k, B, ldb, stream);
  }
  if (bf16x3_apply_applies(P, k)) {
    cudaError_t e = launch_apply_bf16x3_chains(mapV, P, st, k, static_cast<float*>(B), ldb, box_rows, true, stream);
    if (e != cudaSuccess) return e;
    return launch_apply_qt_tree_t<ArithF32>(P, st, k, B, ldb, stream);
  }
  if (prec_df(P.precision)) return launch_apply_qt_t<ArithDF>(mapV, P, st, k, B, ldb, box_rows, stream);
  if (P.precision == kPrecF32) return launch_apply_qt_t<ArithF32>(mapV, P, st, k, B, ldb, box_rows, stream);
  return launch_apply_qt_t<ArithF64>(mapV, P, st, k, B, ldb, box_rows, stream);
}

template <class Ar>
static cudaError_t launch_apply_q_t(const CUtensorMap& mapV, const Plan& P, const Store& st, int64_t k, void* B_,
                                    int64_t ldb, int box_rows, cudaStream_t stream) {
  typename Ar::Out* B = static_cast<typename Ar::Out*>(B_);
  const int kb = pick_kb(k);
  const size_t smem = apply_smem_bytes(P, kb);
  cudaError_t e =
      cudaFuncSetAttribute(apply_q_tree_kernel<Ar>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(apply_q_chain_kernel<Ar>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  for (int64_t c0 = 0; c0 < k; c0 += (int64_t)kb * kMaxColBlocks) {
    const int64_t kc = (k - c0 < (int64_t)kb * kMaxColBlocks) ? (k - c0) : (int64_t)kb * kMaxColBlocks;
    const int ncb = (int)((kc + kb - 1) / kb);
    for (int level = P.depth; level >= 1; --level) {
      apply_q_tree_kernel<Ar><<<dim3(P.level_count[level], ncb), kThreads, smem, stream>>>(
          P, st, level, kc, B + gidx(P, 0, c0, ldb), ldb, kb);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    apply_q_chain_kernel<Ar><<<dim3(P.chains, ncb), kThreads, smem, stream>>>(mapV, P, st, kc, B + gidx(P, 0, c0, ldb),
                                                                               ldb, kb, box_rows);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_apply_q(const CUtensorMap& mapV, const Plan& P, const Store& st, int64_t k, void* B,
                           int64_t ldb, int box_rows, cudaStream_t stream) {
  if (ozaki_apply_applies(P, k)) {  // the tree levels, then the chains on the tensor cores
    cudaError_t e = prec_df(P.precision) ? launch_apply_q_tree_t<ArithDF>(P, st, k, B, ldb, stream)
                                         : launch_apply_q_tree_t<ArithF64>(P, st, k, B, ldb, stream);
    if (e != cudaSuccess) return e;
    return launch_apply_ozaki_chains(mapV, P, st, k, static_cast<double*>(B), ldb, box_rows, false, stream);
  }
  if (bf16x3_apply_applies(P, k)) {
    cudaError_t e = launch_apply_q_tree_t<ArithF32>(P, st, k, B, ldb, stream);
    if (e != cudaSuccess) return e;
    return launch_apply_bf16x3_chains(mapV, P, st, k, static_cast<float*>(B), ldb, box_rows, false, stream);
  }
  if (prec_df(P.precision)) return launch_apply_q_t<ArithDF>(mapV, P, st, k, B, ldb, box_rows, stream);
  if (P.precision == kPrecF32) return launch_apply_q_t<ArithF32>(mapV, P, st, k, B, ldb, box_rows, stream);
  return launch_apply_q_t<ArithF64>(mapV, P, st, k, B, ldb, box_rows, stream);
}

}  // namespace tsqr
