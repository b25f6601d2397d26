// The chain-and-tree schedule of the TSQR factorization, shared by the factor kernels.
//
// Block g owns chain g: leaves [g*chain, ...).  It factors its first leaf with a plain
// Householder QR (Algorithm 1, first step) and each following leaf A_k with the flat-tree step
// QR([R; A_k]) (Algorithm 2), keeping R in shared memory so that only one R per block leaves
// the chip (Sec. 2: the flat tree minimises slow-memory traffic).  Every leaf's reflectors,
// tau and T go to HBM (the reified tree, Sec. 4.1).
//
// The chains' R factors are then reduced up an arity-q tree (Algorithm 1, tree steps) without
// any block waiting for another: each block publishes its R and bumps its parent's counter;
// the block that arrives last stacks the q children's R factors in child order (Algorithm 1:
// "by order of processor ids"), takes their structured QR (eq. fact_2rs) and climbs on.  The
// block that finishes the root writes R with diag(R) >= 0 and the sign vector.
//
// The flat-tree step itself is a parameter: the scheduled FP64-pipe step (chain_qr.cuh) or the
// blocked step whose WY products run on the tensor cores (factor_blocked.cu).
#pragma once

#include "chain_qr.cuh"

namespace tsqr {

template <class E>
struct FactorSmem {
  Tile S;
  E *T_s, *red, *dvec, *sc, *tau_s, *wvec, *invs, *X;
  uint64_t* bar;   // tile loads
  uint64_t* mbar;  // tensor-core completion (the Gram entries on the tensor cores)
  int* flag;
  uint32_t* slot;  // TMEM base address
};

template <class E>
__device__ inline FactorSmem<E> carve_factor(char* raw, const Plan& P) {
  FactorSmem<E> f;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  f.S = Tile{base, P.rows_cap};
  f.T_s = reinterpret_cast<E*>(base + (size_t)P.rows_cap * P.np * 8);
  f.red = f.T_s + tri_size(P.np);
  f.dvec = f.red + kThreads;
  f.sc = f.dvec + P.np;
  f.tau_s = f.sc + 8;
  f.wvec = f.tau_s + P.np;
  f.invs = f.wvec + P.np;
  f.X = f.invs + P.np;
  f.bar = reinterpret_cast<uint64_t*>(f.X + P.np * P.np / 4);
  f.mbar = f.bar + 1;
  f.flag = reinterpret_cast<int*>(f.bar + 2);
  f.slot = reinterpret_cast<uint32_t*>(f.flag + 1);
  return f;
}

// Whether a plan's flat-tree steps can take their Gram entries on the tensor cores: the scheduled
// step of 64 padded columns and 96-row leaves, with the Q factors kept.
__host__ __device__ inline bool gram_tc_applies(const Plan& P) {
  return P.np == 64 && P.h == ChainShape<64>::H && !P.r_only && P.rows_cap >= 64 + ChainShape<64>::H;
}

// The tensor-core Gram's resources inside a FactorSmem: the stage over T_s, red, dvec and sc
// (contiguous in carve_factor and free after the column loop), the column exponents over wvec.
template <class E>
__device__ inline gram::GramTC gram_resources(const FactorSmem<E>& f, uint32_t* phase, uint32_t tmem, int* status) {
  return gram::GramTC{reinterpret_cast<char*>(f.T_s), reinterpret_cast<int*>(f.wvec), f.mbar, phase, tmem, status,
                      f.flag};
}

// The flat-tree step on the tile: the scheduled chain_qr for the default shapes, the generic
// stacked_qr otherwise.  With tc (plans where gram_tc_applies) the 64-column step takes its Gram
// entries on the tensor cores.  False only if a wait on the tensor cores timed out.
template <class Ar>
__device__ inline bool chain_step(const FactorSmem<typename Ar::E>& f, const Plan& P,
                                  const gram::GramTC* tc = nullptr) {
  const int np = P.np, n = P.n, h = P.h;
  const bool want_t = !P.r_only;
  if (np == 64 && h == ChainShape<64>::H) {
    const ChainScratch<Ar, 64> w{f.red, f.dvec, f.wvec, f.invs, f.sc, f.X};
    if (tc != nullptr) return chain_qr<Ar, 64, ChainShape<64>::H, false, true>(f.S, n, f.tau_s, f.T_s, w, want_t, tc);
    chain_qr<Ar, 64>(f.S, n, f.tau_s, f.T_s, w, want_t);
  } else if (np == 32 && h == ChainShape<32>::H) {
    chain_qr<Ar, 32>(f.S, n, f.tau_s, f.T_s, ChainScratch<Ar, 32>{f.red, f.dvec, f.wvec, f.invs, f.sc, f.X}, want_t);
  } else if (np == 16 && h == ChainShape<16>::H) {
    chain_qr<Ar, 16>(f.S, n, f.tau_s, f.T_s, ChainScratch<Ar, 16>{f.red, f.dvec, f.wvec, f.invs, f.sc, f.X}, want_t);
  } else {
    stacked_qr<Ar>(f.S, CHAIN, np + h, np, n, f.tau_s, want_t ? f.T_s : nullptr, f.red, f.dvec, f.sc);
  }
  return true;
}

// A binary tree node (q <= 2 children) by the scheduled chain step in its structured form
// (kTri): the second child's triangle (zeros for a lone child) is the block under the first
// child's R, padded with zero rows to a height the step's schedule takes (64 rows for np = 64 and
// 32, 128 for np = 16); column j's reflector and updates visit only the bottom rows 0..j that
// eq. fact_2rs leaves nonzero, about (2/3) n^3 flops instead of the dense step's 2 n^3.  False
// (nothing done) when the node does not fit that form.
template <class Ar>
__device__ inline bool node_step(const FactorSmem<typename Ar::E>& f, const Plan& P, int q) {
  using E = typename Ar::E;
  const int np = P.np, n = P.n;
  const int H = (np == 16) ? 128 : 64;
  if (q > 2 || np < 16 || P.rows_cap < np + H) return false;
  const int lnp = __ffs(np) - 1;
  for (int i = threadIdx.x; i < (np + H - q * np) * np; i += kThreads)
    at<E>(f.S, q * np + (i >> lnp), i & (np - 1)) = Ar::zero();
  __syncthreads();
  const bool want_t = !P.r_only;
  if (np == 64)
    chain_qr<Ar, 64, 64, true>(f.S, n, f.tau_s, f.T_s, ChainScratch<Ar, 64>{f.red, f.dvec, f.wvec, f.invs, f.sc, f.X},
                               want_t);
  else if (np == 32)
    chain_qr<Ar, 32, 64, true>(f.S, n, f.tau_s, f.T_s, ChainScratch<Ar, 32>{f.red, f.dvec, f.wvec, f.invs, f.sc, f.X},
                               want_t);
  else
    chain_qr<Ar, 16, 128, true>(f.S, n, f.tau_s, f.T_s,
                                ChainScratch<Ar, 16>{f.red, f.dvec, f.wvec, f.invs, f.sc, f.X}, want_t);
  __syncthreads();
  return true;
}

// Rows [r0, r0 + rows) of the tile arrive from TMA as FP64; in double-float mode they are split
// into (hi, lo) pairs in place.
template <class Ar>
__device__ inline void convert_rows_in(const Tile& S, int r0, int rows, int np) {
  if constexpr (Ar::kPrecision != 0) {
    const int lnp = __ffs(np) - 1;  // np is a power of two
    for (int i = threadIdx.x; i < rows * np; i += kThreads) {
      double* p = S.ptr(r0 + (i >> lnp), i & (np - 1));
      *reinterpret_cast<typename Ar::E*>(p) = Ar::from_f64(*p);
    }
    __syncthreads();
  }
}

// Chain g of one factorization, then the tree above it while this block arrives last.  step(f, P)
// takes the flat-tree step QR([R; A_k]) on the tile (R in rows 0..np-1, A_k below), leaving tau
// in f.tau_s and, unless P.r_only, T packed in f.T_s; false if a bounded wait gave up (the
// status word is then set and the block stops).
template <class Ar, class Step>
__device__ __forceinline__ void factor_chain(const CUtensorMap* mapA_p, const CUtensorMap* mapV_p, const Plan& P,
                                             const Store& st, typename Ar::Out* __restrict__ R_out, int64_t ldr,
                                             int box_rows, int g, const FactorSmem<typename Ar::E>& f, Step step) {
  using E = typename Ar::E;
  const Tile& S = f.S;
  const int tid = threadIdx.x;
  const int np = P.np, n = P.n, h = P.h;
  const int lnp = __ffs(np) - 1;  // np is a power of two
  E* tau_leaf = reinterpret_cast<E*>(st.tau_leaf);
  E* t_leaf = reinterpret_cast<E*>(st.t_leaf);
  E* node_r = reinterpret_cast<E*>(st.node_r);
  if (tid == 0) {
    mbar_init(f.bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;

  // ---- the chain: plain QR of the first leaf, then QR([R; A_k]) for each following leaf
  const int64_t l0 = chain_first_leaf(P, g), l1 = chain_end_leaf(P, g);
  for (int64_t leaf = l0; leaf < l1; ++leaf) {
    const bool plain = (leaf == l0);
    const int dst = plain ? 0 : np;
    const int64_t row0 = leaf * h;
    if (!tile_load(S, mapA_p, f.bar, phase, np, row0, h, dst, box_rows, st.status, f.flag)) {
      if (tid == 0) tma_store_wait_all();
      return;
    }
    convert_rows_in<Ar>(S, dst, h, np);
    if (plain) {
      stacked_qr<Ar>(S, PLAIN, h, np, n, f.tau_s, P.r_only ? nullptr : f.T_s, f.red, f.dvec, f.sc);
    } else if (!step(f, P)) {
      if (tid == 0) tma_store_wait_all();
      return;
    }
    if (!P.r_only) {  // the leaf's reflectors, tau and T: the reified tree (Sec. 4.1)
      tile_store(S, mapV_p, np, row0, h, dst, box_rows);
      E* tau_g = tau_leaf + leaf * np;
      E* T_g = t_leaf + leaf * np * np;
      for (int i = tid; i < np; i += kThreads) tau_g[i] = f.tau_s[i];
      for (int i = tid; i < np * np; i += kThreads) {
        const int a = (i >> lnp), b = (i & (np - 1));
        T_g[i] = (b >= a && b < n) ? f.T_s[tri_off(a, np) + (b - a)] : Ar::zero();
      }
      tile_store_drain();
    } else {
      __syncthreads();
    }
    if (plain) {  // rows 0..np-1 now carry R above the diagonal; clear the reflector part below
      for (int i = tid; i < np * np; i += kThreads) {
        const int r = (i >> lnp), c = (i & (np - 1));
        if (c < r) at<E>(S, r, c) = Ar::zero();
      }
      __syncthreads();
    }
  }

  // ---- publish the chain's R (level-0 node g); the reflector stores are complete first
  if (tid == 0) tma_store_wait_all();
  {
    E* Rg = node_r + (size_t)g * np * np;
    for (int i = tid; i < np * np; i += kThreads) {
      const int r = (i >> lnp), c = (i & (np - 1));
      Rg[i] = (c >= r) ? at<E>(S, r, c) : Ar::zero();
    }
  }

  // ---- climb the tree while this block is the last child to arrive
  int idx = g;
  for (int level = 0; level < P.depth; ++level) {
    const int parent = idx / P.arity;
    const int first = parent * P.arity;
    const int q = min(P.arity, P.level_count[level] - first);
    const int pid = P.level_offset[level + 1] + parent;
    const int tn = pid - P.chains;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const int prev = atomicAdd(&st.counters[tn], 1);
      __threadfence();
      *f.flag = (prev == q - 1) ? 1 : 0;
    }
    __syncthreads();
    if (*f.flag == 0) return;
    // stack the children's R factors in child order: child s at rows s*np..s*np+np-1
    for (int s = 0; s < q; ++s) {
      const double* Rc = st.node_r + (size_t)(P.level_offset[level] + first + s) * np * np;
      for (int i = tid; i < np * np; i += kThreads) *S.ptr(s * np + (i >> lnp), (i & (np - 1))) = __ldcg(Rc + i);
    }
    __syncthreads();
    if (!node_step<Ar>(f, P, q))
      stacked_qr<Ar>(S, NODE, q * np, np, n, f.tau_s, P.r_only ? nullptr : f.T_s, f.red, f.dvec, f.sc);
    if (!P.r_only) {  // the node's reflectors (eq. fact_2rs), tau and T
      E* Y = reinterpret_cast<E*>(st.node_y) + (size_t)tn * (P.arity - 1) * np * np;
      for (int s = 1; s < P.arity; ++s) {
        E* Ys = Y + (size_t)(s - 1) * np * np;
        for (int i = tid; i < np * np; i += kThreads) {
          const int r = (i >> lnp), c = (i & (np - 1));
          Ys[i] = (s < q && c >= r) ? at<E>(S, s * np + r, c) : Ar::zero();
        }
      }
      for (int i = tid; i < np; i += kThreads) reinterpret_cast<E*>(st.node_tau)[(size_t)tn * np + i] = f.tau_s[i];
      E* Tn = reinterpret_cast<E*>(st.node_t) + (size_t)tn * np * np;
      for (int i = tid; i < np * np; i += kThreads) {
        const int a = (i >> lnp), b = (i & (np - 1));
        Tn[i] = (b >= a && b < n) ? f.T_s[tri_off(a, np) + (b - a)] : Ar::zero();
      }
    }
    E* Rp = node_r + (size_t)pid * np * np;
    for (int i = tid; i < np * np; i += kThreads) {
      const int r = (i >> lnp), c = (i & (np - 1));
      Rp[i] = (c >= r) ? at<E>(S, r, c) : Ar::zero();
    }
    idx = parent;
  }

  // ---- root: R <- D R with D = diag(sign(R_jj)), sign(0) = +1
  __syncthreads();
  for (int j = tid; j < np; j += kThreads) st.signs[j] = (j < n && Ar::is_neg(at<E>(S, j, j))) ? -1.0 : 1.0;
  using Out = typename Ar::Out;
  for (int i = tid; i < n * n; i += kThreads) {
    const int r = i / n, c = i % n;
    const Out d = Ar::is_neg(at<E>(S, r, r)) ? Out(-1) : Out(1);
    R_out[gidx(P, r, c, ldr)] = (c >= r) ? d * Ar::to_out(at<E>(S, r, c)) : Out(0);
  }
}

}  // namespace tsqr
