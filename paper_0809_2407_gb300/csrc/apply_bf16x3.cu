// Q^T B and Q B of an FP32-storage factorization with the chains' compact-WY products on the
// tensor cores: the bf16x3 counterpart of the chain part of apply_qt_kernel / apply_q_chain_kernel.
//
// Per chain leaf and 64-column block of B (Sec. 3.2, node update with V = [I; Y], or V unit
// lower trapezoidal on the chain's first leaf):
//   W = C + Y^T B_leaf      (first leaf: W = V^T B_leaf)
//   M = T^T W  (Q^T)  or  M = T W  (Q)
//   C -= M,  B_leaf -= Y M  (first leaf: B_leaf -= V M)
// Y^T B_leaf and Y M are bf16x3 term products on tcgen05 (bf16x3_pass.cuh); Y^T B_leaf runs over
// the leaf height in parts of 64 rows accumulated in TMEM.  M = T^T W stays on the FP32 pipe: it
// acts on the carried block C, which every leaf of the chain updates, so it takes FP32 rounding
// rather than the tensor cores' accumulation (the thin Q makes the same split); Y^T B_leaf only
// adds each leaf's own rows once.  B is read and written in the caller's layout; the tree levels
// run on the FP32 pipe in their own launches.
// One block of 256 threads per chain and column block, one SM each; 64 TMEM columns.
#include "bf16x3_pass.cuh"
#include "factor_kernels.h"

namespace tsqr {
namespace {

using namespace bf3;

template <bool kTrans>
__global__ void __launch_bounds__(kT3, 1)
    apply_bf16x3_kernel(const __grid_constant__ CUtensorMap mapV, const Plan P, const Store st, int64_t kcols,
                        float* __restrict__ Bg, int64_t ldb, int box_rows) {
  extern __shared__ char smem_raw[];
  Tc3Smem z = carve_tc3(smem_raw, P.h);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int np = 64, n = P.n, h = P.h;
  const int g = blockIdx.x;
  const int64_t col0 = (int64_t)blockIdx.y * 64;
  if (tid == 0) {
    for (int b = 0; b < 3; ++b) mbar_init(z.bars + b, 1);
    fence_mbar_init();
    *z.flag = 0;
  }
  if (warp == 0) oz::tmem_alloc(z.slot, kTmemCols3);
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  const uint32_t tmem = *z.slot;
  uint32_t mma_phase = 0, y_phase = 0, t_phase = 0;
  float* const W = reinterpret_cast<float*>(z.b);  // W (64 x 65) between the two products

  // C: zero for Q^T (the first leaf's top rows fill it); for Q the chain's top block of B, the
  // signs applied when there is no tree
  const int64_t top = chain_first_leaf(P, g) * h;
  for (int i = tid; i < np * kLd; i += kT3) {
    const int a = i / kLd, b = i % kLd;
    float v = 0.f;
    if (!kTrans && a < n && b < 64 && col0 + b < kcols) {
      v = __ldcg(Bg + gidx(P, top + a, col0 + b, ldb));
      if (P.depth == 0) v *= (float)__ldcg(st.signs + a);
    }
    z.C[i] = v;
  }
  const int64_t l0 = chain_first_leaf(P, g), l1 = chain_end_leaf(P, g);
  const int64_t first = kTrans ? l0 : l1 - 1;
  const int64_t step = kTrans ? 1 : -1;
  bool alive = true;
  for (int64_t leaf = first; leaf >= l0 && leaf < l1 && alive; leaf += step) {
    const bool plain = (leaf == l0);
    const int64_t row0 = leaf * h;
    const int rows_valid = (int)((P.m - row0 < h) ? (P.m - row0) : h);
    const f32x2* Tg = reinterpret_cast<const f32x2*>(st.t_leaf) + leaf * np * np;
    // V's entry (r, a): the stored reflector; on the first leaf 1 on the diagonal, 0 above it
    auto vget = [&](int r, int a) -> float {
      const float v = yv(z.Y, r, a);
      if (!plain) return v;
      return (a < n) ? (r > a ? v : (r == a ? 1.f : 0.f)) : 0.f;
    };
    // B_leaf's entry (r, b); on Q's first leaf the top rows are the carried block C
    auto bget = [&](int r, int b) -> float {
      if (!kTrans && plain && r < n) return z.C[r * kLd + b];
      const int64_t gc = col0 + b;
      return (r < rows_valid && gc < kcols) ? __ldcg(Bg + gidx(P, row0 + r, gc, ldb)) : 0.f;
    };
    // ---- both loads of the leaf start now: T by a bulk copy, the reflector tile by TMA
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      mbar_arrive_expect_tx(z.bars + 2, np * np * 8);
      bulk_copy(z.T, Tg, np * np * 8, z.bars + 2);
      mbar_arrive_expect_tx(z.bars + 0, (uint32_t)h * np * 8);
      for (int pnl = 0; pnl < np / 16; ++pnl)
        for (int r = 0; r < h; r += box_rows)
          tma_load_2d(z.Y.base + (size_t)pnl * h * 128 + (size_t)r * 128, &mapV, z.bars + 0, pnl * 16,
                      (int)(row0 + r));
    }
    {
      const bool ok = wait_all(z, z.bars + 0, y_phase, st.status);
      y_phase ^= 1u;
      if (!ok) {
        alive = false;
        break;
      }
    }
    // ---- V^T B_leaf in TMEM, over the leaf's rows in parts of 64: A = V^T (rows a, k = row),
    //      B = B_leaf (output column b, k-th entry B_leaf[r0 + k][b])
    zero_a_rows(z.a, 64);
    for (int r0 = 0; r0 < h; r0 += 64) {
      const int r1 = (r0 + 64 < h) ? r0 + 64 : h;
      write_terms(z.a, kTermA, 64, [&](int a, int k) { return (r0 + k < r1) ? vget(r0 + k, a) : 0.f; });
      for (int idx = tid; idx < 64 * 32; idx += kT3) {  // coalesced along b
        const int b = idx & 63, k = (idx >> 6) * 2;
        uint32_t t0[3], t1[3];
        split3((r0 + k < r1) ? bget(r0 + k, b) : 0.f, t0);
        split3((r0 + k + 1 < r1) ? bget(r0 + k + 1, b) : 0.f, t1);
        const uint32_t off = oz::op_off(b, k);
#pragma unroll
        for (int s = 0; s < 3; ++s) *reinterpret_cast<uint32_t*>(z.b + s * kTermB + off) = t0[s] | (t1[s] << 16);
      }
      if (!mma_terms(z, tmem, mma_phase, st.status, r0 > 0)) {
        alive = false;
        break;
      }
    }
    if (!alive) break;
    // ---- W = C + V^T B_leaf (into the B-term buffers, free until the second product)
    epilogue(tmem, 64, [&](int a, int b, float v) {
      W[a * kLd + b] = plain ? v : __fadd_rn(z.C[a * kLd + b], v);
    });
    // ---- M = T^T W or T W on the FP32 pipe (T upper triangular); C -= M
    {
      const bool ok = wait_all(z, z.bars + 2, t_phase, st.status);
      t_phase ^= 1u;
      if (!ok) {
        alive = false;
        break;
      }
    }
    for (int o = tid; o < np * np; o += kT3) {
      const int p = o >> 6, b = o & 63;
      float v = 0.f;
      if (p < n) {
        if (kTrans) {
          for (int a = 0; a <= p; ++a) v = __fmaf_rn(z.T[a * np + p].hi, W[a * kLd + b], v);
        } else {
          for (int a = p; a < n; ++a) v = __fmaf_rn(z.T[p * np + a].hi, W[a * kLd + b], v);
        }
      }
      z.M[p * kLd + b] = v;
    }
    __syncthreads();
    if (!plain)
      for (int i = tid; i < np * np; i += kT3) {
        const int o = (i >> 6) * kLd + (i & 63);
        z.C[o] = __fsub_rn(z.C[o], z.M[o]);
      }
    // ---- B_leaf -= V M: A = V (rows of the leaf), B = M (output column b, k-th entry M[k][b])
    write_terms(z.b, kTermB, 64, [&](int b, int k) { return z.M[k * kLd + b]; });
    write_terms(z.a, kTermA, h, [&](int r, int a) { return vget(r, a); });
    if (h < 128) zero_a_rows(z.a, h);
    if (!mma_terms(z, tmem, mma_phase, st.status)) {
      alive = false;
      break;
    }
    epilogue(tmem, rows_valid, [&](int r, int b, float v) {
      const int64_t gc = col0 + b;
      if (gc >= kcols) return;
      const float old = (!kTrans && plain && r < n) ? z.C[r * kLd + b] : __ldcg(Bg + gidx(P, row0 + r, gc, ldb));
      const float nv = __fsub_rn(old, v);
      Bg[gidx(P, row0 + r, gc, ldb)] = nv;
      if (kTrans && plain && r < n) z.C[r * kLd + b] = nv;  // the chain's top block
    });
  }
  if (alive && kTrans) {
    // publish the chain's top block (the thin part with its signs when there is no tree)
    __syncthreads();
    for (int i = tid; i < n * 64; i += kT3) {
      const int a = i >> 6, b = i & 63;
      if (col0 + b < kcols) {
        float v = z.C[a * kLd + b];
        if (P.depth == 0) v *= (float)__ldcg(st.signs + a);
        Bg[gidx(P, top + a, col0 + b, ldb)] = v;
      }
    }
  }
  // after a timeout, give the copies and MMAs in flight one more bounded wait before TMEM is freed
  if (!alive && tid == 0) {
    oz::wait_bar(z.bars + 1, mma_phase);
    oz::wait_bar(z.bars + 0, y_phase);
    oz::wait_bar(z.bars + 2, t_phase);
  }
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  if (warp == 0) oz::tmem_dealloc(tmem, kTmemCols3);
}

}  // namespace

bool bf16x3_apply_applies(const Plan& P, int64_t k) {
  return P.precision == kPrecF32 && P.np == 64 && P.h <= 128 && k >= kTcApplyMinCols;
}

cudaError_t launch_apply_bf16x3_chains(const CUtensorMap& mapV, const Plan& P, const Store& st, int64_t k, float* B,
                                       int64_t ldb, int box_rows, bool trans, cudaStream_t stream) {
  const size_t smem = formq_bf16x3_smem_bytes(P);
  auto kern = trans ? apply_bf16x3_kernel<true> : apply_bf16x3_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  constexpr int64_t kColsPerLaunch = 64 * 1024;
  for (int64_t c0 = 0; c0 < k; c0 += kColsPerLaunch) {
    const int64_t kc = (k - c0 < kColsPerLaunch) ? (k - c0) : kColsPerLaunch;
    const int ncb = (int)((kc + 63) / 64);
    kern<<<dim3(P.chains, ncb), kT3, smem, stream>>>(mapV, P, st, kc, B + gidx(P, 0, c0, ldb), ldb, box_rows);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace tsqr
