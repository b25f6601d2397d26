// Q^T B and Q B with the chains' compact-WY products on the tensor cores (precision modes 2 and
// 3): the Ozaki-split counterpart of the chain part of apply_qt_kernel / apply_q_chain_kernel.
//
// Per chain leaf and 64-column block of B (Sec. 3.2, node update with V = [I; Y], or V unit
// lower trapezoidal on the chain's first leaf):
//   W = C + Y^T B_leaf      (first leaf: W = V^T B_leaf)
//   M = T^T W  (Q^T)  or  M = T W  (Q)
//   C -= M,  B_leaf -= Y M  (first leaf: B_leaf -= V M)
// Each product is an Ozaki-split FP64 product (ozaki.cuh, digit form: 7 balanced base-256 digits,
// 34 digit pairs on tcgen05) with exact FP32 group sums in TMEM.  W's inner dimension is the leaf
// height h (up to 128): it is taken in parts of at most 64 rows, each against its own exponents
// and epilogued into an FP64 partial sum, so every group sum stays below 2^23 as in the thin Q.  M is computed as
// its transpose, with W^T (kept transposed from the epilogue on) as the A operand, so that T's
// slices come from one bulk copy.  B is read
// and written in the caller's layout; the reflector tile arrives by TMA and is loaded twice per
// leaf (once converted with column exponents for W, once with row exponents for the update).
// The tree levels run on the FP64 (or double-float) pipe in their own launches.
// 512 threads, one block per SM (all 512 TMEM columns); needs np = 64 and h <= 128.
#include "factor_kernels.h"
#include "ozaki_pass.cuh"

namespace tsqr {
namespace {

template <bool kPairs, bool kTrans>
__global__ void __launch_bounds__(kOzT, 1)
    apply_ozaki_kernel(const __grid_constant__ CUtensorMap mapV, const Plan P, const Store st, int64_t kcols,
                       double* __restrict__ Bg, int64_t ldb, int box_rows) {
  extern __shared__ char smem_raw[];
  OzSmem z = carve_ozaki(smem_raw, P.h);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int np = 64, n = P.n, h = P.h;
  const int g = blockIdx.x;
  const int64_t col0 = (int64_t)blockIdx.y * 64;
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
  double* const X = z.M;  // W^T (row b holds W's column b), then M (64 x 65)

  // C: zero for Q^T (the first leaf's top rows fill it); for Q the chain's top block of B, the
  // signs applied when there is no tree
  const int64_t top = chain_first_leaf(P, g) * h;
  for (int i = tid; i < np * kOzLd; i += kOzT) {
    const int a = i / kOzLd, b = i % kOzLd;
    double v = 0.0;
    if (!kTrans && a < n && b < 64 && col0 + b < kcols) {
      v = __ldcg(Bg + gidx(P, top + a, col0 + b, ldb));
      if (P.depth == 0) v *= __ldcg(st.signs + a);
    }
    z.C[i] = v;
  }
  const int64_t l0 = chain_first_leaf(P, g), l1 = chain_end_leaf(P, g);
  const int64_t first = kTrans ? l0 : l1 - 1;
  const int64_t step = kTrans ? 1 : -1;
  bool alive = true;
  tile_load_start(z.Y, &mapV, z.bars + 0, np, first * h, h, 0, box_rows);
  for (int64_t leaf = first; leaf >= l0 && leaf < l1 && alive; leaf += step) {
    const bool plain = (leaf == l0);
    const int64_t row0 = leaf * h;
    const int rows_valid = (int)((P.m - row0 < h) ? (P.m - row0) : h);
    const double* Tg = st.t_leaf + leaf * np * np;
    // V's entry (r, a): the stored reflector; on the first leaf 1 on the diagonal, 0 above it
    auto vget = [&](int r, int a) -> double {
      const double v = slot_val<kPairs>(*z.Y.ptr(r, a));
      if (!plain) return v;
      return (a < n) ? (r > a ? v : (r == a ? 1.0 : 0.0)) : 0.0;
    };
    // B_leaf's entry (r, b); on Q's first leaf the top rows are the carried block C
    auto bget = [&](int r, int b) -> double {
      if (!kTrans && plain && r < n) return z.C[r * kOzLd + b];
      const int64_t gr = row0 + r, gc = col0 + b;
      return (r < rows_valid && gc < kcols) ? __ldcg(Bg + gidx(P, gr, gc, ldb)) : 0.0;
    };
    if (!tile_load_finish(z.bars + 0, y_phase, st.status, z.flag)) {
      alive = false;
      break;
    }

    // ---- W = C + V^T B_leaf, over the leaf's rows in parts of 64
    ozaki_zero_a_rows(z, 64, oz::kM);
    for (int r0 = 0; r0 < h; r0 += 64) {
      const int r1 = (r0 + 64 < h) ? r0 + 64 : h;
      for (int j = tid; j < 128; j += kOzT) {
        if (j < 64) z.expA[j] = 0;
        else z.expB[j - 64] = 0;
      }
      __syncthreads();
      {  // column maxima of this part of V and of B_leaf: column = tid & 63, rows strided by 8
        const int c = tid & 63, rg = tid >> 6;
        int ea = 0, eb = 0;
        for (int r = r0 + rg; r < r1; r += kOzT / 64) {
          ea = max(ea, oz::bexp(vget(r, c)));
          eb = max(eb, oz::bexp(bget(r, c)));
        }
        atomicMax(&z.expA[c], ea);
        atomicMax(&z.expB[c], eb);
      }
      __syncthreads();
      // B operand: output column b, k-th entry B_leaf[r0 + k][b] (coalesced along b)
      for (int idx = tid; idx < 64 * 32; idx += kOzT) {
        const int b = idx & 63, k = (idx >> 6) * 2;
        const uint64_t f0 = (r0 + k < r1) ? oz::to_biased54(bget(r0 + k, b), z.expB[b]) : oz::kDigitBias;
        const uint64_t f1 = (r0 + k + 1 < r1) ? oz::to_biased54(bget(r0 + k + 1, b), z.expB[b]) : oz::kDigitBias;
        put_b_digits(z, oz::op_off(b, k), f0, f1);
      }
      // A operand V^T: this part of the tile in fixed point against the column maxima, in place
      // (the tile is loaded again for the update)
      for (int idx = tid; idx < (r1 - r0) * 64; idx += kOzT) {
        const int r = r0 + (idx >> 6), a = idx & 63;
        const double v = vget(r, a);  // reads only element (r, a), which it then replaces
        *reinterpret_cast<uint64_t*>(z.Y.ptr(r, a)) = oz::to_biased54(v, z.expA[a]);
      }
      fence_proxy_async_smem();
      __syncthreads();
      if (!ozaki_mma_pass<true>(  // lanes on a: the tile's row r0 + k is contiguous along a
              z, tmem, 64,
              [&](int a, int k) {
                return (r0 + k < r1) ? *reinterpret_cast<const uint64_t*>(z.Y.ptr(r0 + k, a)) : oz::kDigitBias;
              },
              ph, st.status)) {
        alive = false;
        break;
      }
      const bool first_part = (r0 == 0);
      ozaki_epilogue(z, tmem, 64, [&](int a, int b, double v) {  // stored transposed: W^T
        const int o = b * kOzLd + a;
        X[o] = first_part ? ((plain ? 0.0 : z.C[a * kOzLd + b]) + v) : (X[o] + v);
      });
    }
    if (!alive) break;

    // ---- the tile again for the update, and T, both by copy while M is formed
    tile_load_start(z.Y, &mapV, z.bars + 0, np, row0, h, 0, box_rows);
    if (tid == 0) {
      mbar_arrive_expect_tx(z.bars + 3, np * np * 8);
      bulk_load(z.asl, Tg, np * np * 8, z.bars + 3);
    }
    // ---- M^T = W^T T (Q^T: M = T^T W) or W^T T^T (Q: M = T W); B operand from T: output column
    //      p, k-th entry T[k][p] (Q^T) or T[p][k] (Q).  First the A operand W^T's exponents (the
    //      columns of W) and W's fixed-point form in place.
    for (int j = tid; j < 128; j += kOzT) z.expA[j] = 0;
    __syncthreads();
    for (int idx = tid; idx < np * np; idx += kOzT) warp_max_into(&z.expA[idx >> 6], oz::bexp(X[(idx >> 6) * kOzLd + (idx & 63)]));
    __syncthreads();
    for (int idx = tid; idx < np * np; idx += kOzT) {
      double* p = X + (idx >> 6) * kOzLd + (idx & 63);
      *reinterpret_cast<uint64_t*>(p) = oz::to_biased54(*p, z.expA[idx >> 6]);
    }
    {
      const bool ok = oz_wait_all(z, z.bars + 3, t_phase, st.status);
      t_phase ^= 1u;
      if (!ok) {
        alive = false;
        break;
      }
    }
    const double* Ts = reinterpret_cast<const double*>(z.asl);
    if (kTrans)  // T[k][p]: contiguous along p
      ozaki_b_slices_jmajor(z, [&](int p, int k) { return slot_val<kPairs>(Ts[k * np + p]); });
    else         // T[p][k]: contiguous along k
      ozaki_b_slices(z, [&](int p, int k) { return slot_val<kPairs>(Ts[p * np + k]); });
    ozaki_zero_a_rows(z, 64, oz::kM);  // the copy of T overwrote the A buffers
    if (!ozaki_mma_pass(
            z, tmem, 64, [&](int b, int a) { return *reinterpret_cast<const uint64_t*>(X + b * kOzLd + a); }, ph,
            st.status)) {
      alive = false;
      break;
    }
    ozaki_epilogue(z, tmem, 64, [&](int b, int p, double v) { X[p * kOzLd + b] = v; });  // M[p][b]

    // ---- C -= M; B operand from M: output column b, k-th entry M[k][b]
    if (!plain)
      for (int i = tid; i < np * np; i += kOzT) {
        const int o = (i >> 6) * kOzLd + (i & 63);
        z.C[o] -= X[o];
      }
    ozaki_b_slices(z, [&](int b, int k) { return X[k * kOzLd + b]; });
    if (h < oz::kM) ozaki_zero_a_rows(z, h, oz::kM);
    if (!tile_load_finish(z.bars + 0, y_phase, st.status, z.flag)) {
      alive = false;
      break;
    }
    // A operand V: row exponents, fixed point in place
    for (int r = tid; r < 128; r += kOzT) z.expA[r] = 0;
    __syncthreads();
    for (int idx = tid; idx < h * np; idx += kOzT) warp_max_into(&z.expA[idx >> 6], oz::bexp(vget(idx >> 6, idx & 63)));
    __syncthreads();
    for (int idx = tid; idx < h * np; idx += kOzT) {
      const int r = idx >> 6, a = idx & 63;
      const double v = vget(r, a);
      *reinterpret_cast<uint64_t*>(z.Y.ptr(r, a)) = oz::to_biased54(v, z.expA[r]);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (!ozaki_mma_pass(z, tmem, h, [&](int r, int a) { return *reinterpret_cast<const uint64_t*>(z.Y.ptr(r, a)); },
                        ph, st.status)) {
      alive = false;
      break;
    }
    // the next leaf's tile loads while this leaf's rows are written
    const int64_t next = leaf + step;
    if (next >= l0 && next < l1) tile_load_start(z.Y, &mapV, z.bars + 0, np, next * h, h, 0, box_rows);
    ozaki_epilogue(z, tmem, rows_valid, [&](int r, int b, double v) {
      const int64_t gc = col0 + b;
      if (gc >= kcols) return;
      const double old = (!kTrans && plain && r < n) ? z.C[r * kOzLd + b] : __ldcg(Bg + gidx(P, row0 + r, gc, ldb));
      const double nv = old - v;
      Bg[gidx(P, row0 + r, gc, ldb)] = nv;
      if (kTrans && plain && r < n) z.C[r * kOzLd + b] = nv;  // the chain's top block
    });
  }
  if (alive && kTrans) {
    // publish the chain's top block (the thin part with its signs when there is no tree)
    __syncthreads();
    for (int i = tid; i < n * 64; i += kOzT) {
      const int a = i >> 6, b = i & 63;
      if (col0 + b < kcols) {
        double v = z.C[a * kOzLd + b];
        if (P.depth == 0) v *= __ldcg(st.signs + a);
        Bg[gidx(P, top + a, col0 + b, ldb)] = v;
      }
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

}  // namespace

bool ozaki_apply_applies(const Plan& P, int64_t k) {
  return (P.precision == kPrecOzaki || P.precision == kPrecDFOzaki) && P.np == 64 && P.h <= 128 && k >= kTcApplyMinCols;
}

cudaError_t launch_apply_ozaki_chains(const CUtensorMap& mapV, const Plan& P, const Store& st, int64_t k, double* B,
                                      int64_t ldb, int box_rows, bool trans, cudaStream_t stream) {
  const bool pairs = prec_df(P.precision);
  const size_t smem = formq_ozaki_smem_bytes(P);
  auto kern = trans ? (pairs ? apply_ozaki_kernel<true, true> : apply_ozaki_kernel<false, true>)
                    : (pairs ? apply_ozaki_kernel<true, false> : apply_ozaki_kernel<false, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  constexpr int64_t kColsPerLaunch = 64 * 1024;
  for (int64_t c0 = 0; c0 < k; c0 += kColsPerLaunch) {
    const int64_t kc = (k - c0 < kColsPerLaunch) ? (k - c0) : kColsPerLaunch;
    const int ncb = (int)((kc + 63) / 64);
    kern<<<dim3(P.chains, ncb), kOzT, smem, stream>>>(mapV, P, st, kc, B + gidx(P, 0, c0, ldb), ldb, box_rows);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace tsqr
