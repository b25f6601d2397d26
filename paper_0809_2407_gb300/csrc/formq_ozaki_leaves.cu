// Thin Q with Ozaki products: the leaf products, taken apart from the chain recurrence.
//
// In a flat chain the thin Q flows from the chain's last leaf to its first: with C_k the n x n
// block carried into leaf k's step (Sec. 3.2, Q_k = I - Y_k T_k Y_k^T with Y_k = [I; V_k]),
//   M_k = T_k C_k,   C_{k-1} = C_k - M_k,   Q rows of leaf k = -V_k M_k.
// Only the n x n recurrence carries the chain's dependence.  formq_ozaki_chain<..., kDefer> runs
// it and leaves each M_k in the first n rows of leaf k's own rows of Q; this kernel then takes
// the h x n products -V_k M_k of all those leaves, which are independent of one another, and
// writes them over M_k.
//
// Persistent grid, one block of 512 threads per SM (all 512 TMEM columns), leaves by grid stride.
// Per leaf:
//   - the reflector rows come straight from HBM (one warp per row, two entries per lane, as a
//     16-byte load), their exponent by a warp reduction, their 8 fixed-point bf16 slices into
//     shared memory as the A operand (128 operand rows; rows past the leaf are zero);
//   - M_k (zero past n) as the B operand against its column exponents;
//   - the 36 slice pairs of weight <= 9 as 144 tcgen05 MMAs into the 8 exact FP32 TMEM groups,
//     in one commit (ozaki.cuh has the scheme and its exactness bound);
//   - while they run, the next leaf's reflector rows and M are loaded into registers;
//   - the int64 epilogue writes -V_k M_k.
// Every wait is bounded; a block that gives up sets the status word, waits once more for its
// MMAs in flight and frees its TMEM.
#include "factor_kernels.h"
#include "ozaki_pass.cuh"

namespace tsqr {
namespace {

constexpr int kWarps = kOzT / 32;          // 16
constexpr int kRowsPerWarp = oz::kM / kWarps;  // 8: the 128 operand rows over the warps
constexpr int kMPerThread = 64 * 32 / kOzT;    // 4 pairs (k, k + 1) of M entries per thread

size_t leaves_smem_bytes() {
  return 1024 + 8 * (size_t)oz::kASliceBytes + 8 * (size_t)oz::kBSliceBytes + 128 * 4 + 64 * 4 + 8 + 8 + 8;
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
  char* bsl = asl + 8 * oz::kASliceBytes;
  int* expA = reinterpret_cast<int*>(bsl + 8 * oz::kBSliceBytes);
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
  if (warp == 0) oz::tmem_alloc(slot, oz::kTmemCols);
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  const uint32_t tmem = *slot;
  uint32_t phase = 0;
  OzSmem z{};  // the epilogue reads the exponents only
  z.expA = expA;
  z.expB = expB;

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
      const uint64_t f0 = slot_fixed<kPairs>(vr[u].x, e), f1 = slot_fixed<kPairs>(vr[u].y, e);
      const uint32_t off = oz::op_off(r, 2 * lane);
#pragma unroll
      for (int s = 1; s <= oz::kSlices; ++s)
        *reinterpret_cast<uint32_t*>(asl + (s - 1) * oz::kASliceBytes + off) = slice_pair(f0, f1, s);
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
        const uint64_t f0 = oz::to_fixed(mr[u].x, e), f1 = oz::to_fixed(mr[u].y, e);
        const uint32_t off = oz::op_off(j_own, k);
#pragma unroll
        for (int s = 1; s <= oz::kSlices; ++s)
          *reinterpret_cast<uint32_t*>(bsl + (s - 1) * oz::kBSliceBytes + off) = slice_pair(f0, f1, s);
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    // ---- the 36 slice products, one commit
    if (tid == 0) {
      oz::fence_after_sync();
      const uint32_t idesc = oz::idesc_bf16(oz::kM, oz::kN);
      for (int s = 1; s <= oz::kSlices; ++s) {
        const uint64_t adesc = oz::sw128_desc(smem_u32(asl + (s - 1) * oz::kASliceBytes));
        for (int t = 1; t <= oz::kSlices + 1 - s; ++t) {
          const uint32_t d = tmem + (uint32_t)(s + t - 2) * 64u;
          const uint64_t bdesc = oz::sw128_desc(smem_u32(bsl + (t - 1) * oz::kBSliceBytes));
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)  // K step of 16 bf16 = 32 bytes = 2 descriptor units
            oz::mma_bf16(d, adesc + 2 * kk, bdesc + 2 * kk, idesc, (s > 1 || kk > 0) ? 1u : 0u);
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
    ozaki_epilogue(z, tmem, rv, [&](int i, int j, double v) {
      if (j < n) Q[gidx(P, row0 + i, j, ldq)] = -v;
    });
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
