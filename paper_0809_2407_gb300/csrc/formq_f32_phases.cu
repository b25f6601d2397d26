// Thin Q with FP32 storage (np = 64, h <= 128): the chain recurrence and the leaf products taken
// apart, as for the Ozaki forms (formq_ozaki_phases.cu).
//
// In a flat chain the thin Q flows from the chain's last leaf to its first (Sec. 3.2, V = [I; Y]):
//   M_k = T_k C_k,   C_{k-1} = C_k - M_k,   Q rows of leaf k = -Y_k M_k.
// Three kernels run after the tree levels:
//   1. formq_f32_recur_kernel: per chain, the recurrence on the FP32 pipe.  It carries C from
//      leaf to leaf, so it keeps FP32 rounding rather than the tensor cores' accumulation.  The
//      next leaf's T arrives by a bulk copy into a second buffer while the current M is formed.
//      M_k goes into the first n rows of leaf k's own rows of Q.  The block entering the first
//      leaf goes into node_r[g] (as an FP32 value in an 8-byte slot, the layout of that buffer).
//   2. formq_bf16x3_kernel (formq_bf16x3.cu), split mode: each chain's first leaf.
//   3. formq_bf16x3_leaves_kernel: the products -Y_k M_k of all other leaves.  They are
//      independent, so the kernel is persistent over leaves.  Each FP32 operand value is split
//      into three bf16 terms (bf16x3_pass.cuh).  A term s meets the B terms t = 0 .. 2 - s, which
//      lie one after another, in one MMA of N = 64 (3 - s); region t of the accumulator then
//      holds sum_s A_s B_t, and the epilogue adds the three regions, smallest first.
// A chain that holds a short last leaf (fewer than n rows) is taken whole by kernel 2.  Every
// wait is bounded; a block that gives up sets the status word, waits once more for its copies
// or MMAs in flight and frees its TMEM.
#include "bf16x3_pass.cuh"
#include "factor_kernels.h"

namespace tsqr {
namespace {

// ---- 1. the recurrences ----------------------------------------------------------------------
constexpr int kRT = 256;  // threads of a recurrence block
constexpr int kRLd = 68;  // row stride of C and M in shared memory (floats; rows 16-byte aligned)

size_t f32_recur_smem_bytes() { return 1024 + 2 * 64 * 64 * 8 + 2 * 64 * kRLd * 4 + 2 * 8 + 16; }

__global__ void __launch_bounds__(kRT, 2)
    formq_f32_recur_kernel(const Plan P, const Store st, float* __restrict__ Q, int64_t ldq) {
  extern __shared__ char smem_raw[];
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  f32x2* tbuf = reinterpret_cast<f32x2*>(base);  // 2 x 64 x 64 slots (T of two leaves)
  float* C = reinterpret_cast<float*>(tbuf + 2 * 64 * 64);
  float* M = C + 64 * kRLd;
  uint64_t* bars = reinterpret_cast<uint64_t*>(M + 64 * kRLd);
  int* flag = reinterpret_cast<int*>(bars + 2);
  const int tid = threadIdx.x;
  const int np = 64, n = P.n, h = P.h;
  const int g = blockIdx.x;
  if (formq_chain_short(P, g)) return;  // taken whole by formq_bf16x3_kernel
  const int64_t l0 = chain_first_leaf(P, g), l1 = chain_end_leaf(P, g);
  f32x2* Cg = reinterpret_cast<f32x2*>(st.node_r) + (size_t)g * np * np;
  const f32x2* Tall = reinterpret_cast<const f32x2*>(st.t_leaf);
  if (tid == 0) {
    mbar_init(bars, 1);
    mbar_init(bars + 1, 1);
    fence_mbar_init();
    *flag = 0;
  }
  for (int i = tid; i < np * np; i += kRT) {
    const int a = i >> 6, b = i & 63;
    C[a * kRLd + b] = (P.depth == 0) ? ((a == b && a < n) ? (float)__ldcg(st.signs + a) : 0.f) : Cg[i].hi;
  }
  __syncthreads();
  auto issue_t = [&](int64_t leaf, int buf) {
    mbar_arrive_expect_tx(bars + buf, np * np * 8);
    bf3::bulk_copy(tbuf + buf * np * np, Tall + leaf * np * np, np * np * 8, bars + buf);
  };
  // thread 0 issues the copies and waits for them: its phases and pending flags are the ones
  // that count
  uint32_t phase[2] = {0u, 0u};
  bool pend[2] = {false, false};
  bool alive = true;
  if (l1 - 1 > l0 && tid == 0) {
    issue_t(l1 - 1, 0);
    pend[0] = true;
  }
  int b = 0;
  for (int64_t k = l1 - 1; k > l0; --k, b ^= 1) {
    const int64_t row0 = k * h;
    // the next leaf's T into the other buffer, read last by the previous leaf
    if (k - 1 > l0 && tid == 0) {
      issue_t(k - 1, b ^ 1);
      pend[b ^ 1] = true;
    }
    if (tid == 0) {
      const bool ok = mbar_wait_bounded(bars + b, phase[b], kWaitCycles);
      *flag = ok ? 0 : 1;
      if (ok) {
        phase[b] ^= 1u;
        pend[b] = false;
      } else {
        atomicOr(st.status, kStatusTimeout);
      }
    }
    __syncthreads();
    if (*flag != 0) {
      alive = false;
      break;
    }
    // ---- M = T C (T upper triangular, zero below the diagonal), on the FP32 pipe: each thread
    //      takes 4 rows x 4 columns, so one row of C (a 16-byte load) serves four rows of T
    const f32x2* T = tbuf + b * np * np;
    {
      const int a0 = 4 * (tid >> 4), c0 = 4 * (tid & 15);
      float v[4][4] = {};
      for (int p = a0; p < n; ++p) {
        const float4 cp = *reinterpret_cast<const float4*>(C + p * kRLd + c0);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float t = T[(a0 + r) * np + p].hi;
          v[r][0] = __fmaf_rn(t, cp.x, v[r][0]);
          v[r][1] = __fmaf_rn(t, cp.y, v[r][1]);
          v[r][2] = __fmaf_rn(t, cp.z, v[r][2]);
          v[r][3] = __fmaf_rn(t, cp.w, v[r][3]);
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
        *reinterpret_cast<float4*>(M + (a0 + r) * kRLd + c0) = make_float4(v[r][0], v[r][1], v[r][2], v[r][3]);
    }
    __syncthreads();
    // ---- C -= M, and M (n x n) into the leaf's first n rows of Q for the leaf products
    for (int o = tid; o < np * np; o += kRT) {
      const int a = o >> 6, c = o & 63;
      const float m = M[a * kRLd + c];
      C[a * kRLd + c] = __fsub_rn(C[a * kRLd + c], m);
      if (a < n && c < n) Q[gidx(P, row0 + a, c, ldq)] = m;
    }
    // every read of this T buffer is done before the buffer is refilled
    fence_proxy_async_smem();
    __syncthreads();
  }
  if (alive) {  // the block entering the chain's first leaf, for formq_bf16x3_kernel
    for (int i = tid; i < np * np; i += kRT) Cg[i] = f32x2{C[(i >> 6) * kRLd + (i & 63)], 0.f};
  } else if (tid == 0) {  // copies may still be in flight: one more bounded wait for each
    for (int q = 0; q < 2; ++q)
      if (pend[q]) mbar_wait_bounded(bars + q, phase[q], kWaitCycles);
  }
}

// ---- 3. the leaf products ---------------------------------------------------------------------
// Persistent grid, blocks of 256 threads (two per SM, 256 TMEM columns each), leaves by grid
// stride.  Per leaf: the reflector rows come straight from HBM (each 8-byte slot holds the FP32
// value in its low half; warp w takes rows w + 8 u, two columns per lane), M from the leaf's rows
// of Q; both are split into bf16 terms in shared memory; the three MMAs per K step (A term s
// against B terms 0 .. 2 - s) go out in one commit; the next leaf's rows and M load into
// registers while they run; the epilogue writes -Y M over M.  A row-major Q leaves through a
// shared tile in whole rows (a TMEM lane holds one row, so direct stores would touch a sector per
// lane); a column-major Q is written straight from the lanes, which are then consecutive.
constexpr int kLT = 256;
constexpr int kLWarps = kLT / 32;
constexpr int kLRows = 128 / kLWarps;  // 16 operand rows per warp (h <= 128)
constexpr int kLM = 64 * 32 / kLT;     // 8 pairs (k, k + 1) of M entries per thread
constexpr uint32_t kLTmem = 256;       // 3 regions of 64 columns
constexpr int kStLd = 68;              // row stride of the output tile (floats; rows 16-byte aligned)

// 107 KB: two blocks (512 TMEM columns) share an SM, a third does not fit.
size_t bf16x3_leaves_smem_bytes() {
  return 1024 + 3 * (size_t)bf3::kTermA + 3 * (size_t)bf3::kTermB + 128 * kStLd * 4 + 8 + 8 + 8;
}

__device__ __forceinline__ int64_t next_deferred_f32(const Plan& P, int64_t leaf) {
  while (leaf < P.leaves && !formq_leaf_deferred(P, leaf)) leaf += gridDim.x;
  return leaf;
}

__global__ void __launch_bounds__(kLT, 2)
    formq_bf16x3_leaves_kernel(const Plan P, const Store st, float* __restrict__ Q, int64_t ldq) {
  extern __shared__ char smem_raw[];
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  char* za = base;                  // 3 A terms, 128 operand rows each
  char* zb = za + 3 * bf3::kTermA;  // 3 B terms, 64 operand rows each
  float* stage = reinterpret_cast<float*>(zb + 3 * bf3::kTermB);  // -Y M, 128 x kStLd
  uint64_t* bar = reinterpret_cast<uint64_t*>(stage + 128 * kStLd);
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
  if (warp == 0) oz::tmem_alloc(slot, kLTmem);
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  const uint32_t tmem = *slot;
  uint32_t phase = 0;

  // one leaf's operands in registers: rows warp + 8 u of Y (columns 2 lane, 2 lane + 1), and M
  // entries (k, j), (k + 1, j) with j = tid % 64, k = 2 (tid / 64 + 4 u)
  float2 yr[kLRows], mr[kLM];
  const int j_own = tid & 63;
  auto load = [&](int64_t leaf) {
    const int64_t row0 = leaf * h;
    const int rv = (int)((P.m - row0 < h) ? (P.m - row0) : h);
    const int c = 2 * lane;
#pragma unroll
    for (int u = 0; u < kLRows; ++u) {
      const int r = warp + kLWarps * u;
      float2 y = make_float2(0.f, 0.f);
      if (r < rv && c < n) {
        const double2 d = __ldcg(reinterpret_cast<const double2*>(V + (row0 + r) * ldv + c));
        y.x = __uint_as_float((uint32_t)(unsigned long long)__double_as_longlong(d.x));
        y.y = (c + 1 < n) ? __uint_as_float((uint32_t)(unsigned long long)__double_as_longlong(d.y)) : 0.f;
      }
      yr[u] = y;
    }
#pragma unroll
    for (int u = 0; u < kLM; ++u) {
      const int k = 2 * ((tid >> 6) + 4 * u);
      mr[u].x = (k < n && j_own < n) ? __ldcg(Q + gidx(P, row0 + k, j_own, ldq)) : 0.f;
      mr[u].y = (k + 1 < n && j_own < n) ? __ldcg(Q + gidx(P, row0 + k + 1, j_own, ldq)) : 0.f;
    }
  };

  int64_t leaf = next_deferred_f32(P, blockIdx.x);
  if (leaf < P.leaves) load(leaf);
  bool alive = true;
  while (leaf < P.leaves) {
    const int64_t row0 = leaf * h;
    const int rv = (int)((P.m - row0 < h) ? (P.m - row0) : h);
    // ---- A: the reflector rows' three terms (rows past the leaf are zero)
#pragma unroll
    for (int u = 0; u < kLRows; ++u) {
      const int r = warp + kLWarps * u;
      uint32_t t0[3], t1[3];
      bf3::split3(yr[u].x, t0);
      bf3::split3(yr[u].y, t1);
      const uint32_t off = oz::op_off(r, 2 * lane);
#pragma unroll
      for (int s = 0; s < 3; ++s) *reinterpret_cast<uint32_t*>(za + s * bf3::kTermA + off) = t0[s] | (t1[s] << 16);
    }
    // ---- B: M's terms (output column j, K = M's rows)
#pragma unroll
    for (int u = 0; u < kLM; ++u) {
      const int k = 2 * ((tid >> 6) + 4 * u);
      uint32_t t0[3], t1[3];
      bf3::split3(mr[u].x, t0);
      bf3::split3(mr[u].y, t1);
      const uint32_t off = oz::op_off(j_own, k);
#pragma unroll
      for (int s = 0; s < 3; ++s) *reinterpret_cast<uint32_t*>(zb + s * bf3::kTermB + off) = t0[s] | (t1[s] << 16);
    }
    fence_proxy_async_smem();
    __syncthreads();
    // ---- A term s against B terms 0 .. 2 - s (contiguous) into regions 0 .. 2 - s: one commit
    if (tid == 0) {
      oz::fence_after_sync();
      for (int kk = 0; kk < 4; ++kk)  // K step of 16 bf16 = 32 bytes = 2 descriptor units
        for (int s = 0; s < 3; ++s) {
          const uint64_t ad = oz::sw128_desc(smem_u32(za + s * bf3::kTermA));
          const uint64_t bd = oz::sw128_desc(smem_u32(zb));
          oz::mma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, oz::idesc_bf16(128, 64u * (3 - s)), (s > 0 || kk > 0) ? 1u : 0u);
        }
      oz::mma_commit(bar);
    }
    // ---- the next leaf's operands load while the products run
    const int64_t next = next_deferred_f32(P, leaf + gridDim.x);
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
    // ---- -Y M: warp w reads TMEM lanes 32 (w & 3).. and columns 32 (w >> 2).. of each region
    {
      const int q = warp & 3, i = 32 * q + lane, c0 = 32 * (warp >> 2);
      if (32 * q < rv) {
        uint32_t v[32];
        float acc[32];
        oz::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 128u + (uint32_t)c0, v);  // A_0 B_2
        oz::tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] = __uint_as_float(v[c]);
        oz::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 64u + (uint32_t)c0, v);  // A_0 B_1 + A_1 B_1
        oz::tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] = __fadd_rn(acc[c], __uint_as_float(v[c]));
        oz::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);  // sum_s A_s B_0
        oz::tmem_wait_ld();
        if (P.col_major) {
          if (i < rv) {
#pragma unroll
            for (int c = 0; c < 32; ++c)
              if (c0 + c < n) Q[gidx(P, row0 + i, c0 + c, ldq)] = -__fadd_rn(acc[c], __uint_as_float(v[c]));
          }
        } else {
          float4* srow = reinterpret_cast<float4*>(stage + i * kStLd + c0);
#pragma unroll
          for (int c = 0; c < 32; c += 4)
            srow[c / 4] = make_float4(-__fadd_rn(acc[c], __uint_as_float(v[c])),
                                      -__fadd_rn(acc[c + 1], __uint_as_float(v[c + 1])),
                                      -__fadd_rn(acc[c + 2], __uint_as_float(v[c + 2])),
                                      -__fadd_rn(acc[c + 3], __uint_as_float(v[c + 3])));
        }
      }
      oz::fence_before_sync();
      __syncthreads();
      oz::fence_after_sync();
    }
    // ---- a row-major Q in whole rows; the tile is next written after the next leaf's barrier
    if (!P.col_major) {
      float* qrow0 = Q + row0 * ldq;
      if (n == 64 && (ldq & 3) == 0 && (reinterpret_cast<uintptr_t>(Q) & 15) == 0) {
        for (int e = tid; e < rv * 16; e += kLT) {
          const int r = e >> 4, c4 = e & 15;
          __stcg(reinterpret_cast<float4*>(qrow0 + r * ldq) + c4,
                 *reinterpret_cast<const float4*>(stage + r * kStLd + 4 * c4));
        }
      } else {
        for (int e = tid; e < rv * 64; e += kLT) {
          const int r = e >> 6, c = e & 63;
          if (c < n) __stcg(qrow0 + r * ldq + c, stage[r * kStLd + c]);
        }
      }
    }
    leaf = next;
  }
  // a block that gave up: one more bounded wait for the MMAs in flight before TMEM is freed
  if (!alive && tid == 0) oz::wait_bar(bar, phase ^ 1u);
  oz::fence_before_sync();
  __syncthreads();
  oz::fence_after_sync();
  if (warp == 0) oz::tmem_dealloc(tmem, kLTmem);
}

}  // namespace

cudaError_t launch_formq_f32_recur(const Plan& P, const Store& st, float* Q, int64_t ldq, cudaStream_t stream) {
  const size_t smem = f32_recur_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(formq_f32_recur_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  formq_f32_recur_kernel<<<P.chains, kRT, smem, stream>>>(P, st, Q, ldq);
  return cudaGetLastError();
}

cudaError_t launch_formq_bf16x3_leaves(const Plan& P, const Store& st, float* Q, int64_t ldq, cudaStream_t stream) {
  if (P.leaves <= P.chains) return cudaSuccess;  // every leaf is the first of its chain
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t deferred = P.leaves - P.chains;
  const int blocks = (int)(deferred < 2 * sms ? deferred : 2 * sms);
  const size_t smem = bf16x3_leaves_smem_bytes();
  e = cudaFuncSetAttribute(formq_bf16x3_leaves_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  formq_bf16x3_leaves_kernel<<<blocks, kLT, smem, stream>>>(P, st, Q, ldq);
  return cudaGetLastError();
}

}  // namespace tsqr
