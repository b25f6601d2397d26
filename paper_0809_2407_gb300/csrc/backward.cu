// Backward of the thin QR computed by TSQR, for reverse-mode differentiation.
//
// For (Q, R) = qr(A) and a scalar loss with cotangents Qbar = dL/dQ and Rbar = dL/dR, the
// published adjoint of the thin QR of a full-rank A is
//   M = R Rbar^T - Qbar^T Q,   Abar = (Qbar + Q copyltu(M)) R^{-T},
// copyltu(M) = tril(M) + tril(M, -1)^T.  The implicit Q of the factorization gives both
// products without an explicit Q: Z = Q_full^T Qbar has Q^T Qbar in its top n rows (so
// M = R Rbar^T - Z_top^T), and Q_full (Z + [copyltu(M); 0]) = Qbar + Q copyltu(M).  The steps
// are tsqr_apply_qt, the small kernel below, tsqr_apply_q and a row-wise triangular solve.
#include "../../include/tsqr.h"
#include "factor_kernels.h"
#include "internal.h"

namespace tsqr {

// Z_top += copyltu(R Rbar^T - Z_top^T) for the n x n top block of Z (one block of 256 threads),
// in the element type T of the factorization (double, or float with FP32 storage).
template <class T>
__global__ void backward_small_kernel(int n, const T* __restrict__ R, int64_t ldr, const T* __restrict__ Rbar,
                                      int64_t ldrb, T* __restrict__ Z, int64_t ldz) {
  extern __shared__ __align__(16) unsigned char small_raw[];
  T* Ms = reinterpret_cast<T*>(small_raw);  // n x (n + 1)
  const int ld = n + 1;
  for (int o = threadIdx.x; o < n * n; o += blockDim.x) {
    const int i = o / n, j = o % n;
    T v = -Z[(int64_t)j * ldz + i];
    // (R triu(Rbar)^T)_ij: R's strict lower part is structurally zero, so its cotangent is ignored
    if (Rbar != nullptr)
      for (int k = (i > j ? i : j); k < n; ++k) v = fma(R[(int64_t)i * ldr + k], Rbar[(int64_t)j * ldrb + k], v);
    Ms[i * ld + j] = v;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < n * n; o += blockDim.x) {
    const int i = o / n, j = o % n;
    Z[(int64_t)i * ldz + j] += (i >= j) ? Ms[i * ld + j] : Ms[j * ld + i];
  }
}

// B <- B R^{-T} row by row: each row b solves R x = b by back substitution.  A block stages
// blockDim.x rows (128, fewer when R is large) through shared memory (coalesced loads and
// stores), one thread per row.
constexpr int kSolveRows = 128;

template <class T>
__global__ void __launch_bounds__(kSolveRows)
    trsm_rt_kernel(int64_t m, int n, const T* __restrict__ R, int64_t ldr, T* __restrict__ B, int64_t ldb) {
  extern __shared__ __align__(16) unsigned char solve_raw[];
  const int ldt = n + 1;
  const int block_rows = (int)blockDim.x;
  T* Rs = reinterpret_cast<T*>(solve_raw);  // n x (n + 1)
  T* rinv = Rs + n * ldt;                    // n
  T* tile = rinv + n;                        // block_rows x (n + 1)
  for (int o = threadIdx.x; o < n * n; o += blockDim.x) Rs[(o / n) * ldt + o % n] = R[(int64_t)(o / n) * ldr + o % n];
  for (int i = threadIdx.x; i < n; i += blockDim.x) rinv[i] = T(1) / R[(int64_t)i * ldr + i];
  const int64_t r0 = (int64_t)blockIdx.x * block_rows;
  const int rows = (int)((m - r0 < block_rows) ? (m - r0) : block_rows);
  for (int o = threadIdx.x; o < rows * n; o += blockDim.x) tile[(o / n) * ldt + o % n] = B[(r0 + o / n) * ldb + o % n];
  __syncthreads();
  if (threadIdx.x < rows) {
    T* x = tile + threadIdx.x * ldt;
    for (int i = n - 1; i >= 0; --i) {
      T v = x[i];
      for (int k = i + 1; k < n; ++k) v = fma(-Rs[i * ldt + k], x[k], v);
      x[i] = v * rinv[i];
    }
  }
  __syncthreads();
  for (int o = threadIdx.x; o < rows * n; o += blockDim.x) B[(r0 + o / n) * ldb + o % n] = tile[(o / n) * ldt + o % n];
}

// The steps after the argument checks, for element type T.
template <class T>
static tsqr_status_t backward_t(tsqr_handle_t h, int64_t m, int n, const void* dQbar, int64_t ldqb, const void* dRbar,
                                int64_t ldrb, const void* dR, int64_t ldr, void* dAbar, int64_t ldab,
                                tsqr_stream_t stream) {
  constexpr size_t es = sizeof(T);
  // R (n x n) and a block of rows stay in shared memory for the solve
  constexpr size_t kSmemLimit = 232448;
  int solve_rows = kSolveRows;
  auto solve_smem = [n](int rows) { return ((size_t)n * (n + 1) + n + (size_t)rows * (n + 1)) * es; };
  while (solve_rows > 32 && solve_smem(solve_rows) > kSmemLimit) solve_rows /= 2;
  if (solve_smem(solve_rows) > kSmemLimit)
    return internal_fail(TSQR_ERR_UNSUPPORTED,
                         es == 8 ? "tsqr_backward keeps R in shared memory: n must be <= 154 (FP64)"
                                 : "tsqr_backward keeps R in shared memory: n must be <= 224 (FP32)");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  tsqr_status_t s;
  // Z = Q_full^T Qbar (zero when the loss does not depend on Q)
  if (dQbar)
    e = cudaMemcpy2DAsync(dAbar, ldab * es, dQbar, ldqb * es, (size_t)n * es, (size_t)m, cudaMemcpyDeviceToDevice, cs);
  else
    e = cudaMemset2DAsync(dAbar, ldab * es, 0, (size_t)n * es, (size_t)m, cs);
  if (e != cudaSuccess) return internal_fail(TSQR_ERR_CUDA, cudaGetErrorString(e));
  if (dQbar && (s = tsqr_apply_qt(h, n, dAbar, ldab, stream)) != TSQR_OK) return s;
  // Z_top += copyltu(R Rbar^T - Z_top^T)
  const size_t small_smem = (size_t)n * (n + 1) * es;
  e = cudaFuncSetAttribute(backward_small_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small_smem);
  if (e != cudaSuccess) return internal_fail(TSQR_ERR_CUDA, cudaGetErrorString(e));
  backward_small_kernel<T><<<1, 256, small_smem, cs>>>(n, static_cast<const T*>(dR), ldr, static_cast<const T*>(dRbar),
                                                       ldrb, static_cast<T*>(dAbar), ldab);
  if ((e = cudaGetLastError()) != cudaSuccess) return internal_fail(TSQR_ERR_CUDA, cudaGetErrorString(e));
  // B = Q_full Z = Qbar + Q copyltu(M)
  if ((s = tsqr_apply_q(h, n, dAbar, ldab, stream)) != TSQR_OK) return s;
  // Abar = B R^{-T}
  const size_t smem = solve_smem(solve_rows);
  e = cudaFuncSetAttribute(trsm_rt_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return internal_fail(TSQR_ERR_CUDA, cudaGetErrorString(e));
  const int64_t blocks = (m + solve_rows - 1) / solve_rows;
  trsm_rt_kernel<T><<<(unsigned)blocks, solve_rows, smem, cs>>>(m, n, static_cast<const T*>(dR), ldr,
                                                                static_cast<T*>(dAbar), ldab);
  if ((e = cudaGetLastError()) != cudaSuccess) return internal_fail(TSQR_ERR_CUDA, cudaGetErrorString(e));
  return TSQR_OK;
}

}  // namespace tsqr

extern "C" tsqr_status_t tsqr_backward(tsqr_handle_t h, const void* dQbar, int64_t ldqb, const void* dRbar, int64_t ldrb,
                                       const void* dR, int64_t ldr, void* dAbar, int64_t ldab, tsqr_stream_t stream) {
  using namespace tsqr;
  tsqr_info_t info;
  tsqr_status_t s = tsqr_handle_info(h, &info);
  if (s != TSQR_OK) return s;
  const int64_t m = info.m;
  const int n = (int)info.n;
  if (info.layout != TSQR_ROW_MAJOR) return internal_fail(TSQR_ERR_UNSUPPORTED, "tsqr_backward takes row-major matrices");
  if (!dR || !dAbar) return internal_fail(TSQR_ERR_INVALID_ARG, "R and Abar must be non-NULL");
  if (ldr < n || ldab < n || (dQbar && ldqb < n) || (dRbar && ldrb < n))
    return internal_fail(TSQR_ERR_INVALID_ARG, "leading dimensions must be >= n");
  if (info.dtype == TSQR_F32)
    return backward_t<float>(h, m, n, dQbar, ldqb, dRbar, ldrb, dR, ldr, dAbar, ldab, stream);
  return backward_t<double>(h, m, n, dQbar, ldqb, dRbar, ldrb, dR, ldr, dAbar, ldab, stream);
}
