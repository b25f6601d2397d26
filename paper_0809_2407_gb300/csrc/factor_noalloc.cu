// tsqr_factor_r_noalloc: the R factor of TSQR for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand over a workspace: code inside another runtime's
// allocator or its callbacks (which must not re-enter an allocator), plugins whose host owns all
// device memory and gives them none, or plain C hosts with no device allocator of their own.
// This entry point needs no workspace: the scratch the factorization uses between thread blocks
// (the chains' and tree nodes' R factors, the arrival counters and a status word) lives in one
// file-scope __device__ array of kStaticScratchBytes, which every GPU that loads this library
// holds until the process exits.  It computes only R (diag(R) >= 0); the implicit Q is
// not kept, so the leaf reflectors and T factors are never written.
//
// The array's address is taken once per device with cudaGetSymbolAddress, on the first call
// made with that device current; make that first call before any stream capture begins.  The
// address is kept for the life of the process, so the entry point must not be used on a device
// after cudaDeviceReset (the library's device array may then live elsewhere).  All calls on a
// device share the array and it keeps the previous call's contents: each call clears the
// counters and status word it needs on its stream, and calls that overlap on the GPU
// (different streams, no ordering between them) race on the array.
//
// A device-side wait that gives up (about one second on a TMA copy) sets the status word in
// the array and makes its block fill R with NaN before it returns: that block then never
// reaches its parent in the tree, so no other block writes R and the NaN stays.
// tsqr_noalloc_status_poll reads the word back.
#include <mutex>

#include "factor_kernels.h"
#include "householder.cuh"
#include "internal.h"

namespace tsqr {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // 8 MiB per GPU
static __device__ __align__(256) unsigned char g_noalloc_scratch[kStaticScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the static scratch on the current device (set up on first use).
tsqr_status_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return internal_fail(TSQR_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return internal_fail(TSQR_ERR_UNSUPPORTED, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return internal_fail(TSQR_ERR_CUDA, cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return TSQR_OK;
}

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// Scratch layout: status word, counters (one per tree node), R of every node.
struct NoallocLayout {
  size_t status, counters, node_r, total;
};

NoallocLayout noalloc_layout(const Plan& P) {
  NoallocLayout L;
  L.status = 0;
  L.counters = 256;
  L.node_r = round256(L.counters + sizeof(int) * (size_t)(P.tree_nodes > 0 ? P.tree_nodes : 1));
  L.total = L.node_r + (size_t)P.total_nodes * P.np * P.np * 8;
  return L;
}

}  // namespace

// The factor kernel's chain-and-tree schedule with nothing of Q stored: the same plain leaf QR,
// flat-tree steps QR([R; A_k]) (Algorithm 2) and structured node QRs of stacked triangles
// (Algorithm 1, eq. fact_2rs), without the T recurrence.
__global__ void __launch_bounds__(kThreads, 1)
    factor_r_kernel(const __grid_constant__ CUtensorMap mapA, const Plan P, double* __restrict__ node_r,
                    int* __restrict__ counters, int* __restrict__ status, double* __restrict__ R_out, int64_t ldr,
                    int box_rows) {
  extern __shared__ char smem_raw[];
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const Tile S{base, P.rows_cap};
  double* red = reinterpret_cast<double*>(base + (size_t)P.rows_cap * P.np * 8);
  double* dvec = red + kThreads;
  double* sc = dvec + P.np;
  double* tau_s = sc + 8;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tau_s + P.np);
  int* flag = reinterpret_cast<int*>(bar + 1);
  const int tid = threadIdx.x;
  const int np = P.np, n = P.n, h = P.h;
  const int g = blockIdx.x;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  const int64_t l0 = chain_first_leaf(P, g), l1 = chain_end_leaf(P, g);
  for (int64_t leaf = l0; leaf < l1; ++leaf) {
    const bool plain = (leaf == l0);
    const int dst = plain ? 0 : np;
    if (!tile_load(S, &mapA, bar, phase, np, leaf * h, h, dst, box_rows, status, flag)) {
      // no R can be produced: this block never arrives at its parent, so the root is never
      // factored and nothing else writes R_out; mark R as invalid for the caller
      const double qnan = __longlong_as_double(0x7FF8000000000000LL);
      for (int i = tid; i < n * n; i += kThreads) R_out[(int64_t)(i / n) * ldr + (i % n)] = qnan;
      return;
    }
    stacked_qr<ArithF64>(S, plain ? PLAIN : CHAIN, dst + h, np, n, tau_s, nullptr, red, dvec, sc);
    if (plain) {
      for (int i = tid; i < np * np; i += kThreads) {
        const int r = i / np, c = i % np;
        if (c < r) *S.ptr(r, c) = 0.0;
      }
    }
    __syncthreads();
  }
  double* Rg = node_r + (size_t)g * np * np;
  for (int i = tid; i < np * np; i += kThreads) {
    const int r = i / np, c = i % np;
    Rg[i] = (c >= r) ? *S.ptr(r, c) : 0.0;
  }
  int idx = g;
  for (int level = 0; level < P.depth; ++level) {
    const int parent = idx / P.arity;
    const int first = parent * P.arity;
    const int q = min(P.arity, P.level_count[level] - first);
    const int pid = P.level_offset[level + 1] + parent;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const int prev = atomicAdd(&counters[pid - P.chains], 1);
      __threadfence();
      *flag = (prev == q - 1) ? 1 : 0;
    }
    __syncthreads();
    if (*flag == 0) return;
    for (int s = 0; s < q; ++s) {
      const double* Rc = node_r + (size_t)(P.level_offset[level] + first + s) * np * np;
      for (int i = tid; i < np * np; i += kThreads) *S.ptr(s * np + i / np, i % np) = __ldcg(Rc + i);
    }
    __syncthreads();
    stacked_qr<ArithF64>(S, NODE, q * np, np, n, tau_s, nullptr, red, dvec, sc);
    double* Rp = node_r + (size_t)pid * np * np;
    for (int i = tid; i < np * np; i += kThreads) {
      const int r = i / np, c = i % np;
      Rp[i] = (c >= r) ? *S.ptr(r, c) : 0.0;
    }
    idx = parent;
  }
  __syncthreads();
  for (int i = tid; i < n * n; i += kThreads) {
    const int r = i / n, c = i % n;
    const double d = (*S.ptr(r, r) < 0.0) ? -1.0 : 1.0;
    R_out[(int64_t)r * ldr + c] = (c >= r) ? d * *S.ptr(r, c) : 0.0;
  }
}

static size_t factor_r_smem_bytes(const Plan& P) {
  return 1024 + (size_t)P.rows_cap * P.np * 8 + kThreads * 8 + P.np * 8 + 8 * 8 + P.np * 8 + 8 + 16;
}

}  // namespace tsqr

extern "C" tsqr_status_t tsqr_factor_r_noalloc(int64_t m, int64_t n, const void* dA, int64_t lda, void* dR,
                                               int64_t ldr, tsqr_stream_t stream) {
  using namespace tsqr;
  if (!dA || !dR) return internal_fail(TSQR_ERR_INVALID_ARG, "A and R must be non-NULL");
  if (n < 1 || m < n) return internal_fail(TSQR_ERR_INVALID_ARG, "need m >= n >= 1");
  if (lda < n || lda % 2 != 0) return internal_fail(TSQR_ERR_INVALID_ARG, "lda must be >= n and even");
  if (ldr < n) return internal_fail(TSQR_ERR_INVALID_ARG, "ldr must be >= n");
  if ((reinterpret_cast<uintptr_t>(dA) & 15) != 0) return internal_fail(TSQR_ERR_INVALID_ARG, "A must be 16-byte aligned");
  Plan P;
  tsqr_status_t s = internal_make_plan(m, n, nullptr, &P);
  if (s != TSQR_OK) return s;
  if (noalloc_layout(P).total > kStaticScratchBytes) {
    // fewer, longer chains until the nodes' R factors fit the static scratch.  The default plan's
    // tree is binary, so it has fewer than 2 x chains nodes in all (chains + chains/2 + ...):
    // 2 x chains node R factors bound the scratch; the check below re-verifies the layout.
    const size_t per_node = (size_t)P.np * P.np * 8;
    const int64_t max_chains = (int64_t)((kStaticScratchBytes - 4096) / per_node / 2);
    if (max_chains < 1) return internal_fail(TSQR_ERR_UNSUPPORTED, "n too large for the 8 MiB static scratch");
    tsqr_opts_t o{};
    o.chain = (int32_t)((P.leaves + max_chains - 1) / max_chains);
    if ((s = internal_make_plan(m, n, &o, &P)) != TSQR_OK) return s;
    if (noalloc_layout(P).total > kStaticScratchBytes)
      return internal_fail(TSQR_ERR_UNSUPPORTED, "problem needs more than the 8 MiB static scratch");
  }
  void* scratch = nullptr;
  if ((s = scratch_address(&scratch)) != TSQR_OK) return s;
  const NoallocLayout L = noalloc_layout(P);
  char* w = static_cast<char*>(scratch);
  int* status = reinterpret_cast<int*>(w + L.status);
  int* counters = reinterpret_cast<int*>(w + L.counters);
  double* node_r = reinterpret_cast<double*>(w + L.node_r);
  const int box_rows = P.h < 256 ? P.h : 256;
  CUtensorMap mapA;
  if ((s = internal_make_map(&mapA, dA, m, n, lda, box_rows)) != TSQR_OK) return s;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(w, 0, L.node_r, cs);  // status word and counters start at zero
  if (e != cudaSuccess) return internal_fail(TSQR_ERR_CUDA, cudaGetErrorString(e));
  const size_t smem = factor_r_smem_bytes(P);
  e = cudaFuncSetAttribute(factor_r_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return internal_fail(TSQR_ERR_CUDA, cudaGetErrorString(e));
  factor_r_kernel<<<P.chains, kThreads, smem, cs>>>(mapA, P, node_r, counters, status, static_cast<double*>(dR), ldr,
                                                      box_rows);
  e = cudaGetLastError();
  if (e != cudaSuccess) return internal_fail(TSQR_ERR_CUDA, cudaGetErrorString(e));
  return TSQR_OK;
}

extern "C" tsqr_status_t tsqr_noalloc_status_poll(tsqr_stream_t stream, void** status_word) {
  using namespace tsqr;
  void* scratch = nullptr;
  tsqr_status_t s = scratch_address(&scratch);
  if (s != TSQR_OK) return s;
  int* word = static_cast<int*>(scratch);  // NoallocLayout::status is offset 0
  if (status_word) *status_word = word;
  int v = 0;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&v, word, sizeof(int), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return internal_fail(TSQR_ERR_CUDA, cudaGetErrorString(e));
  if (v & kStatusTimeout) return internal_fail(TSQR_ERR_TIMEOUT, "a device-side bounded wait timed out; R holds NaN");
  return TSQR_OK;
}
