// C-ABI of libtsqr.so: argument checks, the reduction-tree plan, the workspace layout, TMA
// descriptors and the handle.  Declared in include/tsqr.h.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/tsqr.h"
#include "factor_kernels.h"

using tsqr::Plan;
using tsqr::Store;

struct tsqr_batch_s {
  int count = 0, precision = 0;
  int total_chains = 0, max_depth = 0;
  int factor_blocks = 1;  // resident blocks of the persistent factor launch
  // thin Q: chains on the FP64/FP32-pipe kernel, then chains whose WY products run on the tensor
  // cores (tc: 0 none, 1 Ozaki, 2 Ozaki from double-float slots, 3 bf16x3)
  const tsqr::BatchWork* d_formq_work = nullptr;
  int formq_blocks = 0;
  const tsqr::BatchWork* d_tc_work = nullptr;
  int tc_blocks = 0, tc = 0;
  size_t smem_tc = 0;
  size_t smem_factor = 0, smem_formq = 0;
  tsqr::BatchItem* d_items = nullptr;
  tsqr::BatchWork* d_chain_work = nullptr;
  std::vector<const tsqr::BatchWork*> d_level_work;
  std::vector<int> level_blocks;
  int* d_counters = nullptr;
  size_t counters_bytes = 0;
  int* d_status = nullptr;
  bool has_q = false;
  bool widen = false;  // FP32 storage: A is widened into V before the factorization
  struct Stage {
    const double* A;
    int64_t lda;
    double* V;
    int64_t ldv, m;
    int n;
  };
  std::vector<Stage> stages;
};

struct tsqr_handle_s {
  Plan P;
  Store st;
  CUtensorMap mapV;
  int box_rows;
  int inplace;
  // n > 64: a right-looking blocked QR whose panels are TSQRs (the panel factorization and
  // trailing update of Sec. 6, Algorithm 3, on one GPU).  Panel p covers columns c_p..c_p+w_p-1
  // and rows c_p..m-1 of the updated matrix; Q = Q_0 diag(I, Q_1) diag(I, Q_2) ...
  std::vector<tsqr_handle_s*> panels;
  int64_t m = 0, n = 0;
  int f32 = 0;  // FP32 storage (A, R, Q and B are float)
  ~tsqr_handle_s() {
    for (tsqr_handle_s* p : panels) delete p;
  }
};

namespace {

thread_local std::string g_last_error;

tsqr_status_t fail(tsqr_status_t s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

tsqr_status_t cuda_fail(cudaError_t e, const char* where) {
  return fail(TSQR_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

constexpr size_t kSmemLimit = 232448;  // opt-in shared memory per block on GB300

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 152;
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    return 152;
  }
  return sms;
}

int default_leaf_h(int np) {
  switch (np) {
    case 16: return 512;
    case 32: return 256;
    default:
      return 96;  // np = 64: tile + packed T fit twice in one SM's shared memory
  }
}

// Builds the plan of an m x n factorization; see Plan in common.cuh.  FP32 storage (f32) runs
// the FP32 arithmetic, Plan::precision 3.
tsqr_status_t make_plan(int64_t m, int64_t n, const tsqr_opts_t* o, Plan* P, bool f32 = false) {
  tsqr_opts_t d{};
  if (!o) o = &d;
  if (n < 1 || m < n) return fail(TSQR_ERR_INVALID_ARG, "need m >= n >= 1");
  int np = 16;
  while (np < n) np *= 2;
  if (np > 64) return fail(TSQR_ERR_UNSUPPORTED, "n > 64 is not supported by this build");
  if (o->precision < 0 || o->precision > 3)
    return fail(TSQR_ERR_UNSUPPORTED,
                "precision must be 0 (native FP64), 1 (double-float), 2 (Ozaki WY) or 3 (double-float + Ozaki WY)");
  if (f32 && o->precision != 0)
    return fail(TSQR_ERR_UNSUPPORTED, "TSQR_F32 runs FP32 arithmetic: precision must be 0");
  if (f32 && o->inplace) return fail(TSQR_ERR_UNSUPPORTED, "TSQR_F32 keeps A read-only (inplace is not supported)");
  if (o->r_only && o->inplace) return fail(TSQR_ERR_INVALID_ARG, "r_only stores no reflectors: inplace does not apply");
  const int arity = o->arity ? o->arity : 2;
  if (arity < 2 || arity > tsqr::kMaxArity) return fail(TSQR_ERR_INVALID_ARG, "arity must be in 2..8");
  int h = o->leaf_h ? o->leaf_h : default_leaf_h(np);
  if (h < np || h % 8 != 0 || (h > 256 && h % 256 != 0))
    return fail(TSQR_ERR_INVALID_ARG, "leaf_h must be a multiple of 8, >= padded n, and a multiple of 256 above 256");
  if (o->chain < 0) return fail(TSQR_ERR_INVALID_ARG, "chain must be >= 0");
  std::memset(P, 0, sizeof(Plan));
  P->m = m;
  P->n = (int)n;
  P->np = np;
  P->h = h;
  P->arity = arity;
  P->precision = f32 ? tsqr::kPrecF32 : o->precision;
  P->r_only = o->r_only ? 1 : 0;
  P->leaves = (m + h - 1) / h;
  int64_t chain = o->chain;
  if (chain == 0) {
    // Native FP64: two factor blocks per SM, one chain each.  Double-float: eight times as many
    // shorter chains, because the loss of orthogonality grows with the number of reflectors on
    // a row's path to the root (about sqrt(chain * n) units of roundoff), and the double-float
    // unit roundoff is 2^-46.
    const int blocks = (tsqr::prec_df(o->precision) ? 16 : 2) * device_sms();
    chain = (P->leaves + blocks - 1) / blocks;
  }
  if (chain > P->leaves) chain = P->leaves;
  int64_t chains = (P->leaves + chain - 1) / chain;
  const int64_t rows_last = m - (P->leaves - 1) * h;
  // a chain's first leaf must hold at least n real rows (its top block lives there)
  if (chains > 1 && (P->leaves - 1) % chain == 0 && rows_last < n) chains -= 1;
  if (chains > (int64_t)1 << 30) return fail(TSQR_ERR_UNSUPPORTED, "too many chains");
  P->chain = (int)chain;
  P->chains = (int)chains;
  int count = P->chains, depth = 0, offset = 0;
  P->level_count[0] = count;
  P->level_offset[0] = 0;
  offset = count;
  while (count > 1) {
    if (depth + 1 > tsqr::kMaxLevels) return fail(TSQR_ERR_UNSUPPORTED, "tree too deep");
    count = (count + arity - 1) / arity;
    ++depth;
    P->level_count[depth] = count;
    P->level_offset[depth] = offset;
    offset += count;
  }
  P->depth = depth;
  P->total_nodes = offset;
  P->tree_nodes = offset - P->chains;
  int rows_cap = np + h;
  if (arity * np > rows_cap) rows_cap = arity * np;
  P->rows_cap = (rows_cap + 7) / 8 * 8;
  if (tsqr::factor_smem_bytes(*P) > kSmemLimit || tsqr::formq_smem_bytes(*P) > kSmemLimit ||
      tsqr::apply_smem_bytes(*P, 32) > kSmemLimit ||
      (tsqr::ozaki_form_q_applies(*P) && tsqr::formq_ozaki_smem_bytes(*P) > kSmemLimit) ||
      (tsqr::bf16x3_form_q_applies(*P) && tsqr::formq_bf16x3_smem_bytes(*P) > kSmemLimit))
    return fail(TSQR_ERR_UNSUPPORTED, "leaf_h/arity too large for shared memory at this n");
  return TSQR_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t v, tau_leaf, t_leaf, node_r, node_y, node_tau, node_t, signs, counters, status, total;
  int64_t ldv;
};

Layout make_layout(const Plan& P, bool inplace) {
  Layout L{};
  const size_t np = (size_t)P.np, np2 = np * np;
  L.ldv = (P.n + 1) / 2 * 2;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  const size_t q = P.r_only ? 0 : 1;  // R alone keeps no reflectors, tau or T (V only stages A)
  L.v = take(inplace ? 0 : (size_t)P.m * L.ldv * 8);
  L.tau_leaf = take(q * (size_t)P.leaves * np * 8);
  L.t_leaf = take(q * (size_t)P.leaves * np2 * 8);
  L.node_r = take((size_t)P.total_nodes * np2 * 8);
  L.node_y = take(q * (size_t)P.tree_nodes * (P.arity - 1) * np2 * 8);
  L.node_tau = take(q * (size_t)P.tree_nodes * np * 8);
  L.node_t = take(q * (size_t)P.tree_nodes * np2 * 8);
  L.signs = take(np * 8);
  L.counters = take((size_t)(P.tree_nodes > 0 ? P.tree_nodes : 1) * tsqr::kMaxColBlocks * sizeof(int));
  L.status = take(256);
  L.total = off;
  return L;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// Row-major m x n FP64 matrix, boxes of 16 columns x box_rows rows, 128-byte swizzle,
// zero fill outside the matrix.
tsqr_status_t make_map(CUtensorMap* map, const void* ptr, int64_t m, int64_t n, int64_t ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(TSQR_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
  cuuint32_t box[2] = {16, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TSQR_ERR_CUDA, "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
  return TSQR_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// ---- n > 64: panels of 64 columns ---------------------------------------------------------
constexpr int64_t kPanel = 64;
constexpr int64_t kMaxN = 4096;  // 64 panels; wider matrices are not tall-skinny

struct PanelLayout {
  int count = 0;
  int64_t ldw = 0;              // leading dimension of the staged copy of A
  std::vector<size_t> off, bytes;  // each panel's own TSQR workspace
  size_t total = 0;
};

// Every panel is factored in place in the working copy of A (the staged copy, or A itself with
// inplace), with the caller's tree options.
tsqr_opts_t panel_opts(const tsqr_opts_t* o) {
  tsqr_opts_t s{};
  if (o) s = *o;
  s.inplace = 1;
  return s;
}

// FP32 storage: the working copy of A is float and every panel keeps its reflectors in its own
// workspace (the FP32 factorization widens its input into it).
tsqr_status_t make_panel_layout(int64_t m, int64_t n, const tsqr_opts_t* o, PanelLayout* L, bool f32 = false) {
  if (n > kMaxN) return fail(TSQR_ERR_UNSUPPORTED, "n > 4096 is not supported");
  if (o && o->r_only) return fail(TSQR_ERR_UNSUPPORTED, "r_only needs n <= 64 (the panels' updates need Q)");
  if (f32 && o && o->inplace) return fail(TSQR_ERR_UNSUPPORTED, "TSQR_F32 keeps A read-only (inplace is not supported)");
  const bool inplace = o && o->inplace;
  L->count = (int)((n + kPanel - 1) / kPanel);
  L->ldw = (n + 1) / 2 * 2;
  size_t off = inplace ? 0 : align256((size_t)m * L->ldw * (f32 ? 4 : 8));
  tsqr_opts_t so = panel_opts(o);
  if (f32) so.inplace = 0;
  for (int p = 0; p < L->count; ++p) {
    const int64_t c = p * kPanel, w = std::min(kPanel, n - c);
    Plan P;
    tsqr_status_t s = make_plan(m - c, w, &so, &P, f32);
    if (s != TSQR_OK) return fail(s, "panel " + std::to_string(p) + ": " + g_last_error);
    const size_t b = make_layout(P, !f32).total;
    L->off.push_back(off);
    L->bytes.push_back(b);
    off = align256(off + b);
  }
  L->total = off;
  return TSQR_OK;
}

// Blocked factorization: panel p is a TSQR of the updated columns c_p.. (rows c_p..m-1), whose
// Q^T then updates the trailing columns; the top w_p rows of that update are R's block row p.
tsqr_status_t factor_panels(tsqr_dtype_t dtype, int64_t m, int64_t n, const void* dA, int64_t lda, void* dR,
                            int64_t ldr, void* dWork, size_t work_bytes, const tsqr_opts_t* opts, tsqr_stream_t stream,
                            tsqr_handle_t* out) {
  const bool f32 = dtype == TSQR_F32;
  const size_t es = f32 ? 4 : 8;  // element size of A, R and the working copy
  PanelLayout L;
  tsqr_status_t s = make_panel_layout(m, n, opts, &L, f32);
  if (s != TSQR_OK) return s;
  const bool inplace = opts && opts->inplace;
  if (inplace && (lda % 2 != 0 || !aligned16(dA)))
    return fail(TSQR_ERR_INVALID_ARG, "inplace needs an even lda and a 16-byte aligned A");
  if (!dWork || work_bytes < L.total)
    return fail(TSQR_ERR_WORKSPACE, "workspace needs " + std::to_string(L.total) + " bytes");
  if ((reinterpret_cast<uintptr_t>(dWork) & 255) != 0) return fail(TSQR_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  char* w = static_cast<char*>(dWork);
  char* Aw = inplace ? static_cast<char*>(const_cast<void*>(dA)) : w;
  const int64_t ldw = inplace ? lda : L.ldw;
  char* R = static_cast<char*>(dR);
  auto at = [es](char* base, int64_t ld, int64_t r, int64_t c) { return base + (r * ld + c) * (int64_t)es; };
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (!inplace) {
    if (f32)
      e = cudaMemcpy2DAsync(Aw, (size_t)ldw * 4, dA, (size_t)lda * 4, (size_t)n * 4, (size_t)m, cudaMemcpyDeviceToDevice, cs);
    else
      e = tsqr::launch_stage_copy(static_cast<const double*>(dA), lda, reinterpret_cast<double*>(Aw), ldw, m, (int)n, cs);
    if (e != cudaSuccess) return cuda_fail(e, "staging copy");
  }
  if ((e = cudaMemset2DAsync(R, (size_t)ldr * es, 0, (size_t)n * es, (size_t)n, cs)) != cudaSuccess)
    return cuda_fail(e, "cudaMemset2DAsync");
  tsqr_handle_s* h = new (std::nothrow) tsqr_handle_s;
  if (!h) return fail(TSQR_ERR_INVALID_ARG, "out of host memory");
  h->m = m;
  h->n = n;
  h->inplace = inplace ? 1 : 0;
  h->f32 = f32 ? 1 : 0;
  tsqr_opts_t so = panel_opts(opts);
  if (f32) so.inplace = 0;
  for (int p = 0; p < L.count; ++p) {
    const int64_t c = p * kPanel, wp = std::min(kPanel, n - c), rest = n - c - wp;
    tsqr_handle_t hp = nullptr;
    s = tsqr_factor(dtype, TSQR_ROW_MAJOR, m - c, wp, at(Aw, ldw, c, c), ldw, at(R, ldr, c, c), ldr, w + L.off[p],
                    L.bytes[p], &so, stream, &hp);
    if (s == TSQR_OK) h->panels.push_back(hp);
    if (s == TSQR_OK && rest > 0) {
      char* trail = at(Aw, ldw, c, c + wp);
      s = tsqr_apply_qt(hp, rest, trail, ldw, stream);
      if (s == TSQR_OK &&
          (e = cudaMemcpy2DAsync(at(R, ldr, c, c + wp), (size_t)ldr * es, trail, (size_t)ldw * es, (size_t)rest * es,
                                 (size_t)wp, cudaMemcpyDeviceToDevice, cs)) != cudaSuccess)
        s = cuda_fail(e, "cudaMemcpy2DAsync");
    }
    if (s != TSQR_OK) {
      delete h;
      return s;
    }
  }
  *out = h;
  return TSQR_OK;
}

}  // namespace

extern "C" {

const char* tsqr_status_string(tsqr_status_t s) {
  switch (s) {
    case TSQR_OK: return "TSQR_OK";
    case TSQR_ERR_INVALID_ARG: return "TSQR_ERR_INVALID_ARG";
    case TSQR_ERR_UNSUPPORTED: return "TSQR_ERR_UNSUPPORTED";
    case TSQR_ERR_CUDA: return "TSQR_ERR_CUDA";
    case TSQR_ERR_WORKSPACE: return "TSQR_ERR_WORKSPACE";
    case TSQR_ERR_TIMEOUT: return "TSQR_ERR_TIMEOUT";
  }
  return "TSQR_UNKNOWN_STATUS";
}

const char* tsqr_last_error(void) { return g_last_error.c_str(); }

tsqr_status_t tsqr_workspace_size(tsqr_dtype_t dtype, int64_t m, int64_t n, const tsqr_opts_t* opts, size_t* bytes) {
  if (!bytes) return fail(TSQR_ERR_INVALID_ARG, "bytes is NULL");
  if (dtype != TSQR_F64 && dtype != TSQR_F32) return fail(TSQR_ERR_INVALID_ARG, "unknown dtype");
  const bool f32 = dtype == TSQR_F32;
  if (n > kPanel && m >= n) {
    PanelLayout L;
    tsqr_status_t s = make_panel_layout(m, n, opts, &L, f32);
    if (s != TSQR_OK) return s;
    *bytes = L.total;
    return TSQR_OK;
  }
  Plan P;
  tsqr_status_t s = make_plan(m, n, opts, &P, f32);
  if (s != TSQR_OK) return s;
  *bytes = make_layout(P, opts && opts->inplace).total;
  return TSQR_OK;
}

tsqr_status_t tsqr_factor(tsqr_dtype_t dtype, tsqr_layout_t layout, int64_t m, int64_t n, void* dA, int64_t lda,
                          void* dR, int64_t ldr, void* dWork, size_t work_bytes, const tsqr_opts_t* opts,
                          tsqr_stream_t stream, tsqr_handle_t* out) {
  if (!out) return fail(TSQR_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (dtype != TSQR_F64 && dtype != TSQR_F32) return fail(TSQR_ERR_INVALID_ARG, "unknown dtype");
  const bool f32 = dtype == TSQR_F32;
  if (layout != TSQR_ROW_MAJOR && layout != TSQR_COL_MAJOR) return fail(TSQR_ERR_INVALID_ARG, "unknown layout");
  const bool col = layout == TSQR_COL_MAJOR;
  if (!dA || !dR) return fail(TSQR_ERR_INVALID_ARG, "A and R must be non-NULL");
  if (n < 1 || m < n) return fail(TSQR_ERR_INVALID_ARG, "need m >= n >= 1");
  if (lda < (col ? m : n)) return fail(TSQR_ERR_INVALID_ARG, col ? "lda must be >= m (column-major)" : "lda must be >= n");
  if (ldr < n) return fail(TSQR_ERR_INVALID_ARG, "ldr must be >= n");
  if (col && n > kPanel) return fail(TSQR_ERR_UNSUPPORTED, "TSQR_COL_MAJOR needs n <= 64");
  if (col && opts && opts->inplace)
    return fail(TSQR_ERR_INVALID_ARG, "inplace needs a row-major A (the reflectors are stored row-major)");
  const uintptr_t amask = f32 ? 3 : 7;
  if ((reinterpret_cast<uintptr_t>(dA) & amask) != 0 || (reinterpret_cast<uintptr_t>(dR) & amask) != 0)
    return fail(TSQR_ERR_INVALID_ARG, f32 ? "A and R must be 4-byte aligned" : "A and R must be 8-byte aligned");
  if (n > kPanel) return factor_panels(dtype, m, n, dA, lda, dR, ldr, dWork, work_bytes, opts, stream, out);
  Plan P;
  tsqr_status_t s = make_plan(m, n, opts, &P, f32);
  if (s != TSQR_OK) return s;
  P.col_major = col ? 1 : 0;
  const bool inplace = opts && opts->inplace;
  // TMA needs a 16-byte aligned base and a row stride that is a multiple of 16 bytes; any other A
  // is first copied into the reflector storage of the workspace (which then holds V as usual).
  // FP32 input is always widened into it, column-major input transposed into it.
  const bool stage = col || f32 || (lda % 2 != 0) || !aligned16(dA);
  if (stage && inplace)
    return fail(TSQR_ERR_INVALID_ARG, "inplace needs an even lda and a 16-byte aligned A");
  const Layout L = make_layout(P, inplace);
  if (!dWork || work_bytes < L.total)
    return fail(TSQR_ERR_WORKSPACE, "workspace needs " + std::to_string(L.total) + " bytes");
  if ((reinterpret_cast<uintptr_t>(dWork) & 255) != 0) return fail(TSQR_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  char* w = static_cast<char*>(dWork);
  Store st;
  st.v = inplace ? static_cast<double*>(dA) : reinterpret_cast<double*>(w + L.v);
  st.ldv = inplace ? lda : L.ldv;
  st.tau_leaf = reinterpret_cast<double*>(w + L.tau_leaf);
  st.t_leaf = reinterpret_cast<double*>(w + L.t_leaf);
  st.node_r = reinterpret_cast<double*>(w + L.node_r);
  st.node_y = reinterpret_cast<double*>(w + L.node_y);
  st.node_tau = reinterpret_cast<double*>(w + L.node_tau);
  st.node_t = reinterpret_cast<double*>(w + L.node_t);
  st.signs = reinterpret_cast<double*>(w + L.signs);
  st.counters = reinterpret_cast<int*>(w + L.counters);
  st.status = reinterpret_cast<int*>(w + L.status);
  const int box_rows = P.h < 256 ? P.h : 256;
  CUtensorMap mapA, mapV;
  if ((s = make_map(&mapV, st.v, m, n, st.ldv, box_rows)) != TSQR_OK) return s;
  if (stage) {
    mapA = mapV;
  } else if ((s = make_map(&mapA, dA, m, n, lda, box_rows)) != TSQR_OK) {
    return s;
  }
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(st.status, 0, sizeof(int), cs);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  if (stage) {
    e = col   ? tsqr::launch_stage_transpose(dA, f32, lda, st.v, st.ldv, m, (int)n, cs)
        : f32 ? tsqr::launch_stage_widen(static_cast<const float*>(dA), lda, st.v, st.ldv, m, (int)n, cs)
              : tsqr::launch_stage_copy(static_cast<const double*>(dA), lda, st.v, st.ldv, m, (int)n, cs);
    if (e != cudaSuccess) return cuda_fail(e, "staging copy launch");
  }
  e = tsqr::launch_factor(mapA, mapV, P, st, dR, ldr, box_rows, cs);
  if (e != cudaSuccess) return cuda_fail(e, "factor launch");
  tsqr_handle_s* h = new (std::nothrow) tsqr_handle_s;
  if (!h) return fail(TSQR_ERR_INVALID_ARG, "out of host memory");
  h->P = P;
  h->st = st;
  h->mapV = mapV;
  h->box_rows = box_rows;
  h->inplace = inplace ? 1 : 0;
  h->f32 = f32 ? 1 : 0;
  h->m = m;
  h->n = n;
  *out = h;
  return TSQR_OK;
}

tsqr_status_t tsqr_form_q(tsqr_handle_t h, void* dQ, int64_t ldq, tsqr_stream_t stream) {
  if (!h) return fail(TSQR_ERR_INVALID_ARG, "handle is NULL");
  if (!h->panels.empty()) {
    // Q [I_n; 0], column block p: [0; thin Q_p] (rows c_p.. are untouched by the later panels'
    // factors), then the earlier panels' factors applied innermost first.
    if (!dQ || ldq < h->n) return fail(TSQR_ERR_INVALID_ARG, "Q must be non-NULL with ldq >= n");
    char* Q = static_cast<char*>(dQ);
    const int64_t es = h->f32 ? 4 : 8;
    const int count = (int)h->panels.size();
    for (int p = 0; p < count; ++p) {
      const int64_t c = p * kPanel, wp = std::min(kPanel, h->n - c);
      cudaError_t e;
      if (c > 0 && (e = cudaMemset2DAsync(Q + c * es, (size_t)(ldq * es), 0, (size_t)(wp * es), (size_t)c,
                                          static_cast<cudaStream_t>(stream))) != cudaSuccess)
        return cuda_fail(e, "cudaMemset2DAsync");
      tsqr_status_t s = tsqr_form_q(h->panels[p], Q + (c * ldq + c) * es, ldq, stream);
      if (s != TSQR_OK) return s;
    }
    for (int p = count - 2; p >= 0; --p) {
      const int64_t c = p * kPanel;
      tsqr_status_t s = tsqr_apply_q(h->panels[p], h->n - c - kPanel, Q + (c * ldq + c + kPanel) * es, ldq, stream);
      if (s != TSQR_OK) return s;
    }
    return TSQR_OK;
  }
  if (!dQ || ldq < (h->P.col_major ? h->P.m : h->P.n))
    return fail(TSQR_ERR_INVALID_ARG, "Q must be non-NULL with ldq >= n (row-major) or >= m (column-major)");
  if (h->P.r_only) return fail(TSQR_ERR_INVALID_ARG, "the factorization computed R alone (r_only): no Q");
  cudaError_t e = tsqr::launch_form_q(h->mapV, h->P, h->st, dQ, ldq, h->box_rows,
                                      static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "form_q launch");
  return TSQR_OK;
}

tsqr_status_t tsqr_apply_qt(tsqr_handle_t h, int64_t k, void* dB, int64_t ldb, tsqr_stream_t stream) {
  if (!h) return fail(TSQR_ERR_INVALID_ARG, "handle is NULL");
  if (k < 0) return fail(TSQR_ERR_INVALID_ARG, "k must be >= 0");
  if (k == 0) return TSQR_OK;
  if (!dB || ldb < k) return fail(TSQR_ERR_INVALID_ARG, "B must be non-NULL with ldb >= k");
  if (h->panels.empty() && h->P.col_major && ldb < h->P.m)
    return fail(TSQR_ERR_INVALID_ARG, "column-major B needs ldb >= m");
  if (!h->panels.empty()) {  // Q^T = ... diag(I, Q_1^T) Q_0^T: panel p acts on rows c_p..
    char* B = static_cast<char*>(dB);
    const int64_t es = h->f32 ? 4 : 8;
    for (size_t p = 0; p < h->panels.size(); ++p) {
      tsqr_status_t s = tsqr_apply_qt(h->panels[p], k, B + (int64_t)p * kPanel * ldb * es, ldb, stream);
      if (s != TSQR_OK) return s;
    }
    return TSQR_OK;
  }
  if (h->P.r_only) return fail(TSQR_ERR_INVALID_ARG, "the factorization computed R alone (r_only): no Q");
  cudaError_t e = tsqr::launch_apply_qt(h->mapV, h->P, h->st, k, dB, ldb, h->box_rows,
                                        static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "apply_qt launch");
  return TSQR_OK;
}

tsqr_status_t tsqr_apply_q(tsqr_handle_t h, int64_t k, void* dB, int64_t ldb, tsqr_stream_t stream) {
  if (!h) return fail(TSQR_ERR_INVALID_ARG, "handle is NULL");
  if (k < 0) return fail(TSQR_ERR_INVALID_ARG, "k must be >= 0");
  if (k == 0) return TSQR_OK;
  if (!dB || ldb < k) return fail(TSQR_ERR_INVALID_ARG, "B must be non-NULL with ldb >= k");
  if (h->panels.empty() && h->P.col_major && ldb < h->P.m)
    return fail(TSQR_ERR_INVALID_ARG, "column-major B needs ldb >= m");
  if (!h->panels.empty()) {  // Q = Q_0 diag(I, Q_1) ...: the last panel first
    char* B = static_cast<char*>(dB);
    const int64_t es = h->f32 ? 4 : 8;
    for (size_t p = h->panels.size(); p-- > 0;) {
      tsqr_status_t s = tsqr_apply_q(h->panels[p], k, B + (int64_t)p * kPanel * ldb * es, ldb, stream);
      if (s != TSQR_OK) return s;
    }
    return TSQR_OK;
  }
  if (h->P.r_only) return fail(TSQR_ERR_INVALID_ARG, "the factorization computed R alone (r_only): no Q");
  cudaError_t e = tsqr::launch_apply_q(h->mapV, h->P, h->st, k, dB, ldb, h->box_rows,
                                       static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "apply_q launch");
  return TSQR_OK;
}

tsqr_status_t tsqr_status_poll(tsqr_handle_t h, tsqr_stream_t stream) {
  if (!h) return fail(TSQR_ERR_INVALID_ARG, "handle is NULL");
  if (!h->panels.empty()) {
    for (tsqr_handle_s* p : h->panels) {
      tsqr_status_t s = tsqr_status_poll(p, stream);
      if (s != TSQR_OK) return s;
    }
    return TSQR_OK;
  }
  int v = 0;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&v, h->st.status, sizeof(int), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (v & tsqr::kStatusTimeout) return fail(TSQR_ERR_TIMEOUT, "a device-side bounded wait timed out");
  return TSQR_OK;
}

tsqr_status_t tsqr_handle_info(tsqr_handle_t h, tsqr_info_t* info) {
  if (!h || !info) return fail(TSQR_ERR_INVALID_ARG, "NULL argument");
  if (!h->panels.empty()) {  // the first panel's tree, with the whole matrix's shape
    tsqr_status_t s = tsqr_handle_info(h->panels[0], info);
    info->m = h->m;
    info->n = h->n;
    info->panels = (int32_t)h->panels.size();
    return s;
  }
  info->panels = 1;
  info->dtype = h->f32 ? TSQR_F32 : TSQR_F64;
  info->layout = h->P.col_major ? TSQR_COL_MAJOR : TSQR_ROW_MAJOR;
  const Plan& P = h->P;
  info->m = P.m;
  info->n = P.n;
  info->np = P.np;
  info->leaf_h = P.h;
  info->chain = P.chain;
  info->arity = P.arity;
  info->depth = P.depth;
  info->leaves = P.leaves;
  info->chains = P.chains;
  info->tree_nodes = P.tree_nodes;
  info->v = h->st.v;
  info->ldv = h->st.ldv;
  info->tau_leaf = h->st.tau_leaf;
  info->t_leaf = h->st.t_leaf;
  info->node_y = h->st.node_y;
  info->node_tau = h->st.node_tau;
  info->node_t = h->st.node_t;
  info->status = h->st.status;
  info->signs = h->st.signs;
  return TSQR_OK;
}

tsqr_status_t tsqr_destroy(tsqr_handle_t h) {
  delete h;
  return TSQR_OK;
}

}  // extern "C"


// ---------------------------------------------------------------------------------------------
// Batches: many independent factorizations in one launch (plans, workspace layout, descriptors).
namespace {

struct BatchPlan {
  std::vector<Plan> plans;
  std::vector<Layout> layouts;
  std::vector<size_t> item_off;
  size_t items_off = 0, chain_work_off = 0, formq_work_off = 0, level_work_off = 0, counters_off = 0, status_off = 0,
         total = 0;
  int requested_precision = 0;  // before the Ozaki forms map to their factorization's arithmetic
  int total_chains = 0, max_depth = 0, level_items = 0;
  size_t counters_bytes = 0;
};

// Plans of a batch.  item_opts (count entries, or NULL for opts everywhere) lets every matrix
// take its own leaf height, arity and chain length (an autotuner's choice per shape); the
// precision must be the same for all.  An entry with chain = 0 takes the batch's shared chain
// length.
tsqr_status_t make_batch_plan(int32_t count, const int64_t* m, const int64_t* n, const tsqr_opts_t* opts,
                              const tsqr_opts_t* item_opts, BatchPlan* bp, bool f32 = false) {
  if (count < 1) return fail(TSQR_ERR_INVALID_ARG, "count must be >= 1");
  if (!m || !n) return fail(TSQR_ERR_INVALID_ARG, "m and n arrays must be non-NULL");
  std::vector<tsqr_opts_t> io(count);
  for (int i = 0; i < count; ++i) {
    tsqr_opts_t o{};
    if (item_opts) o = item_opts[i];
    else if (opts) o = *opts;
    if (o.inplace) return fail(TSQR_ERR_UNSUPPORTED, "batches keep A read-only (inplace is not supported)");
    if (o.r_only) return fail(TSQR_ERR_UNSUPPORTED, "batches keep Q (r_only is not supported)");
    if (i == 0) bp->requested_precision = o.precision;
    // the batched factorization runs the Ozaki forms in their factorization's arithmetic; their
    // thin Q keeps the tensor-core products (items of padded width 64, leaf height <= 128)
    if (o.precision == tsqr::kPrecOzaki) o.precision = tsqr::kPrecF64;
    if (o.precision == tsqr::kPrecDFOzaki) o.precision = tsqr::kPrecDF;
    if (f32 && o.precision != 0)
      return fail(TSQR_ERR_UNSUPPORTED, "TSQR_F32 runs FP32 arithmetic: precision must be 0");
    if (i > 0 && o.precision != io[0].precision)
      return fail(TSQR_ERR_UNSUPPORTED, "every matrix of a batch takes the same precision");
    io[i] = o;
  }
  // shared chain length: about 16 waves of two blocks per SM over the whole batch; double-float
  // keeps chains of at most 18 leaves (its orthogonality grows with chain length)
  int64_t total_leaves = 0;
  for (int i = 0; i < count; ++i) {
    tsqr_opts_t probe = io[i];
    probe.chain = 1;
    Plan P;
    tsqr_status_t s = make_plan(m[i], n[i], &probe, &P, f32);
    if (s != TSQR_OK) return fail(s, "batch item " + std::to_string(i) + ": " + g_last_error);
    total_leaves += P.leaves;
  }
  {
    const int64_t blocks = 16LL * 2 * device_sms();
    int64_t c = (total_leaves + blocks - 1) / blocks;
    if (c < 1) c = 1;
    if (tsqr::prec_df(io[0].precision) && c > 18) c = 18;
    for (int i = 0; i < count; ++i)
      if (io[i].chain == 0) io[i].chain = (int32_t)c;
  }
  bp->plans.resize(count);
  bp->layouts.resize(count);
  bp->item_off.resize(count);
  for (int i = 0; i < count; ++i) {
    tsqr_status_t s = make_plan(m[i], n[i], &io[i], &bp->plans[i], f32);
    if (s != TSQR_OK) return fail(s, "batch item " + std::to_string(i) + ": " + g_last_error);
    bp->layouts[i] = make_layout(bp->plans[i], false);
    bp->total_chains += bp->plans[i].chains;
    bp->max_depth = std::max(bp->max_depth, bp->plans[i].depth);
    bp->level_items += bp->plans[i].tree_nodes;
    bp->counters_bytes += sizeof(int) * (size_t)(bp->plans[i].tree_nodes > 0 ? bp->plans[i].tree_nodes : 1);
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  bp->status_off = take(256);  // status word, then the persistent factor launch's work counter
  bp->items_off = take(sizeof(tsqr::BatchItem) * (size_t)count);
  bp->chain_work_off = take(sizeof(tsqr::BatchWork) * (size_t)bp->total_chains);
  bp->formq_work_off = take(sizeof(tsqr::BatchWork) * (size_t)bp->total_chains);
  bp->level_work_off = take(sizeof(tsqr::BatchWork) * (size_t)(bp->level_items > 0 ? bp->level_items : 1));
  bp->counters_off = take(bp->counters_bytes);
  for (int i = 0; i < count; ++i) bp->item_off[i] = take(bp->layouts[i].total);
  bp->total = off;
  return TSQR_OK;
}

}  // namespace

extern "C" {

tsqr_status_t tsqr_batch_workspace_size_plans(tsqr_dtype_t dtype, int32_t count, const int64_t* m,
                                              const int64_t* n, const tsqr_opts_t* item_opts, size_t* bytes) {
  if (!bytes) return fail(TSQR_ERR_INVALID_ARG, "bytes is NULL");
  if (!item_opts) return fail(TSQR_ERR_INVALID_ARG, "item_opts is NULL");
  if (dtype != TSQR_F64 && dtype != TSQR_F32) return fail(TSQR_ERR_INVALID_ARG, "unknown dtype");
  BatchPlan bp;
  tsqr_status_t s = make_batch_plan(count, m, n, nullptr, item_opts, &bp, dtype == TSQR_F32);
  if (s != TSQR_OK) return s;
  *bytes = bp.total;
  return TSQR_OK;
}

tsqr_status_t tsqr_batch_workspace_size(tsqr_dtype_t dtype, int32_t count, const int64_t* m, const int64_t* n,
                                        const tsqr_opts_t* opts, size_t* bytes) {
  if (!bytes) return fail(TSQR_ERR_INVALID_ARG, "bytes is NULL");
  if (dtype != TSQR_F64 && dtype != TSQR_F32) return fail(TSQR_ERR_INVALID_ARG, "unknown dtype");
  BatchPlan bp;
  tsqr_status_t s = make_batch_plan(count, m, n, opts, nullptr, &bp, dtype == TSQR_F32);
  if (s != TSQR_OK) return s;
  *bytes = bp.total;
  return TSQR_OK;
}

static tsqr_status_t batch_create(tsqr_dtype_t dtype, int32_t count, const int64_t* m, const int64_t* n,
                                  void* const* dA, const int64_t* lda, void* const* dR, const int64_t* ldr,
                                  void* const* dQ, const int64_t* ldq, void* dWork, size_t work_bytes,
                                  const tsqr_opts_t* opts, const tsqr_opts_t* item_opts, tsqr_stream_t stream,
                                  tsqr_batch_t* out) {
  if (!out) return fail(TSQR_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (dtype != TSQR_F64 && dtype != TSQR_F32) return fail(TSQR_ERR_INVALID_ARG, "unknown dtype");
  const bool f32 = dtype == TSQR_F32;
  if (!dA || !lda || !dR || !ldr) return fail(TSQR_ERR_INVALID_ARG, "A, lda, R and ldr arrays must be non-NULL");
  if (dQ && !ldq) return fail(TSQR_ERR_INVALID_ARG, "ldq array must be given with Q");
  BatchPlan bp;
  tsqr_status_t s = make_batch_plan(count, m, n, opts, item_opts, &bp, f32);
  if (s != TSQR_OK) return s;
  if (!dWork || work_bytes < bp.total)
    return fail(TSQR_ERR_WORKSPACE, "batch workspace needs " + std::to_string(bp.total) + " bytes");
  if ((reinterpret_cast<uintptr_t>(dWork) & 255) != 0) return fail(TSQR_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  char* w = static_cast<char*>(dWork);
  tsqr_batch_s* b = new (std::nothrow) tsqr_batch_s;
  if (!b) return fail(TSQR_ERR_INVALID_ARG, "out of host memory");
  b->count = count;
  b->precision = bp.plans[0].precision;
  b->total_chains = bp.total_chains;
  b->max_depth = bp.max_depth;
  b->d_status = reinterpret_cast<int*>(w + bp.status_off);
  b->d_items = reinterpret_cast<tsqr::BatchItem*>(w + bp.items_off);
  b->d_chain_work = reinterpret_cast<tsqr::BatchWork*>(w + bp.chain_work_off);
  b->d_counters = reinterpret_cast<int*>(w + bp.counters_off);
  b->counters_bytes = bp.counters_bytes;
  b->has_q = dQ != nullptr;
  std::vector<tsqr::BatchItem> items(count);
  std::vector<tsqr::BatchWork> chain_work;
  chain_work.reserve(bp.total_chains);
  size_t counter_ints = 0;
  for (int i = 0; i < count; ++i) {
    const Plan& P = bp.plans[i];
    const Layout& L = bp.layouts[i];
    if (!dA[i] || !dR[i] || (dQ && !dQ[i])) {
      delete b;
      return fail(TSQR_ERR_INVALID_ARG, "batch item " + std::to_string(i) + ": NULL matrix pointer");
    }
    const uintptr_t amask = f32 ? 3 : 7;
    if (lda[i] < n[i] || ldr[i] < n[i] || (dQ && ldq[i] < n[i]) || (reinterpret_cast<uintptr_t>(dA[i]) & amask) != 0 ||
        (reinterpret_cast<uintptr_t>(dR[i]) & amask) != 0 || (dQ && (reinterpret_cast<uintptr_t>(dQ[i]) & amask) != 0)) {
      delete b;
      return fail(TSQR_ERR_INVALID_ARG, "batch item " + std::to_string(i) + ": bad leading dimension or alignment");
    }
    char* wi = w + bp.item_off[i];
    tsqr::BatchItem& it = items[i];
    std::memset(&it, 0, sizeof(it));
    it.plan = P;
    Store& st = it.store;
    st.v = reinterpret_cast<double*>(wi + L.v);
    st.ldv = L.ldv;
    st.tau_leaf = reinterpret_cast<double*>(wi + L.tau_leaf);
    st.t_leaf = reinterpret_cast<double*>(wi + L.t_leaf);
    st.node_r = reinterpret_cast<double*>(wi + L.node_r);
    st.node_y = reinterpret_cast<double*>(wi + L.node_y);
    st.node_tau = reinterpret_cast<double*>(wi + L.node_tau);
    st.node_t = reinterpret_cast<double*>(wi + L.node_t);
    st.signs = reinterpret_cast<double*>(wi + L.signs);
    st.counters = b->d_counters + counter_ints;
    counter_ints += (size_t)(P.tree_nodes > 0 ? P.tree_nodes : 1);
    st.status = b->d_status;
    it.R = dR[i];
    it.ldr = ldr[i];
    it.Q = dQ ? dQ[i] : nullptr;
    it.ldq = dQ ? ldq[i] : 0;
    it.box_rows = P.h < 256 ? P.h : 256;
    if (f32) {  // widened into V by one batched launch before each factorization
      it.A32 = static_cast<const float*>(dA[i]);
      it.lda32 = lda[i];
      b->widen = true;
    }
    const bool stage = !f32 && ((lda[i] % 2 != 0) || !aligned16(dA[i]));
    if ((s = make_map(&it.mapV, st.v, m[i], n[i], st.ldv, it.box_rows)) != TSQR_OK) {
      delete b;
      return s;
    }
    if (stage || f32) it.mapA = it.mapV;
    if (stage) {
      b->stages.push_back({static_cast<const double*>(dA[i]), lda[i], st.v, st.ldv, m[i], (int)n[i]});
    } else if (!f32 && (s = make_map(&it.mapA, dA[i], m[i], n[i], lda[i], it.box_rows)) != TSQR_OK) {
      delete b;
      return s;
    }
    b->smem_factor = std::max(b->smem_factor, tsqr::factor_smem_bytes(P));
    b->smem_formq = std::max(b->smem_formq, tsqr::formq_smem_bytes(P, true));  // the chain kernel double-buffers
    for (int g = 0; g < P.chains; ++g) chain_work.push_back({i, g, 0});
  }
  // longest chains first: the persistent factor launch takes work in this order, so the last
  // items to start are the shortest (longest-processing-time-first balancing)
  auto chain_cost = [&](const tsqr::BatchWork& w) {
    const Plan& P = bp.plans[w.item];
    const int64_t leaves = tsqr::chain_end_leaf(P, w.chain) - tsqr::chain_first_leaf(P, w.chain);
    return (double)leaves * P.h * P.n * P.n;
  };
  std::stable_sort(chain_work.begin(), chain_work.end(),
                   [&](const tsqr::BatchWork& a, const tsqr::BatchWork& c) { return chain_cost(a) > chain_cost(c); });
  // thin-Q chain lists: the tensor-core kernel takes the items of padded width 64 and leaf height
  // <= 128 when the batch asked for a tensor-core form (precision 2 or 3, or FP32 storage)
  b->tc = f32 ? 3 : (bp.requested_precision == tsqr::kPrecOzaki ? 1 : (bp.requested_precision == tsqr::kPrecDFOzaki ? 2 : 0));
  std::vector<tsqr::BatchWork> formq_list, tc_list;
  for (const tsqr::BatchWork& wk : chain_work) {
    const Plan& P = bp.plans[wk.item];
    if (b->tc && P.np == 64 && P.h <= 128)
      tc_list.push_back(wk);
    else
      formq_list.push_back(wk);
  }
  for (const tsqr::BatchWork& wk : tc_list) {
    const Plan& P = bp.plans[wk.item];
    b->smem_tc = std::max(b->smem_tc, b->tc == 3 ? tsqr::formq_bf16x3_smem_bytes(P) : tsqr::formq_ozaki_smem_bytes(P));
  }
  b->formq_blocks = (int)formq_list.size();
  b->tc_blocks = (int)tc_list.size();
  formq_list.insert(formq_list.end(), tc_list.begin(), tc_list.end());
  tsqr::BatchWork* d_formq = reinterpret_cast<tsqr::BatchWork*>(w + bp.formq_work_off);
  b->d_formq_work = d_formq;
  b->d_tc_work = d_formq + b->formq_blocks;
  // tree steps of the batched thin Q, by distance d from each item's root
  std::vector<std::vector<tsqr::BatchWork>> levels(bp.max_depth);
  for (int i = 0; i < count; ++i) {
    const Plan& P = bp.plans[i];
    for (int d = 0; d < P.depth; ++d) {
      const int level = P.depth - d;
      for (int node = 0; node < P.level_count[level]; ++node) levels[d].push_back({i, node, level});
    }
  }
  std::vector<tsqr::BatchWork> level_flat;
  std::vector<size_t> level_start;
  for (int d = 0; d < bp.max_depth; ++d) {
    level_start.push_back(level_flat.size());
    b->level_blocks.push_back((int)levels[d].size());
    level_flat.insert(level_flat.end(), levels[d].begin(), levels[d].end());
  }
  tsqr::BatchWork* d_levels = reinterpret_cast<tsqr::BatchWork*>(w + bp.level_work_off);
  for (int d = 0; d < bp.max_depth; ++d) b->d_level_work.push_back(d_levels + level_start[d]);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(tsqr::BatchItem) * count, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_chain_work, chain_work.data(), sizeof(tsqr::BatchWork) * chain_work.size(),
                        cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess && !level_flat.empty())
    e = cudaMemcpyAsync(d_levels, level_flat.data(), sizeof(tsqr::BatchWork) * level_flat.size(),
                        cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_formq, formq_list.data(), sizeof(tsqr::BatchWork) * formq_list.size(),
                        cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);  // the host arrays above are about to go away
  if (e == cudaSuccess) e = tsqr::prepare_factor_batched(b->precision, b->smem_factor);
  if (e == cudaSuccess) e = tsqr::factor_batched_blocks(b->precision, b->total_chains, b->smem_factor, &b->factor_blocks);
  if (e == cudaSuccess) e = tsqr::prepare_form_q_batched(b->precision, b->smem_formq);
  if (e == cudaSuccess && b->tc_blocks > 0)
    e = b->tc == 3 ? tsqr::prepare_formq_bf16x3_batched(b->smem_tc) : tsqr::prepare_formq_ozaki_batched(b->tc == 2, b->smem_tc);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "batch descriptor upload");
  }
  *out = b;
  return TSQR_OK;
}

tsqr_status_t tsqr_batch_create(tsqr_dtype_t dtype, int32_t count, const int64_t* m, const int64_t* n,
                                void* const* dA, const int64_t* lda, void* const* dR, const int64_t* ldr,
                                void* const* dQ, const int64_t* ldq, void* dWork, size_t work_bytes,
                                const tsqr_opts_t* opts, tsqr_stream_t stream, tsqr_batch_t* out) {
  return batch_create(dtype, count, m, n, dA, lda, dR, ldr, dQ, ldq, dWork, work_bytes, opts, nullptr, stream, out);
}

tsqr_status_t tsqr_batch_create_plans(tsqr_dtype_t dtype, int32_t count, const int64_t* m, const int64_t* n,
                                      void* const* dA, const int64_t* lda, void* const* dR, const int64_t* ldr,
                                      void* const* dQ, const int64_t* ldq, void* dWork, size_t work_bytes,
                                      const tsqr_opts_t* item_opts, tsqr_stream_t stream, tsqr_batch_t* out) {
  if (!item_opts) return fail(TSQR_ERR_INVALID_ARG, "item_opts is NULL");
  return batch_create(dtype, count, m, n, dA, lda, dR, ldr, dQ, ldq, dWork, work_bytes, nullptr, item_opts, stream,
                      out);
}

tsqr_status_t tsqr_batch_factor(tsqr_batch_t b, tsqr_stream_t stream) {
  if (!b) return fail(TSQR_ERR_INVALID_ARG, "batch is NULL");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  // the status word and the persistent launch's work counter (the next int) start at zero
  cudaError_t e = cudaMemsetAsync(b->d_status, 0, 2 * sizeof(int), cs);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counters, 0, b->counters_bytes, cs);
  for (size_t k = 0; e == cudaSuccess && k < b->stages.size(); ++k) {
    const auto& sg = b->stages[k];
    e = tsqr::launch_stage_copy(sg.A, sg.lda, sg.V, sg.ldv, sg.m, sg.n, cs);
  }
  if (e == cudaSuccess && b->widen) e = tsqr::launch_stage_widen_batched(b->d_items, b->count, cs);
  if (e == cudaSuccess)
    e = tsqr::launch_factor_batched(b->d_items, b->d_chain_work, b->total_chains, b->d_status + 1, b->factor_blocks,
                                    b->precision, b->smem_factor, cs);
  if (e != cudaSuccess) return cuda_fail(e, "batched factor launch");
  return TSQR_OK;
}

tsqr_status_t tsqr_batch_form_q(tsqr_batch_t b, tsqr_stream_t stream) {
  if (!b) return fail(TSQR_ERR_INVALID_ARG, "batch is NULL");
  if (!b->has_q) return fail(TSQR_ERR_INVALID_ARG, "the batch was created without Q outputs");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e = tsqr::launch_form_q_batched(b->d_items, b->d_formq_work, b->formq_blocks, b->d_level_work.data(),
                                              b->level_blocks.data(), b->max_depth, b->precision, b->smem_formq, cs);
  if (e == cudaSuccess && b->tc_blocks > 0)
    e = b->tc == 3 ? tsqr::launch_formq_bf16x3_batched(b->d_items, b->d_tc_work, b->tc_blocks, b->smem_tc, cs)
                   : tsqr::launch_formq_ozaki_batched(b->d_items, b->d_tc_work, b->tc_blocks, b->tc == 2, b->smem_tc, cs);
  if (e != cudaSuccess) return cuda_fail(e, "batched form_q launch");
  return TSQR_OK;
}

tsqr_status_t tsqr_batch_status_poll(tsqr_batch_t b, tsqr_stream_t stream) {
  if (!b) return fail(TSQR_ERR_INVALID_ARG, "batch is NULL");
  int v = 0;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&v, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (v & tsqr::kStatusTimeout) return fail(TSQR_ERR_TIMEOUT, "a device-side bounded wait timed out");
  return TSQR_OK;
}

tsqr_status_t tsqr_batch_destroy(tsqr_batch_t b) {
  delete b;
  return TSQR_OK;
}

}  // extern "C"

namespace tsqr {
tsqr_status_t internal_make_plan(int64_t m, int64_t n, const tsqr_opts_t* opts, Plan* P) {
  return make_plan(m, n, opts, P);
}
tsqr_status_t internal_make_map(CUtensorMap* map, const void* ptr, int64_t m, int64_t n, int64_t ld, int box_rows) {
  return make_map(map, ptr, m, n, ld, box_rows);
}
tsqr_status_t internal_fail(tsqr_status_t s, const char* msg) { return fail(s, msg); }
}  // namespace tsqr
