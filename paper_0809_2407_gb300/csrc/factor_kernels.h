// Host-side launchers of the TSQR kernels (internal to libtsqr.so).
#pragma once

#include "common.cuh"

namespace tsqr {

size_t factor_smem_bytes(const Plan& P);
// allow_dbl: the double-buffered chain kernel's layout where it fits (formq_double_buffered)
size_t formq_smem_bytes(const Plan& P, bool allow_dbl = false);
size_t apply_smem_bytes(const Plan& P, int kb);
size_t formq_ozaki_smem_bytes(const Plan& P);
bool ozaki_form_q_applies(const Plan& P);
// Thin Q with Ozaki products in three kernels (formq_ozaki_phases.cu): the chain recurrences,
// the chains' first leaves, and the other leaves' products.  A chain that holds a short last leaf
// (fewer than n rows, merged into the last chain) is taken whole by the first-leaf kernel.
__host__ __device__ inline bool formq_chain_short(const Plan& P, int g) {
  return g == P.chains - 1 && P.m - (P.leaves - 1) * P.h < P.n;
}
// A leaf whose product -V M runs in formq_ozaki_leaves_kernel: not the first of its chain, and
// not in a chain taken whole.
__host__ __device__ inline bool formq_leaf_deferred(const Plan& P, int64_t leaf) {
  const int64_t g = leaf / P.chain < P.chains ? leaf / P.chain : P.chains - 1;
  return leaf != chain_first_leaf(P, (int)g) && !formq_chain_short(P, (int)g);
}
// The recurrences: M = T C of every leaf but the first into that leaf's first n rows of Q, and
// the block entering the first leaf into node_r[g] as plain FP64.
cudaError_t launch_formq_ozaki_recur(const Plan& P, const Store& st, double* Q, int64_t ldq, cudaStream_t stream);
// The products -V M of the deferred leaves, over the M that the recurrences left in Q.
cudaError_t launch_formq_ozaki_leaves(const Plan& P, const Store& st, double* Q, int64_t ldq, cudaStream_t stream);
// Q^T B / Q B with the chains' WY products on the tensor cores (Ozaki splits in precision modes 2
// and 3, bf16x3 terms in FP32 storage): np = 64, h <= 128, and at least this many columns of B
// (narrower B stays on the FP64 / FP32 pipe)
constexpr int64_t kTcApplyMinCols = 32;
bool ozaki_apply_applies(const Plan& P, int64_t k);
// the chain part only (Q^T: before the tree levels; Q: after them); B is double*
cudaError_t launch_apply_ozaki_chains(const CUtensorMap& mapV, const Plan& P, const Store& st, int64_t k, double* B,
                                      int64_t ldb, int box_rows, bool trans, cudaStream_t stream);
size_t formq_bf16x3_smem_bytes(const Plan& P);
bool bf16x3_apply_applies(const Plan& P, int64_t k);
cudaError_t launch_apply_bf16x3_chains(const CUtensorMap& mapV, const Plan& P, const Store& st, int64_t k, float* B,
                                       int64_t ldb, int box_rows, bool trans, cudaStream_t stream);
bool bf16x3_form_q_applies(const Plan& P);
// FP32 storage, as the Ozaki thin Q above (formq_f32_phases.cu): the chains' recurrences M = T C
// on the FP32 pipe (M into each later leaf's rows of Q, the block entering the first leaf into
// node_r), and the other leaves' products -Y M as bf16x3 terms on the tensor cores.
cudaError_t launch_formq_f32_recur(const Plan& P, const Store& st, float* Q, int64_t ldq, cudaStream_t stream);
cudaError_t launch_formq_bf16x3_leaves(const Plan& P, const Store& st, float* Q, int64_t ldq, cudaStream_t stream);
// chains of an FP32-storage thin Q with bf16x3 tensor-core WY products (after the tree levels)
cudaError_t launch_formq_bf16x3_chains(const CUtensorMap& mapV, const Plan& P, const Store& st, float* Q, int64_t ldq,
                                       int box_rows, cudaStream_t stream);

cudaError_t launch_stage_copy(const double* A, int64_t lda, double* V, int64_t ldv, int64_t m, int n,
                              cudaStream_t stream);
cudaError_t launch_stage_widen(const float* A, int64_t lda, double* V, int64_t ldv, int64_t m, int n,
                               cudaStream_t stream);
cudaError_t launch_stage_transpose(const void* A, bool f32, int64_t lda, double* V, int64_t ldv, int64_t m, int n,
                                   cudaStream_t stream);
// Precision mode 2 (Ozaki products) or FP32 storage (bf16x3 products) at np = 64, h = 64, binary
// tree: the blocked flat-tree step whose WY products run on the tensor cores (factor_blocked.cu)
// in place of the FP64- or FP32-pipe step.  R_out is double*, or float* for FP32 storage.
bool blocked_factor_applies(const Plan& P);
cudaError_t launch_factor_blocked(const CUtensorMap& mapA, const CUtensorMap& mapV, const Plan& P, const Store& st,
                                  void* R_out, int64_t ldr, int box_rows, cudaStream_t stream);
// R_out, Q and B are double*, or float* when P.precision == 3 (FP32 storage)
cudaError_t launch_factor(const CUtensorMap& mapA, const CUtensorMap& mapV, const Plan& P, const Store& st,
                          void* R_out, int64_t ldr, int box_rows, cudaStream_t stream);
cudaError_t prepare_factor_batched(int precision, size_t smem);
cudaError_t launch_stage_widen_batched(const BatchItem* items, int count, cudaStream_t stream);
cudaError_t prepare_form_q_batched(int precision, size_t smem);
// the persistent batched factorization: `blocks` resident blocks (factor_batched_blocks: as many
// as fit on the device at `smem`, at most `total`) take the `total` chains in `work` through the
// counter *next (zero before the launch)
cudaError_t factor_batched_blocks(int precision, int total, size_t smem, int* blocks);
cudaError_t launch_factor_batched(const BatchItem* items, const BatchWork* work, int total, int* next, int blocks,
                                  int precision, size_t smem, cudaStream_t stream);
cudaError_t launch_form_q_batched(const BatchItem* items, const BatchWork* chain_work, int chain_blocks,
                                  const BatchWork* const* level_work, const int* level_blocks, int depth,
                                  int precision, size_t smem, cudaStream_t stream);
// Batched thin Q with the chains' WY products on the tensor cores, for the items of padded width
// 64 and leaf height <= 128: Ozaki splits (FP64 storage; pairs: double-float slots) or bf16x3 terms
// (FP32 storage); one block per chain in `work` (after the FP64- or FP32-pipe tree levels).
cudaError_t prepare_formq_ozaki_batched(bool pairs, size_t smem);
cudaError_t launch_formq_ozaki_batched(const BatchItem* items, const BatchWork* work, int blocks, bool pairs,
                                       size_t smem, cudaStream_t stream);
cudaError_t prepare_formq_bf16x3_batched(size_t smem);
cudaError_t launch_formq_bf16x3_batched(const BatchItem* items, const BatchWork* work, int blocks, size_t smem,
                                        cudaStream_t stream);
cudaError_t launch_form_q(const CUtensorMap& mapV, const Plan& P, const Store& st, void* Q, int64_t ldq,
                          int box_rows, cudaStream_t stream);
cudaError_t launch_apply_qt(const CUtensorMap& mapV, const Plan& P, const Store& st, int64_t k, void* B,
                            int64_t ldb, int box_rows, cudaStream_t stream);
cudaError_t launch_apply_q(const CUtensorMap& mapV, const Plan& P, const Store& st, int64_t k, void* B,
                           int64_t ldb, int box_rows, cudaStream_t stream);

}  // namespace tsqr
