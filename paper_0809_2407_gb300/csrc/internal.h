// Host helpers of api.cu shared with other translation units of libtsqr.so (not public).
#pragma once

#include "../../include/tsqr.h"
#include "common.cuh"

namespace tsqr {

// Reduction-tree plan of an m x n factorization (the same one tsqr_factor uses).
tsqr_status_t internal_make_plan(int64_t m, int64_t n, const tsqr_opts_t* opts, Plan* P);
// TMA descriptor of a row-major m x n FP64 matrix (16-column x box_rows boxes, 128B swizzle).
tsqr_status_t internal_make_map(CUtensorMap* map, const void* ptr, int64_t m, int64_t n, int64_t ld, int box_rows);
// Records msg for tsqr_last_error() and returns s.
tsqr_status_t internal_fail(tsqr_status_t s, const char* msg);

}  // namespace tsqr
