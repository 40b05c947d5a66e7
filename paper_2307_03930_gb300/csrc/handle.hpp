// Packed-A handle shared by the pack, SpMM and API translation units.
#pragma once

#include <stdint.h>

#include <map>
#include <mutex>

#include "common.cuh"

namespace rosko {
constexpr uint64_t kHandleMagic = 0x524f534b4f474233ull;  // "ROSKOGB3"
constexpr int kNumFeatures = 16;
}  // namespace rosko

// Device layout of a packed A (Alg. 1 per row panel, panels in order):
//   panel_col[P+1]  first packed column of each panel (int32)
//   col_ind[n_cols] column index k of each packed column          (Alg. 1 col_ind)
//   col_start[n_cols+1] first nonzero of each packed column; the column's
//                   count is col_start[c+1] - col_start[c]         (Alg. 1 nnz)
//   vals[nnz]       nonzero values in column order, rows ascending (Alg. 1 A_p)
//   rows[nnz]       panel-relative row of each value (uint8)       (Alg. 1 loc_m)
//   row_scale[M]    INT8 only: per-row symmetric scale
struct rosko_packed_s {
  uint64_t magic = 0;
  int device = 0;
  int64_t M = 0, K = 0, P = 0;
  int32_t m_r = 0;
  rosko_dtype dt = ROSKO_F32;
  int64_t nnz = 0, n_cols = 0, touched_k = 0;
  void* meta_base = nullptr;  // panel_col, row_scale, features
  void* data_base = nullptr;  // col_ind, col_start, vals, rows
  int32_t* panel_col = nullptr;
  int32_t* col_ind = nullptr;
  int32_t* col_start = nullptr;
  void* vals = nullptr;
  uint8_t* rows = nullptr;
  float* row_scale = nullptr;
  float* feat_dev = nullptr;   // kNumFeatures floats (N-independent part)
  int64_t* panel_nnz_dev = nullptr;  // P+1 nonzero offsets of panels
  std::mutex mu;               // guards the schedule cache
  std::map<int64_t, rosko_tile> sched_cache;  // per N (and mode) chosen tiles
};

namespace rosko {
inline bool handle_ok(const rosko_packed_s* h) { return h && h->magic == kHandleMagic; }

// pack.cu
rosko_status pack_impl(const void* A, rosko_dtype a_dt, int64_t M, int64_t K, int64_t lda,
                       rosko_dtype p_dt, const float* row_scale_in, int32_t m_r,
                       cudaStream_t stream, rosko_packed_s** out);
rosko_status unpack_impl(rosko_packed_s* h, void* A_out, int64_t lda, cudaStream_t stream);

// spmm_sparse.cu
struct SparseLaunch {
  int R, V, W, KC, stages, split;
};
rosko_status sparse_spmm_launch(rosko_packed_s* h, const void* B, rosko_dtype b_dt, int64_t N,
                                int64_t ldb, const float* col_scale, void* C, rosko_dtype c_dt,
                                int64_t ldc, int accumulate, const SparseLaunch& L,
                                cudaStream_t stream);
bool sparse_config_supported(rosko_dtype p_dt, rosko_dtype b_dt, rosko_dtype c_dt, int R, int V);
int sparse_default_V(rosko_dtype p_dt, int R);
}  // namespace rosko
