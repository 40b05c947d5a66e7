// Packed-A handle shared by the pack, SpMM and API translation units.
#pragma once

#include <algorithm>

#include <stdint.h>

#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace rosko {
constexpr uint64_t kHandleMagic = 0x524f534b4f474233ull;  // "ROSKOGB3"
constexpr int kNumFeatures = 16;
}  // namespace rosko

// Device layout of a packed A (Alg. 1 per row panel, panels in order):
//   panel_col[P+1]   first packed column of each panel (int32)
//   colrec[n_cols+1] int2 {k, start}: the column index of each packed column
//                    (Alg. 1 col_ind) and the index of its first nonzero; the
//                    column's count (Alg. 1 nnz) is colrec[c+1].start -
//                    colrec[c].start; colrec[n_cols] = {INT32_MAX, nnz}
//   nz[nnz]          one record per nonzero, in column order with rows
//                    ascending: the value (Alg. 1 A_p) and its panel-relative
//                    row (Alg. 1 loc_m) interleaved, so one load serves both:
//                      BF16, INT8: uint32 = value bits << 16 | row
//                      FP32: uint2 {row, value bits}; FP64: {double, row, pad}
//   row_scale[M]     INT8 only: per-row symmetric scale
// Row-slot execution stream (a second order of the same nonzeros, for the
// row-slot SpMM traversal; built when K < 65280):
//   rowptr[M+1]      first record of each row (rows in panel order)
//   rnz[...]         per row, its nonzeros with k ascending, then one sentinel
//                    record whose k (0xFFFF / INT32_MAX) ends the row:
//                      BF16, INT8: uint32 = value bits << 16 | k
//                      FP32: uint2 {k, value bits}; FP64: {double, k, pad}
// Row-direct work segments: a row longer than twice the mean row length (and
// than kSegRecords) is cut into pieces of that length whose sums are added
// into C atomically, so that power-law rows do not serialise on one warp
// while rows of an even matrix stay whole.
constexpr int kSegRecords = 64;
// One work segment: {row, first record, end record, cut} and, inline, the
// first 48 bytes of the piece's records (12 BF16 / INT8 records, 6 FP32,
// 3 FP64), so that a warp whose piece fits starts its B loads one dependent
// load earlier.  64 bytes: two sectors, one coalesced load of 16 lanes.
struct SegEntry {
  int4 head;
  uint32_t rec[12];
};
static_assert(sizeof(SegEntry) == 64, "a segment entry is 64 bytes");
inline int64_t seg_records_for(int64_t nnz, int64_t M) {
  const int64_t twice_mean = M > 0 ? (2 * nnz + M - 1) / M : 0;
  return std::max<int64_t>(kSegRecords, (twice_mean + 31) / 32 * 32);
}

struct rosko_packed_s {
  uint64_t magic = 0;
  int device = 0;
  int64_t M = 0, K = 0, P = 0;
  int32_t m_r = 0;
  rosko_dtype dt = ROSKO_F32;
  int64_t nnz = 0, n_cols = 0, touched_k = 0;
  void* base = nullptr;  // one device allocation holding every array below
  size_t base_bytes = 0;  // its size
  int32_t* panel_col = nullptr;
  int2* colrec = nullptr;
  void* nz = nullptr;
  float* row_scale = nullptr;
  int32_t* rowptr = nullptr;
  void* rnz = nullptr;
  // Touched-row gather stream (m_r = 16): per 128-row tile t the distinct
  // columns its rows touch (the tile's Alg. 1 col_ind), gu_k[gu_start[t] ..
  // gu_start[t+1]), and per row the records (value, slot) where slot is the
  // position of k in the tile's list (same rowptr as rnz).
  int32_t* gu_start = nullptr;
  int32_t* gu_k = nullptr;
  void* gnz = nullptr;
  int64_t gu_total = 0;
  // Row-direct work segments (row stream only), at two granularities: list
  // 0 cuts every row into pieces of at most kSegRecords nonzeros (many
  // warps for few or long rows), list 1 only rows longer than
  // seg_records_for (twice the mean; few atomics for even matrices).  Per
  // list: one SegEntry per segment (head = the record range of the piece in
  // the row stream, sentinel excluded, and cut = 1 when the row has several
  // pieces; then the piece's first records) in row order (nat) and in
  // panel_order order (ord, packs with dense copies); prefix[i] / split[i]
  // count the segments / the panels with a cut row among the first i panels
  // of panel_order (or of the natural order without one).
  // lpt: every segment of the list, longest piece first (ties in row
  // order) - the order of a launch that runs all panels sparse, so that the
  // longest pieces start first and the 8 items of a block have similar
  // lengths (an inspector-executor ordering of the work, fixed at pack time).
  struct SegList {
    SegEntry* nat = nullptr;
    SegEntry* ord = nullptr;
    SegEntry* lpt = nullptr;
    std::vector<int64_t> prefix;
    std::vector<int32_t> split;
    int32_t records = kSegRecords;
  };
  SegList segs[2];
  float* feat_dev = nullptr;   // kNumFeatures floats (N-independent part)
  int64_t* panel_nnz_dev = nullptr;  // P+1 nonzero offsets of panels
  // Dense-panel split (BF16 only).  128-row tiles sorted by density,
  // descending; the first n_copy of them have a dense BF16 copy in dense_A
  // (row block c holds tile tile_order[c]).  panel_order lists the panels of
  // the tiles in the reverse order (ascending density), so for any threshold
  // the sparse panels are a prefix of it.
  int64_t n_tiles = 0, n_copy = 0, Kpad = 0;
  void* dense_A = nullptr;
  int32_t* tile_order_dev = nullptr;
  int32_t* panel_order_dev = nullptr;
  std::vector<int32_t> tile_order;        // host copy
  std::vector<int32_t> panel_order_host;  // host copy of panel_order
  std::vector<double> tile_density;       // sorted, descending
  std::vector<int32_t> tile_panels;       // panels per tile (indexed by tile id)
  std::vector<int64_t> panel_nnz;         // host copy, P+1 offsets
  std::mutex mu;               // guards the schedule cache
  std::map<int64_t, rosko_tile> sched_cache;  // per N (and mode) chosen tiles
};

namespace rosko {
struct RecF64 {
  double a;
  int32_t r;
  int32_t pad;
};
// bytes of one nonzero record for a packed dtype
inline size_t rec_size(rosko_dtype d) {
  switch (d) {
    case ROSKO_F32: return 8;
    case ROSKO_BF16: return 4;
    case ROSKO_I8: return 4;
    case ROSKO_F64: return 16;
    default: return 0;
  }
}
inline bool handle_ok(const rosko_packed_s* h) { return h && h->magic == kHandleMagic; }

// api.cu: stream-ordered allocation from the library's own memory pool on
// the current device (freed blocks stay mapped, up to 256 MiB per device, so
// repeated packs skip mapping fresh memory); pool_free releases in the order
// of `st`.  Both honour the allocation-failure test hook of dev_malloc.
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t st);
void pool_free(void* p, cudaStream_t st);

// pack.cu
constexpr int kDenseTileRows = 128;
rosko_status pack_impl(const void* A, rosko_dtype a_dt, int64_t M, int64_t K, int64_t lda,
                       rosko_dtype p_dt, const float* row_scale_in, int32_t m_r,
                       int32_t dense_min_pm, cudaStream_t stream, rosko_packed_s** out);
rosko_status transpose_impl(const void* A, rosko_dtype dt, int64_t M, int64_t K, int64_t lda,
                            void* out, cudaStream_t st);
rosko_status unpack_impl(rosko_packed_s* h, void* A_out, int64_t lda, cudaStream_t stream);
constexpr int64_t kRowSlotMaxK = 65280;  // sentinel k = 0xFFFF stays past every slab end

// A zero fill of C (rows x row_bytes at `pitch` bytes) issued right before a
// tensor-core launch: a small kernel that lets the tensor-core launch start
// at once (programmatic dependent launch); only its epilogue waits for the
// fill, so the fill runs under its MMAs.  (The latency-bound row-direct
// kernel is not launched this way: it needs every SM slot from its start,
// and the early start measured slower than a memset ahead of it.)
struct ZeroFill {
  void* C;
  int64_t pitch, row_bytes, rows;
};
// Launch the zero fill (a kernel whose dependents may start at once).
rosko_status zero_fill_launch(const ZeroFill& z, cudaStream_t st);

// spmm_sparse.cu
struct SparseLaunch {
  int R, V, W, KC, stages, split;
  int order;  // 1 = column order (Alg. 2), 2 = row-slot, 3 = row-slot + gather
};
rosko_status sparse_spmm_launch(rosko_packed_s* h, const void* B, rosko_dtype b_dt, int64_t N,
                                int64_t ldb, const float* col_scale, void* C, rosko_dtype c_dt,
                                int64_t ldc, int accumulate, const SparseLaunch& L,
                                const int32_t* panel_list, int64_t n_panels, bool c_zeroed,
                                cudaStream_t stream);
bool sparse_config_supported(rosko_dtype p_dt, rosko_dtype b_dt, rosko_dtype c_dt, int R, int V,
                             int order);
int sparse_default_V(rosko_dtype p_dt, int R, int order);

// spmm_dense_tc.cu
rosko_status dense_spmm_launch(const void* dense_A, int64_t dense_rows, int64_t Kpad,
                               const int32_t* tile_order_dev, int64_t n_tiles, int64_t K,
                               const void* B, int64_t N, int64_t ldb, float* C, int64_t ldc,
                               int64_t M, int accumulate, int TN, int ctas, int MH,
                               bool c_zeroed, const ZeroFill* zf,
                               cudaStream_t st);
// One row-direct (order 4) sparse SpMM of a batch: the panels of h listed in
// panel_list (NULL: all rows), B and C of this problem.
struct DirectJob {
  rosko_packed_s* h;
  const void* B;
  rosko_dtype b_dt;
  int64_t N, ldb;
  const float* col_scale;
  void* C;
  rosko_dtype c_dt;
  int64_t ldc;
  int accumulate;
  const int32_t* panel_list;
  int64_t n_panels;
};
// Row-direct work segments of the listed panels (NULL list: all panels in
// order; else the handle's panel_order prefix of n_panels); NULL if the list
// is of another kind.  *cut: some listed row is cut into several pieces
// (their sums are added into C, which must then be zeroed unless the call
// accumulates).
const SegEntry* direct_segments(const rosko_packed_s* h, const int32_t* panel_list, int64_t n_panels,
                            int which, int64_t* n_segs, bool* cut);
// The list a launch over these panels with width N and V columns per lane
// uses (0 fine, 1 coarse); decided the same way for zero-fill and launch.
int direct_pick(const rosko_packed_s* h, const int32_t* panel_list, int64_t n_panels, int64_t N,
                int V);
// One launch over all jobs (count <= 64, same handle / B / C types, V
// columns per lane); C of jobs with cut rows must be zeroed by the caller
// unless they accumulate.
rosko_status direct_batch_launch(const DirectJob* jobs, int count, int V, cudaStream_t st,
                                 bool pdl = false);
// One dense-panel SpMM of a batch (see dense_batch_launch).
struct DenseJob {
  const void* dense_A;
  int64_t dense_rows, Kpad;
  const int32_t* tile_order_dev;
  int64_t n_tiles, K;
  const void* B;
  int64_t N, ldb;
  float* C;
  int64_t ldc, M;
  int accumulate;
  int kchunk = 0;    // K slabs per exact-integer chunk (INT8 codes), 0: none
  int out_i32 = 0;   // C is INT32 (INT8 codes through the BF16 pipe)
  int pdl = 0;       // launch as a programmatic dependent of the previous kernel
};
// INT8 x INT8 -> INT32 through the BF16 tensor pipe: B is converted to BF16
// (exact) in stream-ordered scratch, the handle's dense copies hold the INT8
// codes as BF16, and every K chunk of <= 1024 (exact in FP32) is converted
// and added into C, which the caller has zeroed unless it accumulates.
rosko_status dense_spmm_i8_launch(const rosko_packed_s* h, int64_t n_tiles, const int8_t* B,
                                  int64_t N, int64_t ldb, int32_t* C, int64_t ldc, int TN,
                                  int ctas, int MH, const ZeroFill* zf, cudaStream_t st);
// One persistent stream-K launch over all jobs' dense tiles (count <= 64);
// C of jobs whose tiles the split cuts must be zeroed by the caller unless
// they accumulate (dense_batch_needs_zero).
rosko_status dense_batch_launch(const DenseJob* jobs, int count, int TN, int ctas, int MH,
                                cudaStream_t st);
void dense_batch_needs_zero(const DenseJob* jobs, int count, int TN, int ctas, int MH,
                            bool* out);
// stream-K grid size and whether some dense tile is split between CTAs
// (MH = 128-row halves per CTA tile: 1 or 2)
int64_t dense_grid(int64_t n_tiles, int64_t N, int64_t K, int TN, int ctas, int MH);
bool dense_needs_zero(int64_t n_tiles, int64_t N, int64_t K, int TN, int ctas, int MH);

// api.cu
rosko_status spmm_validate(rosko_packed_s* A, const void* B_dev, rosko_dtype b_dtype, int64_t N,
                           int64_t ldb, const float* col_scale_dev, void* C_dev,
                           rosko_dtype c_dtype, int64_t ldc, int accumulate, cudaStream_t st,
                           bool* done);
constexpr int kRunSkipDense = 1;
constexpr int kRunZeroed = 2;
constexpr int kRunPlanOnly = 4;   // resolve the schedule, launch nothing (rosko_spmm_plan)
rosko_status spmm_run(rosko_packed_s* A, const void* B_dev, rosko_dtype b_dtype, int64_t N,
                      int64_t ldb, const float* col_scale_dev, void* C_dev, rosko_dtype c_dtype,
                      int64_t ldc, int accumulate, const rosko_tile* tile, cudaStream_t st,
                      int flags);
rosko_status spmm_batched_impl(int32_t count, rosko_packed_s* const* A, const void* const* B,
                               const int64_t* N, const int64_t* ldb, void* const* C,
                               const int64_t* ldc, rosko_dtype b_dt, rosko_dtype c_dt,
                               int accumulate, const rosko_tile* tiles, cudaStream_t st);
rosko_status spmm_forced(rosko_packed_s* h, const void* B, rosko_dtype b_dt, int64_t N, int64_t ldb,
                         const float* col_scale, void* C, rosko_dtype c_dt, int64_t ldc,
                         const rosko_tile* t, cudaStream_t st);
rosko_status schedule_analytic(int64_t M, int64_t K, int64_t N, int64_t nnz, int32_t m_r,
                               rosko_dtype dt, int sms, rosko_tile* t);

// autotune.cu
int num_candidates();
bool candidate_tile(const rosko_packed_s* h, int64_t N, int idx, rosko_tile* t);
int analytic_candidate(const rosko_packed_s* h, int64_t N);
int candidate_index(const rosko_tile* t, rosko_dtype dt);
rosko_status autotune_impl(rosko_packed_s* h, const void* B, rosko_dtype b_dt, int64_t N,
                           int64_t ldb, const float* col_scale, void* C, rosko_dtype c_dt,
                           int64_t ldc, int reps, rosko_tile* best, float* times,
                           int32_t* n_out, cudaStream_t st);

// serialize.cu
rosko_status packed_serialize(const rosko_packed_s* h, void* buf, int64_t cap, int64_t* bytes);
rosko_status packed_deserialize(const void* buf, int64_t bytes, cudaStream_t st,
                                rosko_packed_s** out);

// selector.cu
rosko_status select_learned(rosko_packed_s* h, int64_t N, rosko_tile* out, cudaStream_t st);
rosko_status features_impl(rosko_packed_s* h, int64_t N, double* f, cudaStream_t st);
// Allocation-free variant: FP32 features written to device memory, scratch
// in a static device array (M <= 1 << 20).
rosko_status features_static_impl(rosko_packed_s* h, int64_t N, float* features_dev,
                                  cudaStream_t st);
int64_t mlp_param_count(int n_in, int n_out);
int64_t mlp_workspace_floats(int64_t batch, int n_out);
rosko_status mlp_forward(const float* params, const float* X, int64_t batch, int n_in, int n_out,
                         float* acts, float* logits, cudaStream_t st);
rosko_status mlp_loss_grad(const float* params, const float* X, const float* Y, int64_t batch,
                           int n_in, int n_out, float* grads, float* loss, float* ws,
                           cudaStream_t st);
rosko_status mlp_adam(float* p, const float* g, float* m, float* v, int64_t n, int step, float lr,
                      float b1, float b2, float eps, float wd, cudaStream_t st);
rosko_status selector_set(const float* params, int n_params, int n_out, const double* mean,
                          const double* stdv, const double* lo, const double* hi);
float time_tile(rosko_packed_s* h, const void* B, rosko_dtype b_dt, int64_t N, int64_t ldb,
                const float* col_scale, void* C, rosko_dtype c_dt, int64_t ldc,
                const rosko_tile* t, int reps, cudaStream_t st, rosko_status* err);
}  // namespace rosko
