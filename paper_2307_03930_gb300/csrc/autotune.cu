// Schedule candidates and the per-shape autotuner (Sec. 6 exposes m_c, k_c,
// m_r, n_r for auto-tuning; this library searches them on the device).
//
// The candidate set is a fixed enumeration: a sparse-path configuration
// (traversal order, CTA height m_c, slab depth k_c, K split) crossed with a
// dense-split threshold for BF16 handles.  The learned selector predicts an
// index into the same enumeration, so the autotuner's timings are its labels.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "handle.hpp"

namespace rosko {

namespace {

struct SparseCand {
  int order, W, KC, split, V;   // V = 0: the order's default width
};

// Sparse-path configurations (m_r comes from the pack, n_r from the order
// unless V is given).
const SparseCand kSparse[] = {
    {2, 4, 64, 1, 0}, {2, 4, 64, 4, 0}, {2, 8, 32, 2, 0}, {4, 1, 8, 1, 16},
    {3, 8, 64, 1, 0}, {3, 8, 128, 2, 0}, {3, 8, 128, 4, 0}, {3, 8, 256, 8, 0},
    {1, 4, 64, 1, 0}, {1, 8, 32, 4, 0}, {4, 1, 8, 1, 4}, {4, 1, 8, 1, 8},
};
constexpr int kNumSparse = sizeof(kSparse) / sizeof(kSparse[0]);
// Dense-split thresholds in per mille (1001 = never); 15 is the analytic
// rule's break-even density.
const int kDensePm[] = {1001, 1, 5, 15, 60};
constexpr int kNumDense = sizeof(kDensePm) / sizeof(kDensePm[0]);

}  // namespace

int num_candidates() { return kNumSparse * kNumDense; }

// Fill candidate `idx` for handle h; returns false when it does not apply to
// this handle (missing stream, no dense copies, shared memory too small).
bool candidate_tile(const rosko_packed_s* h, int64_t N, int idx, rosko_tile* t) {
  (void)N;
  if (idx < 0 || idx >= num_candidates()) return false;
  const SparseCand& sc = kSparse[idx / kNumDense];
  const int dpct = kDensePm[idx % kNumDense];
  if (sc.order == 3 && (!h->gnz || h->m_r != 16)) return false;
  if ((sc.order == 2 || sc.order == 4) && !h->rnz) return false;
  if (dpct <= 1000 && !(h->dt == ROSKO_BF16 && h->n_copy > 0)) return false;
  const int V = sc.V > 0 ? sc.V : sparse_default_V(h->dt, h->m_r, sc.order);
  if (sc.order == 4) {
    // the B and C types are those of the handle's usual call
    const rosko_dtype b = h->dt == ROSKO_F64 ? ROSKO_F32 : h->dt;
    const rosko_dtype c = h->dt == ROSKO_I8 ? ROSKO_I32 : (h->dt == ROSKO_F64 ? ROSKO_F64 : ROSKO_F32);
    if (!sparse_config_supported(h->dt, b, c, h->m_r, V, 4)) return false;
  }
  const int W = sc.order == 3 ? 128 / h->m_r : sc.W;
  const size_t esz = h->dt == ROSKO_F64 ? 4 : dtype_size(h->dt);
  if (2 * (size_t)sc.KC * 32 * V * esz > 200 * 1024) return false;
  std::memset(t, 0, sizeof(*t));
  t->m_r = h->m_r;
  t->n_r = 32 * V;
  t->k_c = sc.KC;
  t->m_c = W * h->m_r;
  t->split_k = sc.split;
  t->dense_split_pm = dpct;
  t->order = sc.order;
  t->mode = ROSKO_SCHED_FORCED;
  return true;
}

// Index of the candidate with the schedule of tile t (same traversal, columns
// per lane, dense threshold and, for the slab traversals, CTA height, slab
// depth and K split), or -1; t->m_r is the handle's panel height.
int candidate_index(const rosko_tile* t, rosko_dtype dt) {
  for (int i = 0; i < num_candidates(); ++i) {
    const SparseCand& sc = kSparse[i / kNumDense];
    if (sc.order != t->order || kDensePm[i % kNumDense] != t->dense_split_pm) continue;
    const int V = sc.V > 0 ? sc.V : sparse_default_V(dt, t->m_r, sc.order);
    if (32 * V != t->n_r) continue;
    if (sc.order != 4) {
      const int W = sc.order == 3 ? 128 / t->m_r : sc.W;
      if (W * t->m_r != t->m_c || sc.KC != t->k_c || sc.split != t->split_k) continue;
    }
    return i;
  }
  return -1;
}

// The applicable candidate whose schedule is the analytic rule's for this
// handle and width, or -1.
int analytic_candidate(const rosko_packed_s* h, int64_t N) {
  rosko_tile a;
  schedule_analytic(h->M, h->K, N, h->nnz, h->m_r, h->dt, num_sms(), &a);
  const int i = candidate_index(&a, h->dt);
  rosko_tile t;
  return (i >= 0 && candidate_tile(h, N, i, &t)) ? i : -1;
}

rosko_status spmm_forced(rosko_packed_s* h, const void* B, rosko_dtype b_dt, int64_t N, int64_t ldb,
                         const float* col_scale, void* C, rosko_dtype c_dt, int64_t ldc,
                         const rosko_tile* t, cudaStream_t st);

// A buffer larger than L2 (129 MB on GB300) that the autotuner overwrites
// before every timed launch, so that B is read from HBM as in a real layer.
static void* flush_buffer(size_t* bytes) {
  static void* buf = nullptr;
  static size_t nbytes = 0;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (!buf) {
    int l2 = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    nbytes = (size_t)std::max(l2, 64 << 20) * 2;
    if (cudaMalloc(&buf, nbytes) != cudaSuccess) {
      buf = nullptr;
      nbytes = 0;
      cudaGetLastError();
    }
  }
  *bytes = nbytes;
  return buf;
}

// Mean device time of one launch of candidate t: `reps` launches, each after
// an L2 flush, captured as one CUDA graph on the private stream ts (host
// launch overhead is not measured), minus the same graph without the
// launches.  Returns < 0 on error.
static float time_candidate(rosko_packed_s* h, const void* B, rosko_dtype b_dt, int64_t N,
                            int64_t ldb, const float* col_scale, void* C, rosko_dtype c_dt,
                            int64_t ldc, const rosko_tile* t, int reps, cudaStream_t ts,
                            cudaEvent_t e0, cudaEvent_t e1, rosko_status* err) {
  *err = spmm_forced(h, B, b_dt, N, ldb, col_scale, C, c_dt, ldc, t, ts);  // first-use setup
  if (*err != ROSKO_OK) return -1.0f;
  size_t fbytes = 0;
  void* fbuf = flush_buffer(&fbytes);
  float result[2] = {-1.0f, 0.0f};
  for (int pass = 0; pass < (fbuf ? 2 : 1); ++pass) {
    const bool with_kernel = pass == 0;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    bool graphed = false;
    if (cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      rosko_status s = ROSKO_OK;
      for (int r = 0; r < reps && s == ROSKO_OK; ++r) {
        if (fbuf && cudaMemsetAsync(fbuf, r & 0xff, fbytes, ts) != cudaSuccess) s = ROSKO_ERR_CUDA;
        if (with_kernel && s == ROSKO_OK)
          s = spmm_forced(h, B, b_dt, N, ldb, col_scale, C, c_dt, ldc, t, ts);
      }
      const cudaError_t ec = cudaStreamEndCapture(ts, &g);
      graphed = s == ROSKO_OK && ec == cudaSuccess && g &&
                cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
    }
    cudaGetLastError();
    if (graphed) {
      cudaGraphLaunch(ge, ts);  // warm
      cudaEventRecord(e0, ts);
      cudaGraphLaunch(ge, ts);
      cudaEventRecord(e1, ts);
    } else {
      cudaEventRecord(e0, ts);
      for (int r = 0; r < reps; ++r) {
        if (fbuf) cudaMemsetAsync(fbuf, r & 0xff, fbytes, ts);
        if (with_kernel) spmm_forced(h, B, b_dt, N, ldb, col_scale, C, c_dt, ldc, t, ts);
      }
      cudaEventRecord(e1, ts);
    }
    float ms = -1.0f;
    if (cudaEventSynchronize(e1) == cudaSuccess &&
        cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
      result[pass] = ms / (float)reps;
    else
      *err = ROSKO_ERR_CUDA;
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (*err != ROSKO_OK) return -1.0f;
  }
  return std::max(result[0] - result[1], 1e-4f);
}

float time_tile(rosko_packed_s* h, const void* B, rosko_dtype b_dt, int64_t N, int64_t ldb,
                const float* col_scale, void* C, rosko_dtype c_dt, int64_t ldc,
                const rosko_tile* t, int reps, cudaStream_t st, rosko_status* err) {
  *err = ROSKO_OK;
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    *err = ROSKO_ERR_CUDA;
    return -1.0f;
  }
  cudaStream_t ts;
  cudaEvent_t e0, e1;
  if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess) {
    *err = ROSKO_ERR_CUDA;
    return -1.0f;
  }
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const float ms = time_candidate(h, B, b_dt, N, ldb, col_scale, C, c_dt, ldc, t,
                                  reps < 1 ? 3 : reps, ts, e0, e1, err);
  cudaStreamSynchronize(ts);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(ts);
  return ms;
}

rosko_status autotune_impl(rosko_packed_s* h, const void* B, rosko_dtype b_dt, int64_t N,
                           int64_t ldb, const float* col_scale, void* C, rosko_dtype c_dt,
                           int64_t ldc, int reps, rosko_tile* best, float* times,
                           int32_t* n_out, cudaStream_t st) {
  if (reps < 1) reps = 3;
  const int nc = num_candidates();
  if (cudaStreamSynchronize(st) != cudaSuccess) return ROSKO_ERR_CUDA;
  cudaStream_t ts;
  if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess) return ROSKO_ERR_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) {
    cudaStreamDestroy(ts);
    return ROSKO_ERR_CUDA;
  }
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaStreamDestroy(ts);
    return ROSKO_ERR_CUDA;
  }
  float best_ms = 1e30f;
  int best_i = -1;
  rosko_tile bt{};
  rosko_status ret = ROSKO_OK;
  for (int i = 0; i < nc; ++i) {
    rosko_tile t;
    if (!candidate_tile(h, N, i, &t)) {
      if (times) times[i] = -1.0f;
      continue;
    }
    rosko_status s = ROSKO_OK;
    const float ms = time_candidate(h, B, b_dt, N, ldb, col_scale, C, c_dt, ldc, &t, reps, ts, e0,
                                    e1, &s);
    if (s == ROSKO_ERR_UNSUPPORTED || s == ROSKO_ERR_INVALID_ARG) {
      if (times) times[i] = -1.0f;
      continue;
    }
    if (s != ROSKO_OK) {
      ret = s;
      break;
    }
    if (times) times[i] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best_i = i;
      bt = t;
    }
  }
  cudaStreamSynchronize(ts);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(ts);
  if (ret != ROSKO_OK) return ret;
  if (n_out) *n_out = nc;
  if (best_i < 0) return ROSKO_ERR_UNSUPPORTED;
  *best = bt;
  return ROSKO_OK;
}

}  // namespace rosko
