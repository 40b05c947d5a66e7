// C-ABI entry points (include/rosko.h): argument validation, handle
// management, the analytic schedule and kernel dispatch.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "handle.hpp"

namespace rosko {

namespace {
std::mutex g_mu;
int* g_status[64] = {nullptr};
int g_sms[64] = {0};
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
  {
    // Test hook: ROSKO_FAIL_ALLOC=n makes the n-th device allocation after the
    // variable took its current value fail (host-side fault injection).
    static std::string last;
    static long since = 0;
    std::lock_guard<std::mutex> lk(g_mu);
    const char* f = std::getenv("ROSKO_FAIL_ALLOC");
    if (!f) {
      last.clear();
      since = 0;
    } else {
      if (last != f) {
        last = f;
        since = 0;
      }
      if (std::atol(f) == ++since) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
    }
  }
  return cudaMalloc(p, bytes < 256 ? 256 : bytes);
}

namespace {
std::atomic<int64_t> g_launches{0};
}
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int* device_status_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_status[dev]) {
    void* p = nullptr;
    if (cudaMalloc(&p, 256) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, 256) != cudaSuccess) return nullptr;
    g_status[dev] = static_cast<int*>(p);
  }
  return g_status[dev];
}

int num_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_sms[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 152;
    g_sms[dev] = n;
  }
  return g_sms[dev];
}

CUresult encode_tiled(CUtensorMap* map, CUtensorMapDataType dt, cuuint32_t rank, void* gaddr,
                      const cuuint64_t* dims, const cuuint64_t* strides, const cuuint32_t* box,
                      const cuuint32_t* estrides, CUtensorMapInterleave il, CUtensorMapSwizzle sw,
                      CUtensorMapL2promotion l2, CUtensorMapFloatOOBfill oob) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_encode) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                           &q) != cudaSuccess ||
          q != cudaDriverEntryPointSuccess || !fn)
        return CUDA_ERROR_NOT_FOUND;
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
  }
  return g_encode(map, dt, rank, gaddr, dims, strides, box, estrides, il, sw, l2, oob);
}

// ---------------------------------------------------------------------------
// Analytic schedule: Sec. 4.2 re-derived for one GB300.
//
// Register level (Eq. 3 analog): a warp keeps an m_r x 32V C tile in
// registers; each staged B element is reused d*m_r times, so m_r is as large
// as the register file allows (m_r * V accumulators <= 128 per lane).
// Shared-memory level (Eq. 1 analog, per SM instead of per core): the ring of
// `stages` k_c x n_r B slabs must leave room for two CTAs per SM
// (<= ~100 KB each) so that one CTA's epilogue overlaps another's stream.
// Chip level (Eq. 2 analog): B is re-read from L2 once per CTA row group,
// ceil(M / m_c) times, so m_c = W m_r grows with M; K is split only as far as
// needed to put ~2 CTAs on every SM.
// ---------------------------------------------------------------------------
rosko_status schedule_analytic(int64_t M, int64_t K, int64_t N, int64_t nnz, int32_t m_r,
                               rosko_dtype dt, int sms, rosko_tile* t) {
  (void)nnz;
  if (m_r <= 0) m_r = (dt == ROSKO_F64) ? 16 : 32;
  const int V = sparse_default_V(dt, m_r);
  const int NR = 32 * V;
  const int64_t P = (M + m_r - 1) / m_r;
  int W = 4;
  if (P >= 64) W = 8;
  if (P < 4) W = (int)std::max<int64_t>(P, 1);
  const int KC = 32;
  const int64_t tiles = ((P + W - 1) / W) * ((N + NR - 1) / NR);
  const int64_t slabs = (K + KC - 1) / KC;
  int64_t split = 1;
  const int64_t target = 2LL * sms;
  if (tiles > 0 && tiles < target) split = (target + tiles - 1) / tiles;
  split = std::max<int64_t>(1, std::min<int64_t>(split, std::max<int64_t>(1, slabs / 8)));
  t->m_r = m_r;
  t->n_r = NR;
  t->k_c = KC;
  t->m_c = W * m_r;
  t->split_k = (int32_t)split;
  t->dense_split_pct = 101;
  t->mode = ROSKO_SCHED_ANALYTIC;
  return ROSKO_OK;
}

}  // namespace rosko

using namespace rosko;

extern "C" {

const char* rosko_status_string(rosko_status s) {
  switch (s) {
    case ROSKO_OK: return "ROSKO_OK";
    case ROSKO_ERR_INVALID_ARG: return "ROSKO_ERR_INVALID_ARG";
    case ROSKO_ERR_UNSUPPORTED: return "ROSKO_ERR_UNSUPPORTED";
    case ROSKO_ERR_OOM: return "ROSKO_ERR_OOM";
    case ROSKO_ERR_CUDA: return "ROSKO_ERR_CUDA";
    case ROSKO_ERR_TIMEOUT: return "ROSKO_ERR_TIMEOUT";
    case ROSKO_ERR_BAD_HANDLE: return "ROSKO_ERR_BAD_HANDLE";
    case ROSKO_ERR_DEVICE: return "ROSKO_ERR_DEVICE";
  }
  return "ROSKO_ERR_UNKNOWN";
}

rosko_status rosko_pack(const void* A_dev, rosko_dtype a_dtype, int64_t M, int64_t K, int64_t lda,
                        rosko_dtype packed_dtype, const float* row_scale_dev,
                        const rosko_tile* tile, rosko_stream_t stream, rosko_packed_t* out) {
  if (!out) return ROSKO_ERR_INVALID_ARG;
  *out = nullptr;
  if (!dtype_valid(a_dtype) || !dtype_valid(packed_dtype)) return ROSKO_ERR_INVALID_ARG;
  if (M < 0 || K < 0 || lda < std::max<int64_t>(K, 1)) return ROSKO_ERR_INVALID_ARG;
  if (M * K > 0 && !A_dev) return ROSKO_ERR_INVALID_ARG;
  if (M > 0 && K > 0 && M > (int64_t)INT32_MAX / K) return ROSKO_ERR_INVALID_ARG;
  const bool ok_pair = (a_dtype == ROSKO_F32 && (packed_dtype == ROSKO_F32 ||
                                                 packed_dtype == ROSKO_BF16 ||
                                                 packed_dtype == ROSKO_I8 ||
                                                 packed_dtype == ROSKO_F64)) ||
                       (a_dtype == ROSKO_BF16 && packed_dtype == ROSKO_BF16) ||
                       (a_dtype == ROSKO_I8 && packed_dtype == ROSKO_I8);
  if (!ok_pair) return ROSKO_ERR_UNSUPPORTED;
  if (row_scale_dev && !(a_dtype == ROSKO_I8 && packed_dtype == ROSKO_I8))
    return ROSKO_ERR_INVALID_ARG;
  int32_t m_r = (tile && tile->m_r > 0) ? tile->m_r : (packed_dtype == ROSKO_F64 ? 16 : 32);
  if (m_r != 8 && m_r != 16 && m_r != 32) return ROSKO_ERR_INVALID_ARG;
  const int64_t P = (M + m_r - 1) / m_r;
  if (P > 65535) return ROSKO_ERR_INVALID_ARG;
  rosko_packed_s* h = nullptr;
  rosko_status s = pack_impl(A_dev, a_dtype, M, K, lda, packed_dtype, row_scale_dev, m_r,
                             static_cast<cudaStream_t>(stream), &h);
  if (s != ROSKO_OK) return s;
  *out = h;
  return ROSKO_OK;
}

void rosko_free(rosko_packed_t A) {
  if (!A || A->magic != kHandleMagic) return;
  A->magic = 0;
  if (A->meta_base) cudaFree(A->meta_base);
  if (A->data_base) cudaFree(A->data_base);
  delete A;
}

rosko_status rosko_schedule_analytic(int64_t M, int64_t K, int64_t N, int64_t nnz, int32_t m_r,
                                     rosko_dtype packed_dtype, rosko_tile* tile) {
  if (!tile || M < 0 || K < 0 || N < 0 || nnz < 0 || !dtype_valid(packed_dtype))
    return ROSKO_ERR_INVALID_ARG;
  if (m_r > 0 && m_r != 8 && m_r != 16 && m_r != 32) return ROSKO_ERR_INVALID_ARG;
  return schedule_analytic(M, K, N, nnz, m_r, packed_dtype, 152, tile);
}

rosko_status rosko_spmm(rosko_packed_t A, const void* B_dev, rosko_dtype b_dtype, int64_t N,
                        int64_t ldb, const float* col_scale_dev, void* C_dev,
                        rosko_dtype c_dtype, int64_t ldc, int accumulate,
                        const rosko_tile* tile, rosko_stream_t stream) {
  if (!handle_ok(A)) return ROSKO_ERR_BAD_HANDLE;
  if (!dtype_valid(b_dtype) || !dtype_valid(c_dtype)) return ROSKO_ERR_INVALID_ARG;
  if (N < 0 || ldb < std::max<int64_t>(N, 1) || ldc < std::max<int64_t>(N, 1))
    return ROSKO_ERR_INVALID_ARG;
  if (N > 65535LL * 128) return ROSKO_ERR_INVALID_ARG;
  const rosko_dtype p = A->dt;
  const bool combo = (p == ROSKO_F32 && b_dtype == ROSKO_F32 && c_dtype == ROSKO_F32) ||
                     (p == ROSKO_BF16 && b_dtype == ROSKO_BF16 && c_dtype == ROSKO_F32) ||
                     (p == ROSKO_I8 && b_dtype == ROSKO_I8 &&
                      (c_dtype == ROSKO_I32 || c_dtype == ROSKO_F32)) ||
                     (p == ROSKO_F64 && b_dtype == ROSKO_F32 && c_dtype == ROSKO_F64);
  if (!combo) return ROSKO_ERR_UNSUPPORTED;
  const bool dequant = (p == ROSKO_I8 && c_dtype == ROSKO_F32);
  if (dequant != (col_scale_dev != nullptr)) return ROSKO_ERR_INVALID_ARG;
  if (A->M == 0 || N == 0) return ROSKO_OK;
  if (!C_dev) return ROSKO_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ROSKO_ERR_CUDA;
  if (dev != A->device) return ROSKO_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t csz = dtype_size(c_dtype);
  if (A->K == 0 || A->nnz == 0) {
    if (accumulate) return ROSKO_OK;
    return cudaMemset2DAsync(C_dev, (size_t)ldc * csz, 0, (size_t)N * csz, (size_t)A->M, st) ==
                   cudaSuccess
               ? ROSKO_OK
               : ROSKO_ERR_CUDA;
  }
  if (!B_dev) return ROSKO_ERR_INVALID_ARG;
  const size_t bsz = dtype_size(b_dtype);
  if ((reinterpret_cast<uintptr_t>(B_dev) % 16) != 0 || ((size_t)ldb * bsz) % 16 != 0)
    return ROSKO_ERR_INVALID_ARG;

  rosko_tile t{};
  const bool forced = tile && tile->mode == ROSKO_SCHED_FORCED;
  schedule_analytic(A->M, A->K, N, A->nnz, A->m_r, p, num_sms(), &t);
  if (tile) {
    if (tile->m_r > 0 && tile->m_r != A->m_r) return ROSKO_ERR_INVALID_ARG;
    if (tile->n_r > 0) t.n_r = tile->n_r;
    if (tile->k_c > 0) t.k_c = tile->k_c;
    if (tile->m_c > 0) t.m_c = tile->m_c;
    if (tile->split_k > 0) t.split_k = tile->split_k;
    if (forced && (tile->n_r <= 0 || tile->k_c <= 0 || tile->m_c <= 0 || tile->split_k <= 0))
      return ROSKO_ERR_INVALID_ARG;
  }
  SparseLaunch L;
  L.R = A->m_r;
  if (t.n_r % 32 != 0) return ROSKO_ERR_INVALID_ARG;
  L.V = t.n_r / 32;
  if (t.m_c % A->m_r != 0) return ROSKO_ERR_INVALID_ARG;
  L.W = t.m_c / A->m_r;
  L.KC = t.k_c;
  L.split = t.split_k;
  if (L.W < 1 || L.W > 8 || L.KC < 8 || L.KC > 256 || L.KC % 8 != 0 || L.split < 1 ||
      L.split > 65535)
    return ROSKO_ERR_INVALID_ARG;
  if (!sparse_config_supported(p, b_dtype, c_dtype, L.R, L.V)) return ROSKO_ERR_UNSUPPORTED;
  // B ring: up to 4 slabs, at least 2, within ~200 KB of shared memory
  const size_t stage_bytes = (size_t)L.KC * 32 * L.V * bsz;
  L.stages = (int)std::min<size_t>(4, (200 * 1024) / stage_bytes);
  if (L.stages < 2) return ROSKO_ERR_INVALID_ARG;
  return sparse_spmm_launch(A, B_dev, b_dtype, N, ldb, col_scale_dev, C_dev, c_dtype, ldc,
                            accumulate, L, st);
}

rosko_status rosko_unpack(rosko_packed_t A, void* A_dev_out, int64_t lda, rosko_stream_t stream) {
  if (!handle_ok(A)) return ROSKO_ERR_BAD_HANDLE;
  if (lda < std::max<int64_t>(A->K, 1)) return ROSKO_ERR_INVALID_ARG;
  if (A->M * A->K > 0 && !A_dev_out) return ROSKO_ERR_INVALID_ARG;
  return unpack_impl(A, A_dev_out, lda, static_cast<cudaStream_t>(stream));
}

rosko_status rosko_packed_info(rosko_packed_t A, int64_t* nnz, int64_t* bytes, int64_t* touched_k,
                               int64_t* n_panels, int32_t* m_r, int32_t* packed_dtype,
                               int64_t* n_cols) {
  if (!handle_ok(A)) return ROSKO_ERR_BAD_HANDLE;
  if (nnz) *nnz = A->nnz;
  // values + 1-byte rows + per column (col_ind, start) + panel offsets
  if (bytes)
    *bytes = A->nnz * (int64_t)(dtype_size(A->dt) + 1) + A->n_cols * 8 + (A->P + 1) * 4 + 4;
  if (touched_k) *touched_k = A->touched_k;
  if (n_panels) *n_panels = A->P;
  if (m_r) *m_r = A->m_r;
  if (packed_dtype) *packed_dtype = (int32_t)A->dt;
  if (n_cols) *n_cols = A->n_cols;
  return ROSKO_OK;
}

rosko_status rosko_packed_export(rosko_packed_t A, void* A_p_host, uint8_t* loc_m_host,
                                 int32_t* col_ind_host, int32_t* nnz_host,
                                 int64_t* panel_cols_host) {
  if (!handle_ok(A)) return ROSKO_ERR_BAD_HANDLE;
  const size_t esz = dtype_size(A->dt);
  if (cudaDeviceSynchronize() != cudaSuccess) return ROSKO_ERR_CUDA;
  if (A_p_host && A->nnz &&
      cudaMemcpy(A_p_host, A->vals, (size_t)A->nnz * esz, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ROSKO_ERR_CUDA;
  if (loc_m_host && A->nnz &&
      cudaMemcpy(loc_m_host, A->rows, (size_t)A->nnz, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ROSKO_ERR_CUDA;
  if (col_ind_host && A->n_cols &&
      cudaMemcpy(col_ind_host, A->col_ind, (size_t)A->n_cols * 4, cudaMemcpyDeviceToHost) !=
          cudaSuccess)
    return ROSKO_ERR_CUDA;
  if (nnz_host && A->n_cols) {
    std::vector<int32_t> cs((size_t)A->n_cols + 1);
    if (cudaMemcpy(cs.data(), A->col_start, cs.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return ROSKO_ERR_CUDA;
    for (int64_t c = 0; c < A->n_cols; ++c) nnz_host[c] = cs[c + 1] - cs[c];
  }
  if (panel_cols_host) {
    std::vector<int32_t> pc((size_t)A->P + 1);
    if (cudaMemcpy(pc.data(), A->panel_col, pc.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return ROSKO_ERR_CUDA;
    for (int64_t i = 0; i <= A->P; ++i) panel_cols_host[i] = pc[i];
  }
  return ROSKO_OK;
}

int64_t rosko_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

rosko_status rosko_device_status(int32_t* bits, int clear) {
  if (!bits) return ROSKO_ERR_INVALID_ARG;
  int* w = device_status_word();
  if (!w) return ROSKO_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return ROSKO_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ROSKO_ERR_CUDA;
  *bits = v;
  if (clear && cudaMemset(w, 0, sizeof(int)) != cudaSuccess) return ROSKO_ERR_CUDA;
  return ROSKO_OK;
}

}  // extern "C"
