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
#include <memory>
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

namespace {
// Test hook: ROSKO_FAIL_ALLOC=n makes the n-th device allocation after the
// variable took its current value fail (host-side fault injection).
bool fail_alloc_hook() {
  static std::string last;
  static long since = 0;
  std::lock_guard<std::mutex> lk(g_mu);
  const char* f = std::getenv("ROSKO_FAIL_ALLOC");
  if (!f) {
    last.clear();
    since = 0;
    return false;
  }
  if (last != f) {
    last = f;
    since = 0;
  }
  return std::atol(f) == ++since;
}

// Freed pool memory kept mapped for later packs, per device.
constexpr uint64_t kPoolKeepBytes = 256ull << 20;
cudaMemPool_t g_pool[64] = {};
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
  *p = nullptr;
  if (fail_alloc_hook()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes < 256 ? 256 : bytes);
}

cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (fail_alloc_hook()) return cudaErrorMemoryAllocation;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_pool[dev]) {
      cudaMemPoolProps props;
      std::memset(&props, 0, sizeof(props));
      props.allocType = cudaMemAllocationTypePinned;
      props.handleTypes = cudaMemHandleTypeNone;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t created = nullptr;
      e = cudaMemPoolCreate(&created, &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = kPoolKeepBytes;
      e = cudaMemPoolSetAttribute(created, cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) {
        cudaMemPoolDestroy(created);
        return e;
      }
      g_pool[dev] = created;
    }
    pool = g_pool[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes < 256 ? 256 : bytes, pool, st);
}

void pool_free(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

namespace {
std::atomic<int64_t> g_launches{0};
}

// Failure-detection probe: an mbarrier expecting two arrivals gets one, so
// its phase never completes and the bounded wait runs out.
__global__ void probe_wait_kernel(int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 2);
    fence_barrier_init();
  }
  __syncwarp();
  if (threadIdx.x == 0) mbar_arrive(&bar);
  __syncwarp();
  if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, status);
  __syncwarp();
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

// Tensor-core dense-panel tiles (measured on GB300, stream-K kernel):
//  * K of fewer than 16 slabs (K < 1024): cutting tiles along K buys little
//    and costs a zero fill of C and reduce-adds, so every tile is owned whole
//    by one CTA (one per tile, or one per SM walking several); 128-wide
//    tiles give more of them;
//  * otherwise 256 columns per tile (half the L2 -> SM traffic of A against
//    128) and either 256 rows when each CTA gets enough K work, or 128 rows
//    with one tile per CTA when the tiles nearly fill the GPU, or 128 rows
//    with the (tile, slab) units shared by one CTA per SM (stream-K).
void dense_config(int64_t n_tiles, int64_t N, int64_t K, int sms, int* TN_out, int* ctas_out,
                  int* mc_out, bool chunked) {
  const int64_t slabs = (K + 63) / 64;
  if (slabs < 16) {
    const int64_t tiles = n_tiles * ((N + 127) / 128);
    *TN_out = 128;
    *mc_out = 128;
    // up to two tiles per SM: one CTA per tile; beyond: one persistent CTA
    // per SM walking whole tiles (its epilogue overlaps the next tile's MMAs)
    *ctas_out = (int)std::max<int64_t>(1, tiles <= 2 * sms ? tiles : sms);
    return;
  }
  *TN_out = N > 128 ? 256 : 128;
  const int64_t ntn = (N + *TN_out - 1) / *TN_out;
  // 256-row tiles (two MMAs per B stage: a third less L2 -> SM traffic per
  // flop, eight MMAs per ring step) hold their accumulator in all of TMEM,
  // so the 256 KB epilogue of a CTA (~28 B/clk per SM through the TMA store
  // path) overlaps no MMAs.  They pay when each CTA has enough K work to
  // amortise it: ~20 double slabs or more (1024x4096x4096: 33.7 against
  // 37.5 us; 512x4608x3136, 12 per CTA: 26.9 against 23.0 us).
  // (INT8 codes drain the accumulator every 1,024 K: that needs the second
  // TMEM set to overlap the drains, so their tiles stay 128 rows high;
  // 11008x4096x2048 at 90 %: 205 against 268 us)
  const int64_t pair_units = (n_tiles + 1) / 2 * ntn * slabs;
  if (!chunked && pair_units >= 20LL * sms) {
    *mc_out = 256;
    *ctas_out = sms;
    return;
  }
  *mc_out = 128;
  // one whole tile per CTA when the tiles nearly fill the GPU (no K split:
  // no zero fill of C, no reductions, a store epilogue; 2048^3: 21.4 against
  // 23.7 us), else stream-K over every SM
  const int64_t tiles = n_tiles * ntn;
  *ctas_out = (4 * tiles >= 3 * (int64_t)sms && tiles <= sms) ? (int)tiles : sms;
}

// Density (per mille) from which a 128-row tile runs on the tensor cores.
// Sec. 4.2 balances work against bandwidth; here the balance is between two
// engines: a dense tile costs 2*128*K*N tensor-core flops, its sparse form
// moves nnz*N B values from L2 into the row-direct kernel, so the break-even
// density is the ratio of the two engines' effective rates.  Measured on
// GB300 for a 512 x 4608 x 3136 layer: ~0.8 PFLOP/s of dense work for the
// stream-K tcgen05 kernel against ~12 TB/s of B bytes for the row-direct
// kernel (BF16: 2 bytes per multiply-add), i.e. d = 12e12 / 0.8e15 = 1.5%
// (the autotuner and the selector refine it per shape).
constexpr int kDenseSplitPm = 15;
constexpr int kDenseCopyPm = 1;
// INT8 codes through the BF16 tensor pipe (exact, K chunks of 1024 added into
// INT32 C): against ~15 TOPS of 2*nnz*N for the INT8 row-direct kernel
// (c3 shapes) the break-even tile density is again near 1.5%; dense copies of
// INT8 packs are kept from 1% (the copies are BF16: twice the INT8 bytes).
constexpr int kDenseSplitPmI8 = 15;
constexpr int kDenseCopyPmI8 = 10;

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
  if (m_r <= 0) m_r = 16;
  const double d = (M * K > 0) ? (double)nnz / ((double)M * (double)K) : 0.0;
  // Traversal: row-direct (each C row walks its own nonzeros, k ascending,
  // and reads their B rows straight from L2; needs the 16-bit-k row stream).
  // A staged B slab pays only when many of a CTA's rows use its rows, and
  // From 50% to 99.8% sparsity (512 x 4608 x 3136, FP32 and BF16) it is in
  // fact 3-4x faster than the slab orders everywhere, so it is the default
  // whenever the row stream exists (K < 65280).
  int order = K < kRowSlotMaxK ? 4 : 1;
  int V = sparse_default_V(dt, m_r, order);
  // row-direct, BF16, density below 1.5%: 512-column strips (two 16-byte
  // chunks per lane) halve the work items, and with them the dependent
  // segment and record loads per byte of B (512 x 4608 x 3136 layer: 7.4
  // against 8.3 us at 99.8%, 18.3 against 18.6 us at 99%; denser layers are
  // faster with 256 columns)
  if (order == 4 && dt == ROSKO_BF16 && d < 0.015 && N >= 1024) V = 16;
  const int NR = 32 * V;
  const int64_t P = (M + m_r - 1) / m_r;
  int W = 4;
  if (P >= 64) W = 8;
  if (P < 4) W = (int)std::max<int64_t>(P, 1);
  if (order == 3) W = 128 / m_r;  // one CTA per 128-row tile
  // 4-slab ring within ~100 KB so two CTAs share an SM
  const int64_t bsz = (dt == ROSKO_BF16) ? 2 : (dt == ROSKO_I8 ? 1 : 4);
  int KC = (int)((100 * 1024) / (4 * (int64_t)NR * bsz)) / 8 * 8;
  KC = std::max(8, std::min(64, KC));
  const int64_t tiles = ((P + W - 1) / W) * ((N + NR - 1) / NR);
  // order 3 streams only the touched rows of each tile: ~(1 - (1-d)^128) K
  const double touched = order == 3 ? 1.0 - std::pow(1.0 - d, 128.0) : 1.0;
  const int64_t slabs = std::max<int64_t>(1, (int64_t)((double)K * touched) / KC);
  int64_t split = 1;
  const int64_t target = 2LL * sms;
  if (tiles > 0 && tiles < target) split = (target + tiles - 1) / tiles;
  split = std::max<int64_t>(1, std::min<int64_t>(split, std::max<int64_t>(1, slabs / 8)));
  t->m_r = m_r;
  t->n_r = NR;
  t->k_c = KC;
  t->m_c = W * m_r;
  t->split_k = (int32_t)split;
  t->dense_split_pm =
      (dt == ROSKO_BF16) ? kDenseSplitPm : (dt == ROSKO_I8 ? kDenseSplitPmI8 : 1001);
  if (dt == ROSKO_BF16 && order == 4) {
    // Small or very sparse layers: the tensor-core launch has a fixed cost
    // (set-up, the first cold loads, the epilogue) that row-direct does not.
    // Model both paths on the uniform-density assumption (every tile on one
    // side of the threshold) and keep the layer sparse when row-direct is
    // predicted faster.  Both models are least-squares fits (relative error)
    // to the 5,000 training layers of the selector's measurement sweep
    // (M, K in [64, 4096] and convolution shapes, N in [196, 12544], 50-99.9%
    // sparse, every schedule timed): dense ~10.8 us + 2 M K N at
    // ~0.58 PFLOP/s, row-direct ~5.3 us + the nnz * N BF16 values it moves
    // at ~10.9 TB/s.  On the 2,000 held-out layers picking the faster path
    // by these models costs 5% over the better of the two paths.
    const double t_dense = 10.8 + 2.0 * (double)M * (double)K * (double)N / 0.58e15 * 1e6;
    const double t_direct = 5.3 + (double)nnz * (double)N * 2.0 / 10.9e12 * 1e6;
    if (t_direct < t_dense) t->dense_split_pm = 1001;
  }
  int TN = 256, ds = 1;
  int mc = 128;
  dense_config((M + 127) / 128, N, K, sms, &TN, &ds, &mc, dt == ROSKO_I8);
  t->dense_n_r = TN;
  t->dense_split_k = ds;
  t->dense_m_c = mc;
  t->order = order;
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
  int32_t m_r = (tile && tile->m_r > 0) ? tile->m_r : 0;
  if (m_r != 0 && m_r != 8 && m_r != 16 && m_r != 32) return ROSKO_ERR_INVALID_ARG;
  if (m_r == 0) {
    // Eq. 3 analog: a warp holds m_r rows of C; 16 rows per panel make eight
    // panels per 128-row tile (the unit of the dense split and of the
    // touched-row gather) while leaving registers for wide column strips.
    m_r = 16;
  }
  const int64_t P = (M + m_r - 1) / m_r;
  if (P > 65535) return ROSKO_ERR_INVALID_ARG;
  const int32_t dense_min = (tile && tile->dense_split_pm > 0)
                                ? tile->dense_split_pm
                                : (packed_dtype == ROSKO_I8 ? kDenseCopyPmI8 : kDenseCopyPm);
  rosko_packed_s* h = nullptr;
  rosko_status s = pack_impl(A_dev, a_dtype, M, K, lda, packed_dtype, row_scale_dev, m_r,
                             dense_min, static_cast<cudaStream_t>(stream), &h);
  if (s != ROSKO_OK) return s;
  *out = h;
  return ROSKO_OK;
}

rosko_status rosko_pack_transposed(const void* A_dev, rosko_dtype a_dtype, int64_t M, int64_t K,
                                   int64_t lda, rosko_dtype packed_dtype,
                                   const float* row_scale_dev, const rosko_tile* tile,
                                   rosko_stream_t stream, rosko_packed_t* out) {
  if (!out) return ROSKO_ERR_INVALID_ARG;
  *out = nullptr;
  if (!dtype_valid(a_dtype)) return ROSKO_ERR_INVALID_ARG;
  if (M < 0 || K < 0 || lda < std::max<int64_t>(K, 1)) return ROSKO_ERR_INVALID_ARG;
  if (M * K > 0 && !A_dev) return ROSKO_ERR_INVALID_ARG;
  if (M > 0 && K > 0 && M > (int64_t)INT32_MAX / K) return ROSKO_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // dense transpose (K x M, leading dimension M) in scratch, then Alg. 1 on it
  void* t = nullptr;
  const size_t bytes = (size_t)std::max<int64_t>(M * K, 1) * dtype_size(a_dtype);
  if (pool_malloc(&t, bytes, st) != cudaSuccess) return ROSKO_ERR_OOM;
  rosko_status s = transpose_impl(A_dev, a_dtype, M, K, lda, t, st);
  if (s == ROSKO_OK)
    s = rosko_pack(t, a_dtype, K, M, std::max<int64_t>(M, 1), packed_dtype, row_scale_dev, tile,
                   stream, out);
  // stream-ordered: released after the pack's reads of the copy
  pool_free(t, st);
  return s;
}

void rosko_free(rosko_packed_t A) {
  if (!A || A->magic != kHandleMagic) return;
  A->magic = 0;
  if (A->base) {
    // queued work on any stream may still read the handle: wait for the
    // device, as cudaFree would, then hand the memory back to the pool
    int cur = 0;
    const bool other = cudaGetDevice(&cur) == cudaSuccess && cur != A->device;
    if (other) cudaSetDevice(A->device);
    cudaDeviceSynchronize();
    pool_free(A->base, nullptr);
    if (other) cudaSetDevice(cur);
  }
  delete A;
}

rosko_status rosko_pack_save(rosko_packed_t A, void* buf_host, int64_t capacity, int64_t* bytes) {
  if (!handle_ok(A)) return ROSKO_ERR_BAD_HANDLE;
  if (!bytes || (buf_host && capacity < 0)) return ROSKO_ERR_INVALID_ARG;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return ROSKO_ERR_CUDA;
  if (buf_host && cur != A->device && cudaSetDevice(A->device) != cudaSuccess) return ROSKO_ERR_CUDA;
  const rosko_status s = packed_serialize(A, buf_host, capacity, bytes);
  if (buf_host && cur != A->device) cudaSetDevice(cur);
  return s;
}

rosko_status rosko_pack_load(const void* buf_host, int64_t bytes, rosko_stream_t stream,
                             rosko_packed_t* out) {
  if (!out) return ROSKO_ERR_INVALID_ARG;
  *out = nullptr;
  if (!buf_host || bytes <= 0) return ROSKO_ERR_INVALID_ARG;
  return packed_deserialize(buf_host, bytes, static_cast<cudaStream_t>(stream), out);
}

rosko_status rosko_schedule_analytic(int64_t M, int64_t K, int64_t N, int64_t nnz, int32_t m_r,
                                     rosko_dtype packed_dtype, rosko_tile* tile) {
  if (!tile || M < 0 || K < 0 || N < 0 || nnz < 0 || !dtype_valid(packed_dtype))
    return ROSKO_ERR_INVALID_ARG;
  if (m_r > 0 && m_r != 8 && m_r != 16 && m_r != 32) return ROSKO_ERR_INVALID_ARG;
  return schedule_analytic(M, K, N, nnz, m_r, packed_dtype, 152, tile);
}

}  // extern "C"

namespace rosko {
// Host-side checks shared by every SpMM entry point.  *done is set when the
// call is complete without a launch (empty shapes, all-zero A).
rosko_status spmm_validate(rosko_packed_s* A, const void* B_dev, rosko_dtype b_dtype, int64_t N,
                           int64_t ldb, const float* col_scale_dev, void* C_dev,
                           rosko_dtype c_dtype, int64_t ldc, int accumulate, cudaStream_t st,
                           bool* done) {
  *done = false;
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
  if (A->M == 0 || N == 0) {
    *done = true;
    return ROSKO_OK;
  }
  if (!C_dev) return ROSKO_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ROSKO_ERR_CUDA;
  if (dev != A->device) return ROSKO_ERR_INVALID_ARG;
  const size_t csz = dtype_size(c_dtype);
  if (A->K == 0 || A->nnz == 0) {
    *done = true;
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
  return ROSKO_OK;
}

// Resolve the tile (fields <= 0 take the analytic rule) and launch the dense
// and sparse paths.  Arguments were validated by spmm_validate.
// Output of a plan-only run (kRunPlanOnly), per calling thread.
thread_local rosko_plan* g_plan_out = nullptr;

rosko_status spmm_run(rosko_packed_s* A, const void* B_dev, rosko_dtype b_dtype, int64_t N,
                      int64_t ldb, const float* col_scale_dev, void* C_dev, rosko_dtype c_dtype,
                      int64_t ldc, int accumulate, const rosko_tile* tile, cudaStream_t st,
                      int flags) {
  // flags: kRunSkipDense = the dense tiles were launched elsewhere (batch);
  //        kRunZeroed    = C was zeroed by the caller
  const rosko_dtype p = A->dt;
  const size_t bsz = dtype_size(b_dtype);
  const size_t csz = dtype_size(c_dtype);
  rosko_tile t{};
  const bool forced = tile && tile->mode == ROSKO_SCHED_FORCED;
  const int sms = num_sms();
  schedule_analytic(A->M, A->K, N, A->nnz, A->m_r, p, sms, &t);
  if (tile) {
    if (tile->m_r > 0 && tile->m_r != A->m_r) return ROSKO_ERR_INVALID_ARG;
    if (forced && (tile->n_r <= 0 || tile->k_c <= 0 || tile->m_c <= 0 || tile->split_k <= 0))
      return ROSKO_ERR_INVALID_ARG;
    if (tile->n_r > 0) t.n_r = tile->n_r;
    if (tile->k_c > 0) t.k_c = tile->k_c;
    if (tile->m_c > 0) t.m_c = tile->m_c;
    if (tile->split_k > 0) t.split_k = tile->split_k;
    if (tile->dense_split_pm > 0) t.dense_split_pm = tile->dense_split_pm;
    if (tile->dense_n_r > 0) t.dense_n_r = tile->dense_n_r;
    if (tile->dense_split_k > 0) t.dense_split_k = tile->dense_split_k;
    if (tile->dense_m_c > 0) t.dense_m_c = tile->dense_m_c;
    if (tile->order > 0) t.order = tile->order;
  }
  // ---- dense-panel split: a prefix of the density-sorted dense copies ----
  int64_t n_dense = 0, dense_panels = 0;
  // tensor-core tiles: BF16, or INT8 codes with an INT32 result (exact)
  const bool tc_ok = p == ROSKO_BF16 || (p == ROSKO_I8 && c_dtype == ROSKO_I32);
  if (tc_ok && A->n_copy > 0 && t.dense_split_pm <= 1000) {
    while (n_dense < A->n_copy &&
           A->tile_density[(size_t)n_dense] * 1000.0 >= (double)t.dense_split_pm) {
      dense_panels += A->tile_panels[(size_t)A->tile_order[(size_t)n_dense]];
      ++n_dense;
    }
  }
  if (n_dense > 0) {
    if (t.dense_n_r != 128 && t.dense_n_r != 256) return ROSKO_ERR_INVALID_ARG;
    if (t.dense_split_k < 1 || t.dense_split_k > 65535) return ROSKO_ERR_INVALID_ARG;
    if (t.dense_m_c != 128 && t.dense_m_c != 256) return ROSKO_ERR_INVALID_ARG;
    if (!tile || tile->dense_n_r <= 0 || tile->dense_split_k <= 0 || tile->dense_m_c <= 0) {
      int TN = 256, ds = 1, mc = 128;
      dense_config(n_dense, N, A->K, sms, &TN, &ds, &mc, p == ROSKO_I8);
      if (!tile || tile->dense_n_r <= 0) t.dense_n_r = TN;
      if (!tile || tile->dense_split_k <= 0) t.dense_split_k = ds;
      if (!tile || tile->dense_m_c <= 0) t.dense_m_c = mc;
    }
  }
  const int64_t n_sparse = A->P - dense_panels;

  SparseLaunch L;
  L.R = A->m_r;
  if (tile && tile->order > 0 && tile->n_r <= 0) {
    // order forced without a width: the default width of that order
    t.n_r = 32 * sparse_default_V(p, A->m_r, tile->order);
  }
  if (t.n_r % 32 != 0) return ROSKO_ERR_INVALID_ARG;
  L.V = t.n_r / 32;
  if (t.m_c % A->m_r != 0) return ROSKO_ERR_INVALID_ARG;
  L.W = t.m_c / A->m_r;
  L.KC = t.k_c;
  L.split = t.split_k;
  L.order = t.order;
  if (L.order < 1 || L.order > 4) return ROSKO_ERR_INVALID_ARG;
  if (L.order == 4 && !(A->rnz && sparse_config_supported(p, b_dtype, c_dtype, L.R, L.V, 4))) {
    // no row stream (K >= 65280) or no row-direct variant: column order
    if (tile && tile->order == 4) return ROSKO_ERR_UNSUPPORTED;
    L.order = 1;
    L.V = sparse_default_V(p, A->m_r, 1);
    if (t.k_c < 8) t.k_c = 32;
    L.KC = t.k_c;
  }
  if (L.order == 4) {
    // one warp per C row, B from L2: no slabs, no K split
    L.W = 1;
    L.split = 1;
    L.KC = 8;
  }
  if (L.order == 3 && (!A->gnz || A->m_r != 16)) {
    if (tile && tile->order == 3) return ROSKO_ERR_UNSUPPORTED;
    L.order = 2;
  }
  if (L.order == 2 && !A->rnz) {
    if (tile && tile->order == 2) return ROSKO_ERR_UNSUPPORTED;
    L.order = 1;
    L.V = sparse_default_V(p, A->m_r, 1);
  }
  if (L.order == 3) {
    if (tile && tile->m_c > 0 && tile->m_c != 128) return ROSKO_ERR_INVALID_ARG;
    L.W = 8;
  }
  if (L.W < 1 || L.W > 8 || L.KC < 8 || L.KC > 256 || L.KC % 8 != 0 || L.split < 1 ||
      L.split > 65535)
    return ROSKO_ERR_INVALID_ARG;
  if (L.order == 2 && !sparse_config_supported(p, b_dtype, c_dtype, L.R, L.V, 2) &&
      !(tile && tile->order == 2)) {
    // no row-slot variant for this panel height: Alg. 2's column order
    L.order = 1;
    if (!(tile && tile->n_r > 0)) L.V = sparse_default_V(p, A->m_r, 1);
  }
  if (!sparse_config_supported(p, b_dtype, c_dtype, L.R, L.V, L.order))
    return ROSKO_ERR_UNSUPPORTED;
  // B ring: up to 4 slabs, at least 2, within ~200 KB of shared memory
  const size_t stage_bytes = (size_t)L.KC * 32 * L.V * bsz;
  L.stages = (int)std::min<size_t>(4, (200 * 1024) / stage_bytes);
  if (L.order == 4) L.stages = 2;   // unused
  if (L.stages < 2) return ROSKO_ERR_INVALID_ARG;

  // one zero fill of C serves every kernel that adds partial sums atomically
  const bool skip_dense = (flags & kRunSkipDense) != 0;
  bool direct_cut = false;
  if (L.order == 4 && n_sparse > 0) {
    int64_t ns = 0;
    const int which = direct_pick(A, A->panel_order_dev, n_sparse, N, L.V);
    if (!direct_segments(A, A->panel_order_dev, n_sparse, which, &ns, &direct_cut))
      return ROSKO_ERR_UNSUPPORTED;
  }
  // (INT8 tensor-core tiles add every K chunk into C)
  const bool zero_c =
      !accumulate && ((n_sparse > 0 && (L.split > 1 || direct_cut)) ||
                      (!skip_dense && n_dense > 0 &&
                       (p == ROSKO_I8 || dense_needs_zero(n_dense, N, A->K, t.dense_n_r,
                                                          t.dense_split_k, t.dense_m_c / 128))));
  if (flags & kRunPlanOnly) {
    // report the split and the resolved schedule, launch nothing
    rosko_plan* out = g_plan_out;
    if (out) {
      out->dense_tiles = skip_dense ? 0 : n_dense;
      out->sparse_panels = n_sparse;
      out->order = n_sparse > 0 ? L.order : 0;
      out->zero_fill = zero_c ? 1 : 0;
      out->tile = t;
      out->tile.order = L.order;
      out->tile.n_r = 32 * L.V;
      out->tile.split_k = L.split;
    }
    return ROSKO_OK;
  }
  // the zero fill runs under the tensor-core launch when there is one (a
  // small kernel it depends on programmatically), else as a memset
  const bool run_dense = n_dense > 0 && !skip_dense;
  const bool fill = zero_c && !(flags & kRunZeroed);
  const ZeroFill zf{C_dev, ldc * (int64_t)csz, N * (int64_t)csz, A->M};
  if (fill && !run_dense &&
      cudaMemset2DAsync(C_dev, (size_t)ldc * csz, 0, (size_t)N * csz, (size_t)A->M, st) !=
          cudaSuccess)
    return ROSKO_ERR_CUDA;
  if (run_dense) {
    const ZeroFill* z = fill ? &zf : nullptr;
    rosko_status s =
        p == ROSKO_I8
            ? dense_spmm_i8_launch(A, n_dense, static_cast<const int8_t*>(B_dev), N, ldb,
                                   static_cast<int32_t*>(C_dev), ldc, t.dense_n_r,
                                   t.dense_split_k, t.dense_m_c / 128, z, st)
            : dense_spmm_launch(A->dense_A, A->n_copy * 128, A->Kpad, A->tile_order_dev, n_dense,
                                A->K, B_dev, N, ldb, static_cast<float*>(C_dev), ldc, A->M,
                                accumulate, t.dense_n_r, t.dense_split_k, t.dense_m_c / 128,
                                zero_c, z, st);
    if (s != ROSKO_OK) return s;
  }
  if (L.order == 3) {
    // work list of 128-row tiles: those not taken by the dense path (the
    // density-sorted tile order's tail), or every tile
    const int64_t T = (A->M + 127) / 128;
    const int32_t* list = A->tile_order_dev ? A->tile_order_dev + n_dense : nullptr;
    return sparse_spmm_launch(A, B_dev, b_dtype, N, ldb, col_scale_dev, C_dev, c_dtype, ldc,
                              accumulate, L, list, T - n_dense, zero_c, st);
  }
  return sparse_spmm_launch(A, B_dev, b_dtype, N, ldb, col_scale_dev, C_dev, c_dtype, ldc,
                            accumulate, L, A->panel_order_dev, n_sparse, zero_c, st);
}


rosko_status spmm_forced(rosko_packed_s* h, const void* B, rosko_dtype b_dt, int64_t N, int64_t ldb,
                         const float* col_scale, void* C, rosko_dtype c_dt, int64_t ldc,
                         const rosko_tile* t, cudaStream_t st) {
  return spmm_run(h, B, b_dt, N, ldb, col_scale, C, c_dt, ldc, 0, t, st, 0);
}

// Number of dense-path tiles (a prefix of the density-sorted copies) of a
// handle for a resolved threshold, and the panels they cover.
static void dense_prefix(const rosko_packed_s* A, int32_t pm, int64_t* n_dense,
                         int64_t* dense_panels) {
  *n_dense = 0;
  *dense_panels = 0;
  if (A->dt != ROSKO_BF16 || A->n_copy <= 0 || pm > 1000) return;
  while (*n_dense < A->n_copy && A->tile_density[(size_t)*n_dense] * 1000.0 >= (double)pm) {
    *dense_panels += A->tile_panels[(size_t)A->tile_order[(size_t)*n_dense]];
    ++*n_dense;
  }
}

rosko_status spmm_batched_impl(int32_t count, rosko_packed_s* const* A, const void* const* B,
                               const int64_t* N, const int64_t* ldb, void* const* C,
                               const int64_t* ldc, rosko_dtype b_dt, rosko_dtype c_dt,
                               int accumulate, const rosko_tile* tiles, cudaStream_t st) {
  const int sms = num_sms();
  std::vector<DenseJob> jobs;
  std::vector<int> job_of;        // problem index of each dense job
  std::vector<rosko_tile> rest;   // per problem: tile for the sparse remainder
  std::vector<char> active((size_t)count, 0), dense_any((size_t)count, 0);
  std::vector<char> direct_cut((size_t)count, 0);
  rest.resize((size_t)count);
  // dense tiles run in one launch per CTA-tile shape (TN x 128 MH): each
  // problem takes the shape the analytic rule (or its tile) gives it
  std::vector<int> job_tn, job_mh;
  for (int32_t i = 0; i < count; ++i) {
    bool done = false;
    rosko_status v = spmm_validate(A[i], B[i], b_dt, N[i], ldb[i], nullptr, C[i], c_dt, ldc[i],
                                   accumulate, st, &done);
    if (v != ROSKO_OK) return v;
    if (done) continue;
    active[(size_t)i] = 1;
    rosko_tile t{};
    schedule_analytic(A[i]->M, A[i]->K, N[i], A[i]->nnz, A[i]->m_r, A[i]->dt, sms, &t);
    if (tiles) {
      const rosko_tile& u = tiles[i];
      if (u.dense_split_pm > 0) t.dense_split_pm = u.dense_split_pm;
    }
    // the batch's tensor-core launches are BF16 only: other packs run sparse
    if (A[i]->dt != ROSKO_BF16) t.dense_split_pm = 1001;
    int64_t nd = 0, dp = 0;
    dense_prefix(A[i], t.dense_split_pm, &nd, &dp);
    if (nd > 0) {
      if (b_dt != ROSKO_BF16 || c_dt != ROSKO_F32) return ROSKO_ERR_UNSUPPORTED;
      DenseJob j;
      j.dense_A = A[i]->dense_A;
      j.dense_rows = A[i]->n_copy * 128;
      j.Kpad = A[i]->Kpad;
      j.tile_order_dev = A[i]->tile_order_dev;
      j.n_tiles = nd;
      j.K = A[i]->K;
      j.B = B[i];
      j.N = N[i];
      j.ldb = ldb[i];
      j.C = static_cast<float*>(C[i]);
      j.ldc = ldc[i];
      j.M = A[i]->M;
      j.accumulate = accumulate;
      int tn = 256, ds = 1, mc = 128;
      dense_config(nd, N[i], A[i]->K, sms, &tn, &ds, &mc, false);
      if (tiles && tiles[i].dense_n_r > 0) tn = tiles[i].dense_n_r;
      if (tiles && tiles[i].dense_m_c > 0) mc = tiles[i].dense_m_c;
      if ((tn != 128 && tn != 256) || (mc != 128 && mc != 256)) return ROSKO_ERR_INVALID_ARG;
      jobs.push_back(j);
      job_of.push_back(i);
      job_tn.push_back(tn);
      job_mh.push_back(mc / 128);
      dense_any[(size_t)i] = 1;
    }
    // the sparse remainder keeps this problem's tile; spmm_run recomputes the
    // same dense prefix from the same threshold and skips launching it
    rosko_tile r = tiles ? tiles[i] : t;
    r.dense_split_pm = t.dense_split_pm;
    if (r.split_k <= 0) r.split_k = t.split_k;
    if ((r.order > 0 ? r.order : t.order) == 4) {
      r.split_k = 1;   // row-direct: no K split, but cut rows add into C
      int64_t ns = 0;
      bool cut = false;
      const int V = r.n_r > 0 ? r.n_r / 32 : sparse_default_V(A[i]->dt, A[i]->m_r, 4);
      const int which = direct_pick(A[i], A[i]->panel_order_dev, A[i]->P - dp, N[i], V);
      if (A[i]->rnz &&
          direct_segments(A[i], A[i]->panel_order_dev, A[i]->P - dp, which, &ns, &cut) && cut)
        direct_cut[(size_t)i] = 1;
    }
    rest[(size_t)i] = r;
    // whole-dense problems need no sparse launch
    if (dp == A[i]->P) rest[(size_t)i].m_r = -1;
  }
  // zero every C that some kernel adds into: dense tiles cut by the stream-K
  // split, or a sparse remainder split along K (before any launch)
  std::vector<char> zeroed((size_t)count, 0);
  if (!accumulate) {
    std::vector<char> need((size_t)count, 0);
    for (int g = 0; g < 4; ++g) {
      const int tn = (g & 1) ? 256 : 128, mh = (g & 2) ? 2 : 1;
      std::vector<DenseJob> gj;
      std::vector<int> gi;
      for (size_t k = 0; k < jobs.size(); ++k)
        if (job_tn[k] == tn && job_mh[k] == mh) {
          gj.push_back(jobs[k]);
          gi.push_back(job_of[k]);
        }
      if (gj.empty()) continue;
      std::unique_ptr<bool[]> nj(new bool[gj.size()]);
      dense_batch_needs_zero(gj.data(), (int)gj.size(), tn, sms, mh, nj.get());
      for (size_t k = 0; k < gj.size(); ++k)
        if (nj[k]) need[(size_t)gi[k]] = 1;
    }
    for (int32_t i = 0; i < count; ++i) {
      if (!active[(size_t)i]) continue;
      if (rest[(size_t)i].m_r != -1 && (rest[(size_t)i].split_k > 1 || direct_cut[(size_t)i]))
        need[(size_t)i] = 1;
      if (!need[(size_t)i]) continue;
      const size_t csz = dtype_size(c_dt);
      if (cudaMemset2DAsync(C[i], (size_t)ldc[i] * csz, 0, (size_t)N[i] * csz, (size_t)A[i]->M,
                            st) != cudaSuccess)
        return ROSKO_ERR_CUDA;
      zeroed[(size_t)i] = 1;
    }
  }
  for (int g = 0; g < 4; ++g) {
    const int tn = (g & 1) ? 256 : 128, mh = (g & 2) ? 2 : 1;
    std::vector<DenseJob> gj;
    for (size_t k = 0; k < jobs.size(); ++k)
      if (job_tn[k] == tn && job_mh[k] == mh) gj.push_back(jobs[k]);
    if (gj.empty()) continue;
    rosko_status s = dense_batch_launch(gj.data(), (int)gj.size(), tn, sms, mh, st);
    if (s != ROSKO_OK) return s;
  }
  // sparse remainders (the dense tiles were launched above): the row-direct
  // ones (order 4, one V) share one launch, the others run one per problem
  std::vector<DirectJob> direct;
  std::vector<char> in_direct((size_t)count, 0);
  int direct_V = 0;
  for (int32_t i = 0; i < count; ++i) {
    if (!active[(size_t)i] || rest[(size_t)i].m_r == -1) continue;
    const rosko_tile& r = rest[(size_t)i];
    rosko_tile t{};
    schedule_analytic(A[i]->M, A[i]->K, N[i], A[i]->nnz, A[i]->m_r, A[i]->dt, sms, &t);
    const int ord = r.order > 0 ? r.order : t.order;
    if (ord != 4 || !A[i]->rnz) continue;
    const int V = r.n_r > 0 ? r.n_r / 32 : sparse_default_V(A[i]->dt, A[i]->m_r, 4);
    if (!sparse_config_supported(A[i]->dt, b_dt, c_dt, A[i]->m_r, V, 4)) continue;
    if (direct_V != 0 && V != direct_V) continue;
    int64_t nd = 0, dp = 0;
    dense_prefix(A[i], r.dense_split_pm, &nd, &dp);
    DirectJob j{A[i], B[i], b_dt, N[i], ldb[i], nullptr, C[i], c_dt, ldc[i], accumulate,
                A[i]->panel_order_dev, A[i]->P - dp};
    direct.push_back(j);
    direct_V = V;
    in_direct[(size_t)i] = 1;
  }
  if (!direct.empty()) {
    rosko_status s = direct_batch_launch(direct.data(), (int)direct.size(), direct_V, st);
    if (s != ROSKO_OK) return s;
  }
  for (int32_t i = 0; i < count; ++i) {
    if (!active[(size_t)i] || rest[(size_t)i].m_r == -1 || in_direct[(size_t)i]) continue;
    rosko_tile r = rest[(size_t)i];
    r.m_r = 0;
    const int flags = kRunSkipDense | (zeroed[(size_t)i] ? kRunZeroed : 0);
    rosko_status s = spmm_run(A[i], B[i], b_dt, N[i], ldb[i], nullptr, C[i], c_dt, ldc[i],
                              accumulate, &r, st, flags);
    if (s != ROSKO_OK) return s;
  }
  return ROSKO_OK;
}
}  // namespace rosko

extern "C" {

static rosko_status spmm_dispatch(rosko_packed_t A, const void* B_dev, rosko_dtype b_dtype,
                                  int64_t N, int64_t ldb, const float* col_scale_dev, void* C_dev,
                                  rosko_dtype c_dtype, int64_t ldc, int accumulate,
                                  const rosko_tile* tile, rosko_stream_t stream, int flags) {
  bool done = false;
  rosko_status v = spmm_validate(A, B_dev, b_dtype, N, ldb, col_scale_dev, C_dev, c_dtype, ldc,
                                 accumulate, static_cast<cudaStream_t>(stream), &done);
  if (v != ROSKO_OK || done) return v;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int mode = tile ? tile->mode : ROSKO_SCHED_ANALYTIC;
  if (mode == ROSKO_SCHED_AUTOTUNE || mode == ROSKO_SCHED_LEARNED) {
    rosko_tile chosen{};
    bool have = false;
    {
      std::lock_guard<std::mutex> lk(A->mu);
      auto it = A->sched_cache.find(N * 4 + mode);
      if (it != A->sched_cache.end()) {
        chosen = it->second;
        have = true;
      }
    }
    if (!have && mode == ROSKO_SCHED_AUTOTUNE && !accumulate) {
      // the search writes C, which this call overwrites anyway
      rosko_status s = autotune_impl(A, B_dev, b_dtype, N, ldb, col_scale_dev, C_dev, c_dtype,
                                     ldc, 3, &chosen, nullptr, nullptr, st);
      if (s != ROSKO_OK) return s;
      have = true;
    }
    if (!have && mode == ROSKO_SCHED_LEARNED) {
      rosko_status s = select_learned(A, N, &chosen, st);
      if (s == ROSKO_OK) {
        have = true;
      } else if (s == ROSKO_ERR_UNSUPPORTED) {
        // no network, or features outside its training range: the analytic
        // rule, remembered like a learned choice (later calls, e.g. under
        // stream capture, neither recompute the features nor allocate)
        std::memset(&chosen, 0, sizeof(chosen));
        chosen.mode = ROSKO_SCHED_ANALYTIC;
        have = true;
      } else {
        return s;
      }
    }
    if (have) {
      {
        std::lock_guard<std::mutex> lk(A->mu);
        A->sched_cache[N * 4 + mode] = chosen;
      }
      return spmm_run(A, B_dev, b_dtype, N, ldb, col_scale_dev, C_dev, c_dtype, ldc, accumulate,
                      chosen.mode == ROSKO_SCHED_ANALYTIC ? nullptr : &chosen, st, flags);
    }
    // no cached choice and none can be made here: the analytic rule
    return spmm_run(A, B_dev, b_dtype, N, ldb, col_scale_dev, C_dev, c_dtype, ldc, accumulate,
                    nullptr, st, flags);
  }
  return spmm_run(A, B_dev, b_dtype, N, ldb, col_scale_dev, C_dev, c_dtype, ldc, accumulate, tile,
                  st, flags);
}

rosko_status rosko_spmm(rosko_packed_t A, const void* B_dev, rosko_dtype b_dtype, int64_t N,
                        int64_t ldb, const float* col_scale_dev, void* C_dev,
                        rosko_dtype c_dtype, int64_t ldc, int accumulate,
                        const rosko_tile* tile, rosko_stream_t stream) {
  return spmm_dispatch(A, B_dev, b_dtype, N, ldb, col_scale_dev, C_dev, c_dtype, ldc, accumulate,
                       tile, stream, 0);
}

rosko_status rosko_spmm_plan(rosko_packed_t A, const void* B_dev, rosko_dtype b_dtype, int64_t N,
                             int64_t ldb, const float* col_scale_dev, void* C_dev,
                             rosko_dtype c_dtype, int64_t ldc, int accumulate,
                             const rosko_tile* tile, rosko_plan* out, rosko_stream_t stream) {
  if (!out) return ROSKO_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  g_plan_out = out;
  const rosko_status s = spmm_dispatch(A, B_dev, b_dtype, N, ldb, col_scale_dev, C_dev, c_dtype,
                                       ldc, accumulate, tile, stream, kRunPlanOnly);
  g_plan_out = nullptr;
  return s;
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
  // device-format bytes the SpMM reads: nonzero records, column records and
  // panel offsets
  if (bytes)
    *bytes = A->nnz * (int64_t)rec_size(A->dt) + (A->n_cols + 1) * 8 + (A->P + 1) * 4;
  if (touched_k) *touched_k = A->touched_k;
  if (n_panels) *n_panels = A->P;
  if (m_r) *m_r = A->m_r;
  if (packed_dtype) *packed_dtype = (int32_t)A->dt;
  if (n_cols) *n_cols = A->n_cols;
  return ROSKO_OK;
}

rosko_status rosko_packed_shape(rosko_packed_t A, int64_t* M, int64_t* K, int64_t* device_bytes) {
  if (!handle_ok(A)) return ROSKO_ERR_BAD_HANDLE;
  if (M) *M = A->M;
  if (K) *K = A->K;
  if (device_bytes) *device_bytes = (int64_t)A->base_bytes;
  return ROSKO_OK;
}

rosko_status rosko_packed_export(rosko_packed_t A, void* A_p_host, uint8_t* loc_m_host,
                                 int32_t* col_ind_host, int32_t* nnz_host,
                                 int64_t* panel_cols_host) {
  if (!handle_ok(A)) return ROSKO_ERR_BAD_HANDLE;
  const size_t esz = dtype_size(A->dt);
  const size_t rsz = rec_size(A->dt);
  if (cudaDeviceSynchronize() != cudaSuccess) return ROSKO_ERR_CUDA;
  std::vector<unsigned char> recs((size_t)A->nnz * rsz);
  std::vector<int2> cr((size_t)A->n_cols + 1);
  if (A->nnz && cudaMemcpy(recs.data(), A->nz, recs.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
    return ROSKO_ERR_CUDA;
  if (cudaMemcpy(cr.data(), A->colrec, cr.size() * sizeof(int2), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return ROSKO_ERR_CUDA;
  // decode the interleaved records into the canonical Alg. 1 arrays
  for (int64_t e = 0; e < A->nnz; ++e) {
    const unsigned char* w = recs.data() + (size_t)e * rsz;
    uint32_t row = 0;
    if (A->dt == ROSKO_F32) {
      std::memcpy(&row, w, 4);
      if (A_p_host) std::memcpy(static_cast<char*>(A_p_host) + e * esz, w + 4, 4);
    } else if (A->dt == ROSKO_F64) {
      std::memcpy(&row, w + 8, 4);
      if (A_p_host) std::memcpy(static_cast<char*>(A_p_host) + e * esz, w, 8);
    } else {
      uint32_t v;
      std::memcpy(&v, w, 4);
      row = v & 0xFFFFu;
      if (A_p_host) {
        if (A->dt == ROSKO_BF16) {
          const uint16_t b = (uint16_t)(v >> 16);
          std::memcpy(static_cast<char*>(A_p_host) + e * 2, &b, 2);
        } else {
          const int8_t q = (int8_t)(uint8_t)(v >> 16);
          static_cast<int8_t*>(A_p_host)[e] = q;
        }
      }
    }
    if (loc_m_host) loc_m_host[e] = (uint8_t)row;
  }
  for (int64_t c = 0; c < A->n_cols; ++c) {
    if (col_ind_host) col_ind_host[c] = cr[(size_t)c].x;
    if (nnz_host) nnz_host[c] = cr[(size_t)c + 1].y - cr[(size_t)c].y;
  }
  if (panel_cols_host) {
    std::vector<int32_t> pc((size_t)A->P + 1);
    if (cudaMemcpy(pc.data(), A->panel_col, pc.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return ROSKO_ERR_CUDA;
    for (int64_t i = 0; i <= A->P; ++i) panel_cols_host[i] = pc[i];
  }
  return ROSKO_OK;
}

rosko_status rosko_spmm_batched(int32_t count, const rosko_packed_t* A, const void* const* B,
                                const int64_t* N, const int64_t* ldb, void* const* C,
                                const int64_t* ldc, rosko_dtype b_dtype, rosko_dtype c_dtype,
                                int accumulate, const rosko_tile* tiles, rosko_stream_t stream) {
  if (count < 0 || count > 64) return ROSKO_ERR_INVALID_ARG;
  if (count == 0) return ROSKO_OK;
  if (!A || !B || !N || !ldb || !C || !ldc) return ROSKO_ERR_INVALID_ARG;
  return spmm_batched_impl(count, A, B, N, ldb, C, ldc, b_dtype, c_dtype, accumulate, tiles,
                           static_cast<cudaStream_t>(stream));
}

int32_t rosko_num_candidates(void) { return (int32_t)num_candidates(); }

rosko_status rosko_candidate(rosko_packed_t A, int64_t N, int32_t index, rosko_tile* out) {
  if (!handle_ok(A)) return ROSKO_ERR_BAD_HANDLE;
  if (!out || N < 0 || index < 0 || index >= num_candidates()) return ROSKO_ERR_INVALID_ARG;
  return candidate_tile(A, N, index, out) ? ROSKO_OK : ROSKO_ERR_UNSUPPORTED;
}

rosko_status rosko_autotune(rosko_packed_t A, const void* B_dev, rosko_dtype b_dtype, int64_t N,
                            int64_t ldb, const float* col_scale_dev, void* C_dev,
                            rosko_dtype c_dtype, int64_t ldc, int32_t reps, rosko_tile* best,
                            float* times_ms, rosko_stream_t stream) {
  if (!best) return ROSKO_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bool done = false;
  rosko_status v = spmm_validate(A, B_dev, b_dtype, N, ldb, col_scale_dev, C_dev, c_dtype, ldc, 0,
                                 st, &done);
  if (v != ROSKO_OK) return v;
  if (done) {
    schedule_analytic(A->M, A->K, N, A->nnz, A->m_r, A->dt, num_sms(), best);
    return ROSKO_OK;
  }
  rosko_status s = autotune_impl(A, B_dev, b_dtype, N, ldb, col_scale_dev, C_dev, c_dtype, ldc,
                                 reps, best, times_ms, nullptr, st);
  if (s != ROSKO_OK) return s;
  std::lock_guard<std::mutex> lk(A->mu);
  A->sched_cache[N * 4 + ROSKO_SCHED_AUTOTUNE] = *best;
  return ROSKO_OK;
}

rosko_status rosko_time_tile(rosko_packed_t A, const void* B_dev, rosko_dtype b_dtype, int64_t N,
                             int64_t ldb, const float* col_scale_dev, void* C_dev,
                             rosko_dtype c_dtype, int64_t ldc, const rosko_tile* tile,
                             int32_t reps, float* ms, rosko_stream_t stream) {
  if (!ms) return ROSKO_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bool done = false;
  rosko_status v = spmm_validate(A, B_dev, b_dtype, N, ldb, col_scale_dev, C_dev, c_dtype, ldc, 0,
                                 st, &done);
  if (v != ROSKO_OK) return v;
  if (done) {
    *ms = 0.0f;
    return ROSKO_OK;
  }
  rosko_status err = ROSKO_OK;
  *ms = time_tile(A, B_dev, b_dtype, N, ldb, col_scale_dev, C_dev, c_dtype, ldc, tile, reps, st,
                  &err);
  return err;
}

int32_t rosko_candidate_index(const rosko_tile* tile, rosko_dtype packed_dtype) {
  if (!tile || !dtype_valid(packed_dtype) || tile->m_r <= 0) return -1;
  return candidate_index(tile, packed_dtype);
}

rosko_status rosko_features(rosko_packed_t A, int64_t N, double* features16,
                            rosko_stream_t stream) {
  if (!handle_ok(A)) return ROSKO_ERR_BAD_HANDLE;
  if (!features16 || N < 1) return ROSKO_ERR_INVALID_ARG;
  // the feature kernels read the handle's arrays: only on its own device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ROSKO_ERR_CUDA;
  if (dev != A->device) return ROSKO_ERR_INVALID_ARG;
  return features_impl(A, N, features16, static_cast<cudaStream_t>(stream));
}

rosko_status rosko_features_static(rosko_packed_t A, int64_t N, float* features16_dev,
                                   rosko_stream_t stream) {
  if (!handle_ok(A)) return ROSKO_ERR_BAD_HANDLE;
  if (!features16_dev || N < 1 || reinterpret_cast<uintptr_t>(features16_dev) % 4 != 0)
    return ROSKO_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ROSKO_ERR_CUDA;
  if (dev != A->device) return ROSKO_ERR_INVALID_ARG;
  return features_static_impl(A, N, features16_dev, static_cast<cudaStream_t>(stream));
}

int64_t rosko_mlp_param_count(int32_t n_in, int32_t n_out) {
  if (n_in < 1 || n_out < 1) return 0;
  return mlp_param_count(n_in, n_out);
}

int64_t rosko_mlp_workspace_floats(int64_t batch, int32_t n_out) {
  if (batch < 1 || n_out < 1) return 0;
  return mlp_workspace_floats(batch, n_out);
}

rosko_status rosko_mlp_forward(const float* params_dev, const float* X_dev, int64_t batch,
                               int32_t n_in, int32_t n_out, float* acts_dev, float* logits_dev,
                               rosko_stream_t stream) {
  if (!params_dev || !X_dev || !acts_dev || !logits_dev || batch < 1 || n_in < 1 || n_out < 1)
    return ROSKO_ERR_INVALID_ARG;
  return mlp_forward(params_dev, X_dev, batch, n_in, n_out, acts_dev, logits_dev,
                     static_cast<cudaStream_t>(stream));
}

rosko_status rosko_mlp_loss_grad(const float* params_dev, const float* X_dev, const float* Y_dev,
                                 int64_t batch, int32_t n_in, int32_t n_out, float* grads_dev,
                                 float* loss_dev, float* workspace_dev, rosko_stream_t stream) {
  if (!params_dev || !X_dev || !Y_dev || !grads_dev || !loss_dev || !workspace_dev ||
      batch < 1 || n_in < 1 || n_out < 1)
    return ROSKO_ERR_INVALID_ARG;
  return mlp_loss_grad(params_dev, X_dev, Y_dev, batch, n_in, n_out, grads_dev, loss_dev,
                       workspace_dev, static_cast<cudaStream_t>(stream));
}

rosko_status rosko_mlp_adam(float* params_dev, const float* grads_dev, float* m_dev, float* v_dev,
                            int64_t n, int32_t step, float lr, float beta1, float beta2,
                            float eps, float weight_decay, rosko_stream_t stream) {
  if (!params_dev || !grads_dev || !m_dev || !v_dev || n < 1 || step < 1 || !(weight_decay >= 0))
    return ROSKO_ERR_INVALID_ARG;
  return mlp_adam(params_dev, grads_dev, m_dev, v_dev, n, step, lr, beta1, beta2, eps,
                  weight_decay, static_cast<cudaStream_t>(stream));
}

rosko_status rosko_selector_set(const float* params_host, int64_t n_params, const double* mean16,
                                const double* std16, const double* lo16, const double* hi16) {
  if (!params_host || !mean16 || !std16 || !lo16 || !hi16) return ROSKO_ERR_INVALID_ARG;
  return selector_set(params_host, (int)n_params, num_candidates(), mean16, std16, lo16, hi16);
}

int64_t rosko_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

rosko_status rosko_set_wait_limit(int64_t ns) {
  if (ns < 0) return ROSKO_ERR_INVALID_ARG;
  int* w = device_status_word();
  if (!w) return ROSKO_ERR_CUDA;
  const unsigned long long v = (unsigned long long)ns;
  return cudaMemcpy(reinterpret_cast<char*>(w) + kWaitLimitOffset, &v, sizeof(v),
                    cudaMemcpyHostToDevice) == cudaSuccess
             ? ROSKO_OK
             : ROSKO_ERR_CUDA;
}

rosko_status rosko_probe_bounded_wait(rosko_stream_t stream) {
  int* w = device_status_word();
  if (!w) return ROSKO_ERR_CUDA;
  probe_wait_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(w);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
}

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
