// Device packer: Alg. 1 (Sec. 4.1) applied to every row panel of A.
//
// Alg. 1 walks a tile column by column and, within a column, row by row,
// appending each nonzero to A_p / loc_m and, for a non-empty column, its
// index to col_ind and its count to nnz.  On the GPU the per-(panel, column)
// counts are independent, so the walk becomes three passes:
//   1. count   one thread per (panel, column): nonzeros of that panel column
//   2. scan    exclusive prefix sums of (count, count != 0) in panel-major,
//              column-ascending order = Alg. 1's append order
//   3. scatter one thread per (panel, column): writes its column record and
//              its values/rows (rows ascending) at the scanned offsets
// Threads of a warp own consecutive columns, so every read of A is a
// coalesced row segment.  The packer is bound by reading A (twice: count and
// scatter) and writing the packed stream.
#include <algorithm>
#include <cstring>
#include <new>

#include "handle.hpp"

namespace rosko {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// ----------------------------------------------------------------------------
// Value test and conversion per (source, packed) type pair.
template <class S, class D> struct Conv;
template <> struct Conv<float, float> {
  __device__ static bool get(float a, float, float& out) { out = a; return a != 0.0f; }
};
template <> struct Conv<float, __nv_bfloat16> {
  // The mask is taken from the FP32 value; a value that rounds to 0 stays packed.
  __device__ static bool get(float a, float, __nv_bfloat16& out) {
    out = __float2bfloat16_rn(a);
    return a != 0.0f;
  }
};
template <> struct Conv<float, double> {
  __device__ static bool get(float a, float, double& out) { out = (double)a; return a != 0.0f; }
};
template <> struct Conv<float, int8_t> {
  // Symmetric per-row code q = clamp(rint(a / s), -127, 127); the mask is q != 0.
  __device__ static bool get(float a, float s, int8_t& out) {
    float q = rintf(__fdiv_rn(a, s));
    q = fminf(fmaxf(q, -127.0f), 127.0f);
    out = (int8_t)(int)q;
    return out != 0;
  }
};
template <> struct Conv<__nv_bfloat16, __nv_bfloat16> {
  __device__ static bool get(__nv_bfloat16 a, float, __nv_bfloat16& out) {
    out = a;
    return __bfloat162float(a) != 0.0f;
  }
};
template <> struct Conv<int8_t, int8_t> {
  __device__ static bool get(int8_t a, float, int8_t& out) { out = a; return a != 0; }
};

// Per-row symmetric INT8 scale s_i = max_k |a_ik| / 127 (1 for an all-zero row).
__global__ void rowscale_kernel(const float* __restrict__ A, int64_t M, int64_t K, int64_t lda,
                                float* __restrict__ scale) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= M) return;
  float m = 0.0f;
  for (int64_t k = lane; k < K; k += 32) m = fmaxf(m, fabsf(A[row * lda + k]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) scale[row] = (m == 0.0f) ? 1.0f : __fdiv_rn(m, 127.0f);
}

// Pass 1: cnt[p*K + k] = (nonzeros of column k in panel p, 1 if non-empty).
template <class S, class D>
__global__ void count_kernel(const S* __restrict__ A, int64_t M, int64_t K, int64_t lda, int m_r,
                             const float* __restrict__ scale, int2* __restrict__ cnt,
                             int* __restrict__ touched) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t p = blockIdx.y;
  if (k >= K) return;
  const int64_t m0 = p * m_r;
  const int64_t m1 = min(M, m0 + m_r);
  int c = 0;
  for (int64_t m = m0; m < m1; ++m) {
    D v;
    c += Conv<S, D>::get(A[m * lda + k], scale ? scale[m] : 1.0f, v) ? 1 : 0;
  }
  cnt[p * K + k] = make_int2(c, c != 0);
  if (c) touched[k] = 1;
}

__device__ __forceinline__ int2 add2(int2 a, int2 b) { return make_int2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ int2 warp_incl_scan(int2 v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int2 t;
    t.x = __shfl_up_sync(0xffffffffu, v.x, o);
    t.y = __shfl_up_sync(0xffffffffu, v.y, o);
    if (lane >= o) v = add2(v, t);
  }
  return v;
}

// Exclusive block scan of one int2 per thread; returns the block total in *total.
__device__ int2 block_excl_scan(int2 v, int2* total) {
  __shared__ int2 warp_sums[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int2 inc = warp_incl_scan(v);
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int2 w = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : make_int2(0, 0);
    w = warp_incl_scan(w);
    warp_sums[lane] = w;
  }
  __syncthreads();
  int2 base = warp ? warp_sums[warp - 1] : make_int2(0, 0);
  *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return make_int2(base.x + inc.x - v.x, base.y + inc.y - v.y);
}

// Scan pass A: per-tile sums.
__global__ void scan_reduce_kernel(const int2* __restrict__ in, int64_t n, int2* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int2 s = make_int2(0, 0);
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
    if (idx < n) s = add2(s, in[idx]);
  }
  int2 total;
  block_excl_scan(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Scan pass B: exclusive scan of the tile sums (one block, chunked), writes the
// grand total to sums[nb].
__global__ void scan_spine_kernel(int2* __restrict__ sums, int64_t nb) {
  int2 carry = make_int2(0, 0);
  for (int64_t c0 = 0; c0 < nb; c0 += kScanThreads) {
    const int64_t idx = c0 + threadIdx.x;
    int2 v = idx < nb ? sums[idx] : make_int2(0, 0);
    int2 total;
    int2 ex = block_excl_scan(v, &total);
    if (idx < nb) sums[idx] = add2(ex, carry);
    carry = add2(carry, total);
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

// Scan pass C: in-place exclusive scan of each tile with its offset; the
// element n receives the grand total.
__global__ void scan_down_kernel(int2* __restrict__ data, int64_t n, const int2* __restrict__ sums,
                                 int64_t nb) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int2 v[kScanItems];
  int2 s = make_int2(0, 0);
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? data[base + i] : make_int2(0, 0);
    s = add2(s, v[i]);
  }
  int2 total;
  int2 off = add2(block_excl_scan(s, &total), sums[blockIdx.x]);
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) data[base + i] = off;
    off = add2(off, v[i]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) data[n] = sums[nb];
}

__global__ void sum_flags_kernel(const int* __restrict__ f, int64_t n, int* __restrict__ out) {
  int s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += f[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// Pass 3: column records and values.  off[p*K+k] = (first nonzero, first
// packed column) of that panel column; the count is the difference with the
// next entry.
template <class S, class D>
__global__ void scatter_kernel(const S* __restrict__ A, int64_t M, int64_t K, int64_t lda, int m_r,
                               const float* __restrict__ scale, const int2* __restrict__ off,
                               int32_t* __restrict__ col_ind, int32_t* __restrict__ col_start,
                               D* __restrict__ vals, uint8_t* __restrict__ rows,
                               int32_t* __restrict__ panel_col, int64_t* __restrict__ panel_nnz) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t p = blockIdx.y;
  if (k >= K) return;
  const int64_t pk = p * K + k;
  const int2 o = off[pk];
  if (k == 0) {
    panel_col[p] = o.y;
    panel_nnz[p] = o.x;
  }
  const int cnt = off[pk + 1].x - o.x;
  if (cnt == 0) return;
  col_ind[o.y] = (int32_t)k;
  col_start[o.y] = o.x;
  const int64_t m0 = p * m_r;
  const int64_t m1 = min(M, m0 + m_r);
  int64_t e = o.x;
  for (int64_t m = m0; m < m1; ++m) {
    D v;
    if (Conv<S, D>::get(A[m * lda + k], scale ? scale[m] : 1.0f, v)) {
      vals[e] = v;
      rows[e] = (uint8_t)(m - m0);
      ++e;
    }
  }
}

template <class D>
__global__ void unpack_kernel(const int32_t* __restrict__ panel_col,
                              const int32_t* __restrict__ col_ind,
                              const int32_t* __restrict__ col_start, const D* __restrict__ vals,
                              const uint8_t* __restrict__ rows, int m_r, int64_t lda,
                              D* __restrict__ out) {
  const int64_t p = blockIdx.x;
  for (int64_t c = panel_col[p] + threadIdx.x; c < panel_col[p + 1]; c += blockDim.x) {
    const int64_t k = col_ind[c];
    for (int32_t e = col_start[c]; e < col_start[c + 1]; ++e)
      out[(p * m_r + rows[e]) * lda + k] = vals[e];
  }
}

struct Scratch {
  void* p = nullptr;
  ~Scratch() {
    if (p) cudaFree(p);
  }
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <class S, class D>
rosko_status pack_typed(const S* A, int64_t M, int64_t K, int64_t lda, const float* scale_in,
                        bool quantize_rows, rosko_packed_s* h, cudaStream_t st) {
  const int64_t P = h->P;
  const int64_t n = P * K;
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  // scratch: cnt/off (n+1 int2), tile sums (nb+1 int2), touched flags (K int),
  // three ints of totals
  const size_t off_cnt = 0;
  const size_t off_sums = align_up(off_cnt + (size_t)(n + 1) * sizeof(int2), 256);
  const size_t off_touch = align_up(off_sums + (size_t)(nb + 1) * sizeof(int2), 256);
  const size_t off_tot = align_up(off_touch + (size_t)K * sizeof(int), 256);
  const size_t scratch_bytes = off_tot + 256;
  Scratch scr;
  if (dev_malloc(&scr.p, scratch_bytes) != cudaSuccess) return ROSKO_ERR_OOM;
  char* sb = static_cast<char*>(scr.p);
  int2* cnt = reinterpret_cast<int2*>(sb + off_cnt);
  int2* sums = reinterpret_cast<int2*>(sb + off_sums);
  int* touched = reinterpret_cast<int*>(sb + off_touch);
  int* tot = reinterpret_cast<int*>(sb + off_tot);

  // meta allocation: panel_col (P+1 int32), panel_nnz (P+1 int64), row_scale (M),
  // features
  const size_t m_pc = 0;
  const size_t m_pn = align_up(m_pc + (size_t)(P + 1) * 4, 256);
  const size_t m_rs = align_up(m_pn + (size_t)(P + 1) * 8, 256);
  const size_t m_ft = align_up(m_rs + (size_t)std::max<int64_t>(M, 1) * 4, 256);
  const size_t meta_bytes = m_ft + 256;
  if (dev_malloc(&h->meta_base, meta_bytes) != cudaSuccess) return ROSKO_ERR_OOM;
  char* mb = static_cast<char*>(h->meta_base);
  h->panel_col = reinterpret_cast<int32_t*>(mb + m_pc);
  h->panel_nnz_dev = reinterpret_cast<int64_t*>(mb + m_pn);
  h->row_scale = reinterpret_cast<float*>(mb + m_rs);
  h->feat_dev = reinterpret_cast<float*>(mb + m_ft);

  if (cudaMemsetAsync(touched, 0, (size_t)K * sizeof(int) + 0, st) != cudaSuccess ||
      cudaMemsetAsync(tot, 0, 16, st) != cudaSuccess)
    return ROSKO_ERR_CUDA;

  const float* scale = nullptr;
  if (quantize_rows) {
    const int wpb = 8;
    if (M > 0)
      rowscale_kernel<<<(unsigned)((M + wpb - 1) / wpb), wpb * 32, 0, st>>>(
          reinterpret_cast<const float*>(A), M, K, lda, h->row_scale);
    if (M > 0) count_launches(1);
    scale = h->row_scale;
  } else if (h->dt == ROSKO_I8) {
    if (scale_in) {
      if (cudaMemcpyAsync(h->row_scale, scale_in, (size_t)M * 4, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess)
        return ROSKO_ERR_CUDA;
    } else {
      // all-ones scales: write with a trivial fill through memset of 0x3f800000
      // is not byte-uniform, so use a host copy of ones
      float* ones = new (std::nothrow) float[M > 0 ? M : 1];
      if (!ones) return ROSKO_ERR_OOM;
      for (int64_t i = 0; i < M; ++i) ones[i] = 1.0f;
      cudaError_t e = cudaMemcpyAsync(h->row_scale, ones, (size_t)M * 4, cudaMemcpyHostToDevice, st);
      cudaError_t e2 = cudaStreamSynchronize(st);
      delete[] ones;
      if (e != cudaSuccess || e2 != cudaSuccess) return ROSKO_ERR_CUDA;
    }
  }

  const int T = 256;
  const dim3 grid((unsigned)((K + T - 1) / T), (unsigned)P);
  if (n > 0) {
    count_kernel<S, D><<<grid, T, 0, st>>>(A, M, K, lda, h->m_r, scale, cnt, touched);
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(cnt, n, sums);
    scan_spine_kernel<<<1, kScanThreads, 0, st>>>(sums, nb);
    scan_down_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(cnt, n, sums, nb);
    sum_flags_kernel<<<std::min<int64_t>((K + 255) / 256, 1024), 256, 0, st>>>(touched, K, tot + 2);
    count_launches(5);
  } else {
    if (cudaMemsetAsync(cnt, 0, sizeof(int2), st) != cudaSuccess) return ROSKO_ERR_CUDA;
  }
  if (cudaGetLastError() != cudaSuccess) return ROSKO_ERR_CUDA;
  int host_tot[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(host_tot, cnt + n, sizeof(int2), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(host_tot + 2, tot + 2, sizeof(int), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ROSKO_ERR_CUDA;
  h->nnz = host_tot[0];
  h->n_cols = host_tot[1];
  h->touched_k = host_tot[2];

  const size_t esz = sizeof(D);
  const size_t d_ci = 0;
  const size_t d_cs = align_up(d_ci + (size_t)h->n_cols * 4, 256);
  const size_t d_v = align_up(d_cs + (size_t)(h->n_cols + 1) * 4, 256);
  const size_t d_r = align_up(d_v + (size_t)h->nnz * esz, 256);
  const size_t data_bytes = d_r + align_up((size_t)h->nnz, 16) + 256;
  if (dev_malloc(&h->data_base, data_bytes) != cudaSuccess) return ROSKO_ERR_OOM;
  char* db = static_cast<char*>(h->data_base);
  h->col_ind = reinterpret_cast<int32_t*>(db + d_ci);
  h->col_start = reinterpret_cast<int32_t*>(db + d_cs);
  h->vals = db + d_v;
  h->rows = reinterpret_cast<uint8_t*>(db + d_r);

  if (n > 0)
    scatter_kernel<S, D><<<grid, T, 0, st>>>(A, M, K, lda, h->m_r, scale, cnt, h->col_ind,
                                             h->col_start, reinterpret_cast<D*>(h->vals), h->rows,
                                             h->panel_col, h->panel_nnz_dev);
  if (n > 0) count_launches(1);
  // tails: panel_col[P] = n_cols, panel_nnz[P] = nnz, col_start[n_cols] = nnz
  int32_t tail32[2] = {(int32_t)h->n_cols, (int32_t)h->nnz};
  int64_t tail64 = h->nnz;
  if (cudaMemcpyAsync(h->panel_col + P, &tail32[0], 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(h->col_start + h->n_cols, &tail32[1], 4, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(h->panel_nnz_dev + P, &tail64, 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return ROSKO_ERR_CUDA;
  if (P == 0 || K == 0) {
    // no scatter ran: every panel starts at 0
    if (P > 0 && (cudaMemsetAsync(h->panel_col, 0, (size_t)P * 4, st) != cudaSuccess ||
                  cudaMemsetAsync(h->panel_nnz_dev, 0, (size_t)P * 8, st) != cudaSuccess))
      return ROSKO_ERR_CUDA;
  }
  // the scratch and the host tails above must outlive the queued work
  if (cudaStreamSynchronize(st) != cudaSuccess) return ROSKO_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return ROSKO_ERR_CUDA;
  return ROSKO_OK;
}

}  // namespace

rosko_status pack_impl(const void* A, rosko_dtype a_dt, int64_t M, int64_t K, int64_t lda,
                       rosko_dtype p_dt, const float* row_scale_in, int32_t m_r,
                       cudaStream_t stream, rosko_packed_s** out) {
  rosko_packed_s* h = new (std::nothrow) rosko_packed_s();
  if (!h) return ROSKO_ERR_OOM;
  cudaGetDevice(&h->device);
  h->M = M;
  h->K = K;
  h->m_r = m_r;
  h->P = (M + m_r - 1) / m_r;
  h->dt = p_dt;
  rosko_status s = ROSKO_ERR_UNSUPPORTED;
  if (a_dt == ROSKO_F32 && p_dt == ROSKO_F32)
    s = pack_typed<float, float>((const float*)A, M, K, lda, nullptr, false, h, stream);
  else if (a_dt == ROSKO_F32 && p_dt == ROSKO_BF16)
    s = pack_typed<float, __nv_bfloat16>((const float*)A, M, K, lda, nullptr, false, h, stream);
  else if (a_dt == ROSKO_F32 && p_dt == ROSKO_F64)
    s = pack_typed<float, double>((const float*)A, M, K, lda, nullptr, false, h, stream);
  else if (a_dt == ROSKO_F32 && p_dt == ROSKO_I8)
    s = pack_typed<float, int8_t>((const float*)A, M, K, lda, nullptr, true, h, stream);
  else if (a_dt == ROSKO_BF16 && p_dt == ROSKO_BF16)
    s = pack_typed<__nv_bfloat16, __nv_bfloat16>((const __nv_bfloat16*)A, M, K, lda, nullptr,
                                                 false, h, stream);
  else if (a_dt == ROSKO_I8 && p_dt == ROSKO_I8)
    s = pack_typed<int8_t, int8_t>((const int8_t*)A, M, K, lda, row_scale_in, false, h, stream);
  if (s != ROSKO_OK) {
    if (h->meta_base) cudaFree(h->meta_base);
    if (h->data_base) cudaFree(h->data_base);
    delete h;
    return s;
  }
  h->magic = kHandleMagic;
  *out = h;
  return ROSKO_OK;
}

rosko_status unpack_impl(rosko_packed_s* h, void* A_out, int64_t lda, cudaStream_t st) {
  const size_t esz = dtype_size(h->dt);
  if (h->M > 0 && h->K > 0 &&
      cudaMemset2DAsync(A_out, (size_t)lda * esz, 0, (size_t)h->K * esz, (size_t)h->M, st) !=
          cudaSuccess)
    return ROSKO_ERR_CUDA;
  if (h->P == 0 || h->nnz == 0) return ROSKO_OK;
  const unsigned g = (unsigned)h->P;
  switch (h->dt) {
    case ROSKO_F32:
      unpack_kernel<float><<<g, 256, 0, st>>>(h->panel_col, h->col_ind, h->col_start,
                                              (const float*)h->vals, h->rows, h->m_r, lda,
                                              (float*)A_out);
      break;
    case ROSKO_BF16:
      unpack_kernel<__nv_bfloat16><<<g, 256, 0, st>>>(h->panel_col, h->col_ind, h->col_start,
                                                      (const __nv_bfloat16*)h->vals, h->rows,
                                                      h->m_r, lda, (__nv_bfloat16*)A_out);
      break;
    case ROSKO_I8:
      unpack_kernel<int8_t><<<g, 256, 0, st>>>(h->panel_col, h->col_ind, h->col_start,
                                               (const int8_t*)h->vals, h->rows, h->m_r, lda,
                                               (int8_t*)A_out);
      break;
    case ROSKO_F64:
      unpack_kernel<double><<<g, 256, 0, st>>>(h->panel_col, h->col_ind, h->col_start,
                                               (const double*)h->vals, h->rows, h->m_r, lda,
                                               (double*)A_out);
      break;
    default:
      return ROSKO_ERR_UNSUPPORTED;
  }
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
}

}  // namespace rosko
