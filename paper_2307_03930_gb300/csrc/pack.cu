// Device packer: Alg. 1 (Sec. 4.1) applied to every row panel of A.
//
// Alg. 1 walks a tile column by column and, within a column, row by row,
// appending each nonzero to A_p / loc_m and, for a non-empty column, its
// index to col_ind and its count to nnz.  On the GPU the per-(panel, column)
// counts are independent, so the walk becomes count / scan / scatter:
//   count   one thread per (panel, column): nonzeros of that panel column
//   scan    exclusive prefix sums of (count, count != 0) in panel-major,
//           column-ascending order = Alg. 1's append order
//   scatter one thread per (panel, column): writes its column record and
//           its values/rows (rows ascending) at the scanned offsets
// The execution layouts of the SpMM (row stream, touched-row gather, dense
// BF16 tile copies) are built the same way, and the independent passes share
// launches: phase 1 is one counting launch and one three-array scan, phase 2
// one writing launch, with one host round trip between them (pack_typed).
// Threads of a warp own consecutive columns (or, for row passes, one warp owns
// a row), so every read of A is a coalesced row segment.
#include <algorithm>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

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

// One nonzero record (value + panel-relative row), see handle.hpp.
__device__ __forceinline__ void put_rec(void* nz, int64_t e, float v, int r) {
  reinterpret_cast<uint2*>(nz)[e] = make_uint2((uint32_t)r, __float_as_uint(v));
}
__device__ __forceinline__ void put_rec(void* nz, int64_t e, __nv_bfloat16 v, int r) {
  reinterpret_cast<uint32_t*>(nz)[e] = ((uint32_t)__bfloat16_as_ushort(v) << 16) | (uint32_t)r;
}
__device__ __forceinline__ void put_rec(void* nz, int64_t e, int8_t v, int r) {
  reinterpret_cast<uint32_t*>(nz)[e] = ((uint32_t)(uint8_t)v << 16) | (uint32_t)r;
}
__device__ __forceinline__ void put_rec(void* nz, int64_t e, double v, int r) {
  RecF64 w;
  w.a = v;
  w.r = r;
  w.pad = 0;
  reinterpret_cast<RecF64*>(nz)[e] = w;
}
__device__ __forceinline__ float get_val(const void* nz, int64_t e, float) {
  return __uint_as_float(reinterpret_cast<const uint2*>(nz)[e].y);
}
__device__ __forceinline__ __nv_bfloat16 get_val(const void* nz, int64_t e, __nv_bfloat16) {
  return __ushort_as_bfloat16((unsigned short)(reinterpret_cast<const uint32_t*>(nz)[e] >> 16));
}
__device__ __forceinline__ int8_t get_val(const void* nz, int64_t e, int8_t) {
  return (int8_t)(uint8_t)(reinterpret_cast<const uint32_t*>(nz)[e] >> 16);
}
__device__ __forceinline__ double get_val(const void* nz, int64_t e, double) {
  return reinterpret_cast<const RecF64*>(nz)[e].a;
}
__device__ __forceinline__ int get_row(const void* nz, int64_t e, float) {
  return (int)reinterpret_cast<const uint2*>(nz)[e].x;
}
template <class D>
__device__ __forceinline__ int get_row(const void* nz, int64_t e, D) {
  return (int)(reinterpret_cast<const uint32_t*>(nz)[e] & 0xFFFFu);
}
__device__ __forceinline__ int get_row(const void* nz, int64_t e, double) {
  return reinterpret_cast<const RecF64*>(nz)[e].r;
}

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

// Up to three independent exclusive scans of int2 arrays in place, sharing
// each of the three launches of a tiled scan: job i owns blocks
// [first[i], first[i+1]) of the tile passes and block i of the spine pass.
// data[n] receives the total; sums holds nb + 1 entries (nb = tiles of job).
struct ScanJob {
  int2* data;
  int64_t n;
  int2* sums;
  int64_t nb;
};
struct ScanSet {
  ScanJob job[3];
  int64_t first[4];
  int count;
};

__device__ __forceinline__ int scan_job_of(const ScanSet& s, int64_t b) {
  int i = 0;
  while (i + 1 < s.count && b >= s.first[i + 1]) ++i;
  return i;
}

// Tile pass A: per-tile sums.
__global__ void scan_reduce_kernel(ScanSet s) {
  const int j = scan_job_of(s, blockIdx.x);
  const ScanJob J = s.job[j];
  const int64_t base = ((int64_t)blockIdx.x - s.first[j]) * kScanTile;
  int2 v = make_int2(0, 0);
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
    if (idx < J.n) v = add2(v, J.data[idx]);
  }
  int2 total;
  block_excl_scan(v, &total);
  if (threadIdx.x == 0) J.sums[blockIdx.x - s.first[j]] = total;
}

// Spine pass B: exclusive scan of one job's tile sums (chunked), total to
// sums[nb].
__global__ void scan_spine_kernel(ScanSet s) {
  const ScanJob J = s.job[blockIdx.x];
  int2 carry = make_int2(0, 0);
  for (int64_t c0 = 0; c0 < J.nb; c0 += kScanThreads) {
    const int64_t idx = c0 + threadIdx.x;
    int2 v = idx < J.nb ? J.sums[idx] : make_int2(0, 0);
    int2 total;
    int2 ex = block_excl_scan(v, &total);
    if (idx < J.nb) J.sums[idx] = add2(ex, carry);
    carry = add2(carry, total);
    __syncthreads();
  }
  if (threadIdx.x == 0) J.sums[J.nb] = carry;
}

// Tile pass C: in-place exclusive scan of each tile with its offset.
__global__ void scan_down_kernel(ScanSet s) {
  const int j = scan_job_of(s, blockIdx.x);
  const ScanJob J = s.job[j];
  const int64_t tile = (int64_t)blockIdx.x - s.first[j];
  const int64_t base = tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int2 v[kScanItems];
  int2 sum = make_int2(0, 0);
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < J.n) ? J.data[base + i] : make_int2(0, 0);
    sum = add2(sum, v[i]);
  }
  int2 total;
  int2 off = add2(block_excl_scan(sum, &total), J.sums[tile]);
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < J.n) J.data[base + i] = off;
    off = add2(off, v[i]);
  }
  if (tile == 0 && threadIdx.x == 0) J.data[J.n] = J.sums[J.nb];
}

// Dense BF16 copies of 128-row tiles for the tensor-core dense-panel path:
// row block c holds rows tile_order[c]*128 .. +127 of A (zero past M and past
// K; row stride Kpad), converted exactly as the packer converts them.
__device__ __forceinline__ __nv_bfloat16 to_bf16(__nv_bfloat16 a) { return a; }
// INT8 codes are integers of magnitude <= 127: exact in BF16
__device__ __forceinline__ __nv_bfloat16 to_bf16(int8_t a) { return __float2bfloat16_rn((float)a); }

// Row-slot stream records (value + column k) and the per-row sentinel.
__device__ __forceinline__ void put_row_rec(void* rnz, int64_t e, float v, int k) {
  reinterpret_cast<uint2*>(rnz)[e] = make_uint2((uint32_t)k, __float_as_uint(v));
}
__device__ __forceinline__ void put_row_rec(void* rnz, int64_t e, __nv_bfloat16 v, int k) {
  reinterpret_cast<uint32_t*>(rnz)[e] = ((uint32_t)__bfloat16_as_ushort(v) << 16) | (uint32_t)k;
}
__device__ __forceinline__ void put_row_rec(void* rnz, int64_t e, int8_t v, int k) {
  reinterpret_cast<uint32_t*>(rnz)[e] = ((uint32_t)(uint8_t)v << 16) | (uint32_t)k;
}
__device__ __forceinline__ void put_row_rec(void* rnz, int64_t e, double v, int k) {
  RecF64 w;
  w.a = v;
  w.r = k;
  w.pad = 0;
  reinterpret_cast<RecF64*>(rnz)[e] = w;
}
template <class D>
__device__ __forceinline__ void put_row_sentinel(void* rnz, int64_t e) {
  if constexpr (sizeof(D) <= 2) {
    reinterpret_cast<uint32_t*>(rnz)[e] = 0xFFFFu;
  } else if constexpr (sizeof(D) == 4) {
    reinterpret_cast<uint2*>(rnz)[e] = make_uint2(0x7FFFFFFFu, 0u);
  } else {
    RecF64 w;
    w.a = 0.0;
    w.r = 0x7FFFFFFF;
    w.pad = 0;
    reinterpret_cast<RecF64*>(rnz)[e] = w;
  }
}

// ----------------------------------------------------------------------------
// The passes of one phase share a launch: a 1-D grid of 256-thread blocks in
// consecutive ranges, one range per pass (a block runs exactly one pass).
constexpr int kPackThreads = 256;
constexpr int kRowsPerBlock = kPackThreads / 32;   // row passes: one warp per row

struct PackGeom {
  int64_t M, K, lda, P, T;
  int m_r;
  int64_t gx;   // 256-column groups, ceil(K / 256)
};

// Counting pass, Alg. 1's per-column nnz: cnt[p*K + k] = (nonzeros of column
// k in panel p, 1 if non-empty); a column's first nonzero seen anywhere
// counts it as touched.  The same visit of the panel yields the other two
// counts: the nonzeros of each row (a ballot per row across the warp, summed
// over the block in shared memory, one atomic add per row and block into
// rcnt, which starts at 0; the block of columns 0..255 adds the row's
// sentinel) and, for the gather stream, flag[t*K + k].x = 1 when column k of
// 128-row tile t is non-empty (flag starts at 0).
template <class S, class D>
__device__ void col_count(const S* __restrict__ A, const PackGeom& g,
                          const float* __restrict__ scale, int64_t b, int2* __restrict__ cnt,
                          int* __restrict__ touched, int* __restrict__ touched_total,
                          int2* __restrict__ rcnt, int2* __restrict__ flag) {
  __shared__ int row_sum[32];   // m_r <= 32
  const int64_t bx = b % g.gx;
  const int64_t k = bx * kPackThreads + threadIdx.x;
  const int64_t p = b / g.gx;
  const bool in = k < g.K;
  const int lane = threadIdx.x & 31;
  const int64_t m0 = p * g.m_r, m1 = min(g.M, m0 + g.m_r);
  if (rcnt) {
    if (threadIdx.x < 32) row_sum[threadIdx.x] = 0;
    __syncthreads();
  }
  int c = 0;
  // bounds are uniform across the block: every lane takes every ballot
#pragma unroll 8
  for (int64_t m = m0; m < m1; ++m) {
    D v;
    const bool nz = in && Conv<S, D>::get(A[m * g.lda + k], scale ? scale[m] : 1.0f, v);
    c += nz ? 1 : 0;
    if (rcnt) {
      const unsigned mask = __ballot_sync(0xffffffffu, nz);
      if (lane == 0 && mask) atomicAdd(&row_sum[m - m0], __popc(mask));
    }
  }
  if (rcnt) {
    __syncthreads();
    const int64_t r = m0 + threadIdx.x;
    if (threadIdx.x < 32 && r < m1) {
      const int add = row_sum[threadIdx.x] + (bx == 0 ? 1 : 0);
      if (add) atomicAdd(&rcnt[r].x, add);
    }
  }
  if (!in) return;
  cnt[p * g.K + k] = make_int2(c, c != 0);
  if (c && atomicExch(&touched[k], 1) == 0) atomicAdd(touched_total, 1);
  if (c && flag) flag[(m0 / kDenseTileRows) * g.K + k] = make_int2(1, 0);
}

// Counting pass of the row-slot stream: rcnt[row] = (nonzeros of the row + 1
// sentinel, 0); lanes over consecutive columns (coalesced).
template <class S, class D>
__device__ void row_count(const S* __restrict__ A, const PackGeom& g,
                          const float* __restrict__ scale, int64_t b, int2* __restrict__ rcnt) {
  const int64_t row = b * kRowsPerBlock + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= g.M) return;
  const float sc = scale ? scale[row] : 1.0f;
  int c = 0;
#pragma unroll 8
  for (int64_t k = lane; k < g.K; k += 32) {
    D v;
    c += Conv<S, D>::get(A[row * g.lda + k], sc, v) ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) rcnt[row] = make_int2(c + 1, 0);
}

// Phase 1 in one launch: blocks [0, b_col) count panel columns (and rows and
// tile columns, see col_count); with K = 0 there are no column blocks and
// the remaining blocks give each row its sentinel count instead.
template <class S, class D>
__global__ void __launch_bounds__(kPackThreads)
    pack_count_kernel(const S* __restrict__ A, PackGeom g, const float* __restrict__ scale,
                      int2* __restrict__ cnt, int* __restrict__ touched,
                      int* __restrict__ touched_total, int2* __restrict__ rcnt,
                      int2* __restrict__ flag, int64_t b_col) {
  const int64_t b = blockIdx.x;
  if (b < b_col) {
    col_count<S, D>(A, g, scale, b, cnt, touched, touched_total, rcnt, flag);
    return;
  }
  row_count<S, D>(A, g, scale, b - b_col, rcnt);
}

// Pointers and block ranges of the writing phase.  Scanned offsets:
// cnt[p*K+k] = (first nonzero, first packed column) of a panel column,
// rcnt[row].x = first record of a row, flag[t*K+k].x = slot of column k in
// tile t's union list (plus the tile's base).
struct WriteArgs {
  const int2* cnt;
  int2* colrec;
  void* nz;
  int32_t* panel_col;
  int64_t* panel_nnz;
  const int2* rcnt;
  int32_t* rowptr;
  void* rnz;
  const int2* flag;
  int32_t* gu_start;
  int32_t* gu_k;
  void* gnz;
  const int32_t* tile_order;
  __nv_bfloat16* dense_A;
  int64_t dense_rows, Kpad, gxd, ry;
  int64_t nnz, n_cols, gu_total;
  int zero_panels;
  int64_t b_scatter, b_row, b_union, b_dense;
};

// Alg. 1's append: each non-empty panel column writes its column record and
// its values with rows ascending at the scanned offsets.
template <class S, class D>
__device__ void scatter(const S* __restrict__ A, const PackGeom& g,
                        const float* __restrict__ scale, int64_t b, const WriteArgs& w) {
  const int64_t k = (b % g.gx) * kPackThreads + threadIdx.x;
  const int64_t p = b / g.gx;
  if (k >= g.K) return;
  const int64_t pk = p * g.K + k;
  const int2 o = w.cnt[pk];
  if (k == 0) {
    w.panel_col[p] = o.y;
    w.panel_nnz[p] = o.x;
  }
  const int cnt = w.cnt[pk + 1].x - o.x;
  if (cnt == 0) return;
  w.colrec[o.y] = make_int2((int32_t)k, o.x);
  const int64_t m0 = p * g.m_r, m1 = min(g.M, m0 + g.m_r);
  int64_t e = o.x;
  for (int64_t m = m0; m < m1; ++m) {
    D v;
    if (Conv<S, D>::get(A[m * g.lda + k], scale ? scale[m] : 1.0f, v)) {
      put_rec(w.nz, e, v, (int)(m - m0));
      ++e;
    }
  }
}

// Row-slot stream: each row's records (k ascending) at its scanned offset,
// then its sentinel; with the gather stream, the same record re-addressed by
// the slot of k in the tile's union list goes to the same position of gnz.
template <class S, class D>
__device__ void row_write(const S* __restrict__ A, const PackGeom& g,
                          const float* __restrict__ scale, int64_t b, const WriteArgs& w) {
  const int64_t row = b * kRowsPerBlock + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= g.M) return;
  const float sc = scale ? scale[row] : 1.0f;
  int64_t pos = w.rcnt[row].x;
  if (lane == 0) w.rowptr[row] = (int32_t)pos;
  const int2* tf = w.flag ? w.flag + (row / kDenseTileRows) * g.K : nullptr;
  const int32_t base = tf ? tf[0].x : 0;
  // eight 32-column groups per step: their loads are issued together, then
  // the records are written in k order
  constexpr int G = 8;
  for (int64_t k0 = 0; k0 < g.K; k0 += 32 * G) {
    S a[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int64_t k = k0 + u * 32 + lane;
      a[u] = k < g.K ? A[row * g.lda + k] : S(0);
    }
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int64_t k = k0 + u * 32 + lane;
      D v;
      const bool nzf = (k < g.K) && Conv<S, D>::get(a[u], sc, v);
      const unsigned mask = __ballot_sync(0xffffffffu, nzf);
      if (nzf) {
        const int64_t q = pos + __popc(mask & ((1u << lane) - 1u));
        put_row_rec(w.rnz, q, v, (int)k);
        if (tf) put_row_rec(w.gnz, q, v, (int)(tf[k].x - base));
      }
      pos += __popc(mask);
    }
  }
  if (lane == 0) {
    put_row_sentinel<D>(w.rnz, pos);
    if (tf) put_row_sentinel<D>(w.gnz, pos);
  }
}

// Gather stream: the union list gu_k of each tile and its offset gu_start.
__device__ void tile_union(const PackGeom& g, int64_t b, const WriteArgs& w) {
  const int64_t k = (b % g.gx) * kPackThreads + threadIdx.x;
  const int64_t t = b / g.gx;
  if (k >= g.K) return;
  const int64_t i = t * g.K + k;
  if (k == 0) w.gu_start[t] = w.flag[i].x;
  if (w.flag[i + 1].x != w.flag[i].x) w.gu_k[w.flag[i].x] = (int32_t)k;
}

// The dense copy holds each entry converted exactly as the packer converts
// it (BF16 packs: the BF16 value; INT8 packs: the INT8 code, exact in BF16).
template <class S, class D>
__device__ void densify(const S* __restrict__ A, const PackGeom& g,
                        const float* __restrict__ scale, int64_t b, const WriteArgs& w) {
  const int64_t k = (b % w.gxd) * kPackThreads + threadIdx.x;
  if (k >= w.Kpad) return;
  for (int64_t rr = b / w.gxd; rr < w.dense_rows; rr += w.ry) {
    const int64_t row = (int64_t)w.tile_order[rr / kDenseTileRows] * kDenseTileRows +
                        rr % kDenseTileRows;
    __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
    if (row < g.M && k < g.K) {
      D q;
      Conv<S, D>::get(A[row * g.lda + k], scale ? scale[row] : 1.0f, q);
      v = to_bf16(q);
    }
    w.dense_A[rr * w.Kpad + k] = v;
  }
}

// Terminating entries: panel_col[P] = packed columns, panel_nnz[P] = nnz,
// colrec[n_cols] = colrec[n_cols + 1] = {INT32_MAX, nnz}, rowptr[M] = nnz + M
// (row stream), gu_start[T] = union total (gather stream); with no scatter
// (K = 0) every panel starts at 0.
__device__ void tails(const PackGeom& g, const WriteArgs& w) {
  if (w.zero_panels)
    for (int64_t p = threadIdx.x; p < g.P; p += blockDim.x) {
      w.panel_col[p] = 0;
      w.panel_nnz[p] = 0;
    }
  if (threadIdx.x == 0) {
    w.panel_col[g.P] = (int32_t)w.n_cols;
    w.panel_nnz[g.P] = w.nnz;
    w.colrec[w.n_cols] = make_int2(INT32_MAX, (int32_t)w.nnz);
    w.colrec[w.n_cols + 1] = make_int2(INT32_MAX, (int32_t)w.nnz);
    if (w.rowptr) w.rowptr[g.M] = (int32_t)(w.nnz + g.M);
    if (w.gu_start) w.gu_start[g.T] = (int32_t)w.gu_total;
  }
}

// Phase 2 in one launch: scatter, row write (+ gather records), union lists,
// dense copies, then one block of terminating entries.
template <class S, class D>
__global__ void __launch_bounds__(kPackThreads)
    pack_write_kernel(const S* __restrict__ A, PackGeom g, const float* __restrict__ scale,
                      WriteArgs w) {
  int64_t b = blockIdx.x;
  if (b < w.b_scatter) {
    scatter<S, D>(A, g, scale, b, w);
    return;
  }
  b -= w.b_scatter;
  if (b < w.b_row) {
    row_write<S, D>(A, g, scale, b, w);
    return;
  }
  b -= w.b_row;
  if (b < w.b_union) {
    tile_union(g, b, w);
    return;
  }
  b -= w.b_union;
  if constexpr (std::is_same<D, __nv_bfloat16>::value || std::is_same<D, int8_t>::value) {
    if (b < w.b_dense) {
      densify<S, D>(A, g, scale, b, w);
      return;
    }
  }
  tails(g, w);
}

template <class D>
__global__ void unpack_kernel(const int32_t* __restrict__ panel_col,
                              const int2* __restrict__ colrec, const void* __restrict__ nz,
                              int m_r, int64_t lda, D* __restrict__ out) {
  const int64_t p = blockIdx.x;
  for (int64_t c = panel_col[p] + threadIdx.x; c < panel_col[p + 1]; c += blockDim.x) {
    const int64_t k = colrec[c].x;
    for (int32_t e = colrec[c].y; e < colrec[c + 1].y; ++e)
      out[(p * m_r + get_row(nz, e, D())) * lda + k] = get_val(nz, e, D());
  }
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Stream-ordered scratch from the library's pool, released in the order of
// its stream (so an early return never frees memory that queued work uses).
struct PoolScratch {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  ~PoolScratch() { pool_free(p, st); }
};

__global__ void fill_kernel(float* __restrict__ out, int64_t n, float v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v;
}

// What the host needs to lay out the handle, gathered from the scans into one
// array so that a single copy brings it back:
//   sum64[0..3]    nonzeros, packed columns, touched columns, gather-union total
//   sum64[4..4+P]  nonzero offset of every panel, then the total
//   rowptr[0..M]   row-stream offsets (row stream only)
__global__ void pack_summary_kernel(const int2* __restrict__ cnt, int64_t n, int64_t P, int64_t K,
                                    const int* __restrict__ touched_total,
                                    const int2* __restrict__ rcnt, int64_t M,
                                    const int2* __restrict__ flag, int64_t nf,
                                    int64_t* __restrict__ sum64, int32_t* __restrict__ rowptr) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    sum64[0] = cnt[n].x;
    sum64[1] = cnt[n].y;
    sum64[2] = *touched_total;
    sum64[3] = flag ? flag[nf].x : 0;
  }
  if (i <= P) sum64[4 + i] = i < P ? cnt[i * K].x : cnt[n].x;
  if (rcnt && i <= M) rowptr[i] = rcnt[i].x;
}

// Dense-panel split bookkeeping (BF16 packs): 128-row tiles sorted by density,
// descending; the tiles at or above dense_min_pm per mille get a dense copy;
// panel_order lists the panels tile by tile in ascending density.
void plan_dense_tiles(rosko_packed_s* h, int32_t dense_min_pm) {
  const int64_t M = h->M, K = h->K, P = h->P;
  const int64_t T = (M + kDenseTileRows - 1) / kDenseTileRows;
  const int64_t ppt = kDenseTileRows / h->m_r;
  std::vector<double> dens((size_t)T);
  h->tile_panels.assign((size_t)T, 0);
  for (int64_t t = 0; t < T; ++t) {
    const int64_t p0 = t * ppt, p1 = std::min<int64_t>(P, p0 + ppt);
    const int64_t rows = std::min<int64_t>(kDenseTileRows, M - t * kDenseTileRows);
    dens[(size_t)t] = (double)(h->panel_nnz[(size_t)p1] - h->panel_nnz[(size_t)p0]) /
                      ((double)rows * (double)K);
    h->tile_panels[(size_t)t] = (int32_t)(p1 - p0);
  }
  h->tile_order.resize((size_t)T);
  for (int64_t t = 0; t < T; ++t) h->tile_order[(size_t)t] = (int32_t)t;
  std::stable_sort(h->tile_order.begin(), h->tile_order.end(),
                   [&](int32_t a, int32_t b) { return dens[(size_t)a] > dens[(size_t)b]; });
  h->tile_density.resize((size_t)T);
  int64_t n_copy = 0;
  for (int64_t c = 0; c < T; ++c) {
    h->tile_density[(size_t)c] = dens[(size_t)h->tile_order[(size_t)c]];
    if (h->tile_density[(size_t)c] * 1000.0 >= (double)dense_min_pm) n_copy = c + 1;
  }
  std::vector<int32_t>& panel_order = h->panel_order_host;
  panel_order.clear();
  panel_order.reserve((size_t)P);
  for (int64_t c = T - 1; c >= 0; --c) {
    const int64_t t = h->tile_order[(size_t)c];
    for (int64_t q = 0; q < h->tile_panels[(size_t)t]; ++q)
      panel_order.push_back((int32_t)(t * ppt + q));
  }
  h->n_tiles = T;
  h->n_copy = n_copy;
  h->Kpad = (K + 7) / 8 * 8;
}

// Row-direct work segments (see rosko_packed_s) from the row-stream offsets,
// at both granularities: {row, first record, end record, cut} in row order
// (nat) and, with a panel order, in that order (ord).
void plan_segments(rosko_packed_s* h, const int32_t* rp, const std::vector<int32_t>* panel_order,
                   std::vector<int4> nat[2], std::vector<int4> ord[2], std::vector<int4> lpt[2]) {
  const int64_t M = h->M, P = h->P;
  const int64_t lens[2] = {kSegRecords, seg_records_for(h->nnz, M)};
  for (int g = 0; g < 2; ++g) {
    const int64_t seg = lens[g];
    rosko_packed_s::SegList& L = h->segs[g];
    L.records = (int32_t)seg;
    nat[g].reserve((size_t)M + (size_t)(h->nnz / seg) + 1);
    std::vector<int64_t> panel_seg((size_t)P + 1, 0);
    std::vector<char> panel_split((size_t)P, 0);
    for (int64_t p = 0; p < P; ++p) {
      panel_seg[(size_t)p] = (int64_t)nat[g].size();
      for (int64_t r = p * h->m_r; r < std::min<int64_t>(M, (p + 1) * h->m_r); ++r) {
        const int64_t nr = (int64_t)rp[r + 1] - rp[r] - 1;   // minus the sentinel
        const int64_t ns = std::max<int64_t>(1, (nr + seg - 1) / seg);
        if (ns > 1) panel_split[(size_t)p] = 1;
        const int64_t row_end = (int64_t)rp[r + 1] - 1;
        for (int64_t k = 0; k < ns; ++k) {
          const int64_t e0 = (int64_t)rp[r] + k * seg;
          // the entry's head; its inline records are written on the device
          nat[g].push_back(make_int4((int)r, (int)e0, (int)std::min<int64_t>(e0 + seg, row_end),
                                     ns > 1 ? 1 : 0));
        }
      }
    }
    panel_seg[(size_t)P] = (int64_t)nat[g].size();
    L.prefix.assign((size_t)P + 1, 0);
    L.split.assign((size_t)P + 1, 0);
    for (int64_t i = 0; i < P; ++i) {
      const int64_t p = panel_order ? (*panel_order)[(size_t)i] : i;
      if (panel_order)
        ord[g].insert(ord[g].end(), nat[g].begin() + panel_seg[(size_t)p],
                      nat[g].begin() + panel_seg[(size_t)p + 1]);
      L.prefix[(size_t)i + 1] = L.prefix[(size_t)i] + (panel_seg[(size_t)p + 1] - panel_seg[(size_t)p]);
      L.split[(size_t)i + 1] = L.split[(size_t)i] + panel_split[(size_t)p];
    }
    lpt[g] = nat[g];
    std::stable_sort(lpt[g].begin(), lpt[g].end(), [](const int4& a, const int4& b) {
      return a.z - a.y > b.z - b.y;
    });
  }
}

// The work segments' entries: each head (staged from the host, 16 bytes)
// and the first 48 bytes of the piece's records in the row stream (written
// by the phase-2 launch); one thread per (segment, 4-byte word: 4 of head,
// 12 of records), over up to six lists.
struct InlineLists {
  SegEntry* list[6];
  const int4* heads[6];
  int64_t n[6];
  int64_t first[7];   // first thread of each list
};
__global__ void seg_inline_kernel(InlineLists L, const uint32_t* __restrict__ rnz, int rec_words) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int l = 0;
  while (l < 5 && t >= L.first[l + 1]) ++l;
  if (t >= L.first[6]) return;
  const int64_t local = t - L.first[l];
  const int64_t s = local / 16;
  const int w = (int)(local - s * 16);
  const int4 hd = L.heads[l][s];
  SegEntry& e = L.list[l][s];
  if (w < 4) {
    reinterpret_cast<int*>(&e.head)[w] = w == 0 ? hd.x : (w == 1 ? hd.y : (w == 2 ? hd.z : hd.w));
    return;
  }
  const int rw = w - 4;
  const int64_t words = (int64_t)(hd.z - hd.y) * rec_words;
  if (rw < words && rw / rec_words < 12 / rec_words) e.rec[rw] = rnz[(int64_t)hd.y * rec_words + rw];
}

// Bump allocator over byte offsets, each region 256-byte aligned.
struct Layout {
  size_t top = 0;
  size_t take(size_t bytes, size_t align = 256) {
    top = align_up(top, align);
    const size_t at = top;
    top += bytes;
    return at;
  }
};

// The whole pack in two phases with one host round trip:
//   1. every counting pass (per panel column: Alg. 1's counts; per row: the
//      row stream; per 128-row tile and column: the gather union), their
//      scans, and one summary array copied back;
//   2. the host lays out the handle in one allocation (plus the tile order
//      and segment lists it derives from the summary, staged in one copy),
//      then every writing pass runs.
template <class S, class D>
rosko_status pack_typed(const S* A, int64_t lda, const float* scale_in, bool quantize_rows,
                        int32_t dense_min_pm, rosko_packed_s* h, cudaStream_t st) {
  const int64_t M = h->M, K = h->K, P = h->P;
  const int64_t n = P * K;
  const int64_t T = (M + kDenseTileRows - 1) / kDenseTileRows;
  const bool rows = M > 0 && K < kRowSlotMaxK;
  const bool gather = rows && h->m_r == 16 && K > 0;
  const bool dense = (std::is_same<D, __nv_bfloat16>::value || std::is_same<D, int8_t>::value) &&
                     dense_min_pm <= 1000 && M > 0 && K > 0;
  const int64_t nf = gather ? T * K : 0;
  auto blocks_for = [](int64_t x) { return (x + kScanTile - 1) / kScanTile + 1; };

  // ---- phase 1: counts ------------------------------------------------------
  Layout s;
  const size_t o_cnt = s.take((size_t)(n + 1) * sizeof(int2));
  const size_t o_sums = s.take((size_t)blocks_for(n) * sizeof(int2));
  const size_t o_touch = s.take((size_t)std::max<int64_t>(K, 1) * sizeof(int));
  const size_t o_tot = s.take(16);
  const size_t o_rcnt = s.take(rows ? (size_t)(M + 1) * sizeof(int2) : 0);
  const size_t o_rsums = s.take(rows ? (size_t)blocks_for(M) * sizeof(int2) : 0);
  const size_t o_flag = s.take((size_t)(nf + 1) * sizeof(int2));
  const size_t o_fsums = s.take((size_t)blocks_for(nf) * sizeof(int2));
  const size_t o_scale = s.take(quantize_rows ? (size_t)M * 4 : 0);
  const size_t o_sum64 = s.take((size_t)(P + 5) * 8);
  const size_t o_rp = s.take(rows ? (size_t)(M + 1) * 4 : 0);
  const size_t summary_bytes = s.top - o_sum64;
  PoolScratch scr;
  scr.st = st;
  if (pool_malloc(&scr.p, s.top + 256, st) != cudaSuccess) return ROSKO_ERR_OOM;
  char* sb = static_cast<char*>(scr.p);
  int2* cnt = reinterpret_cast<int2*>(sb + o_cnt);
  int* touched = reinterpret_cast<int*>(sb + o_touch);
  int* tot = reinterpret_cast<int*>(sb + o_tot);
  int2* rcnt = rows ? reinterpret_cast<int2*>(sb + o_rcnt) : nullptr;
  int2* flag = gather ? reinterpret_cast<int2*>(sb + o_flag) : nullptr;

  // touched flags, totals, row counts (and their tile sums) and tile flags
  // are adjacent: one memset
  if (cudaMemsetAsync(touched, 0, o_fsums - o_touch, st) != cudaSuccess ||
      (n == 0 && cudaMemsetAsync(cnt, 0, sizeof(int2), st) != cudaSuccess))
    return ROSKO_ERR_CUDA;
  const float* scale = nullptr;
  if (quantize_rows) {
    scale = reinterpret_cast<float*>(sb + o_scale);
    const int wpb = 8;
    if (M > 0) {
      rowscale_kernel<<<(unsigned)((M + wpb - 1) / wpb), wpb * 32, 0, st>>>(
          reinterpret_cast<const float*>(A), M, K, lda, const_cast<float*>(scale));
      count_launches(1);
    }
  }
  PackGeom geo;
  geo.M = M;
  geo.K = K;
  geo.lda = lda;
  geo.P = P;
  geo.T = T;
  geo.m_r = h->m_r;
  geo.gx = (K + kPackThreads - 1) / kPackThreads;
  const int64_t b_col = n > 0 ? geo.gx * P : 0;
  // rows are counted by the column blocks; without columns (K = 0) every row
  // still gets its sentinel from a row block
  const int64_t b_row_count = (rows && n == 0) ? (M + kRowsPerBlock - 1) / kRowsPerBlock : 0;
  if (b_col + b_row_count > 0) {
    pack_count_kernel<S, D><<<(unsigned)(b_col + b_row_count), kPackThreads, 0, st>>>(
        A, geo, scale, cnt, touched, tot + 2, rcnt, flag, b_col);
    count_launches(1);
  }
  // the writing phase's ranges
  const int64_t b_row = rows ? (M + kRowsPerBlock - 1) / kRowsPerBlock : 0;
  const int64_t b_tile = gather ? geo.gx * T : 0;
  {
    ScanSet ss;
    std::memset(&ss, 0, sizeof(ss));
    auto add = [&](int2* data, int64_t len, size_t o_s) {
      if (len <= 0) return;
      ScanJob& J = ss.job[ss.count];
      J.data = data;
      J.n = len;
      J.sums = reinterpret_cast<int2*>(sb + o_s);
      J.nb = (len + kScanTile - 1) / kScanTile;
      ss.first[ss.count + 1] = ss.first[ss.count] + J.nb;
      ++ss.count;
    };
    add(cnt, n, o_sums);
    if (rows) add(rcnt, M, o_rsums);
    if (gather) add(flag, nf, o_fsums);
    if (ss.count > 0) {
      const unsigned tiles = (unsigned)ss.first[ss.count];
      scan_reduce_kernel<<<tiles, kScanThreads, 0, st>>>(ss);
      scan_spine_kernel<<<(unsigned)ss.count, kScanThreads, 0, st>>>(ss);
      scan_down_kernel<<<tiles, kScanThreads, 0, st>>>(ss);
      count_launches(3);
    }
  }
  {
    const int64_t span = std::max<int64_t>(P, M) + 1;
    pack_summary_kernel<<<(unsigned)((span + 255) / 256), 256, 0, st>>>(
        cnt, n, P, K, tot + 2, rcnt, M, flag, nf, reinterpret_cast<int64_t*>(sb + o_sum64),
        rows ? reinterpret_cast<int32_t*>(sb + o_rp) : nullptr);
    count_launches(1);
  }
  std::vector<int64_t> summary((summary_bytes + 7) / 8);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(summary.data(), sb + o_sum64, summary_bytes, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ROSKO_ERR_CUDA;

  // ---- host: sizes, dense tiles, segments, layout ----------------------------
  h->nnz = summary[0];
  h->n_cols = summary[1];
  h->touched_k = summary[2];
  h->gu_total = gather ? summary[3] : 0;
  h->panel_nnz.assign(summary.begin() + 4, summary.begin() + 5 + P);
  const int32_t* rp =
      rows ? reinterpret_cast<const int32_t*>(reinterpret_cast<const char*>(summary.data()) +
                                              (o_rp - o_sum64))
           : nullptr;
  if (dense) plan_dense_tiles(h, dense_min_pm);
  std::vector<int4> nat[2], ord[2], lpt[2];
  if (rows) plan_segments(h, rp, dense ? &h->panel_order_host : nullptr, nat, ord, lpt);

  const size_t rsz = rec_size(h->dt);
  const int64_t nnz = h->nnz, n_cols = h->n_cols;
  Layout L;
  // staged from the host in one copy
  const size_t o_to = L.take(dense ? (size_t)T * 4 : 0);
  const size_t o_po = L.take(dense ? (size_t)P * 4 : 0);
  const size_t staged = L.top;
  // written on the device (the segment entries: heads staged apart, below)
  size_t o_seg[6];
  for (int g = 0; g < 2; ++g) {
    o_seg[3 * g] = L.take(nat[g].size() * sizeof(SegEntry));
    o_seg[3 * g + 1] = L.take(ord[g].size() * sizeof(SegEntry));
    o_seg[3 * g + 2] = L.take(lpt[g].size() * sizeof(SegEntry));
  }
  // written on the device
  const size_t o_pc = L.take((size_t)(P + 1) * 4);
  const size_t o_pn = L.take((size_t)(P + 1) * 8);
  const size_t o_rs = L.take((size_t)std::max<int64_t>(M, 1) * 4);
  const size_t o_ft = L.take(256);
  const size_t o_cr = L.take((size_t)(n_cols + 2) * 8);
  const size_t o_nz = L.take((size_t)(nnz + 1) * rsz);
  const size_t o_rowptr = L.take(rows ? (size_t)(M + 1) * 4 : 0);
  const size_t o_rnz = L.take(rows ? (size_t)(nnz + M) * rsz : 0);
  const size_t o_gs = L.take(gather ? (size_t)(T + 1) * 4 : 0);
  const size_t o_gk = L.take(gather ? (size_t)std::max<int64_t>(h->gu_total, 1) * 4 : 0);
  const size_t o_gnz = L.take(gather ? (size_t)(nnz + M) * rsz : 0);
  const size_t o_da =
      L.take(dense ? (size_t)h->n_copy * kDenseTileRows * (size_t)h->Kpad * 2 : 0, 1024);
  if (pool_malloc(&h->base, L.top + 256, st) != cudaSuccess) return ROSKO_ERR_OOM;
  h->base_bytes = L.top + 256;
  char* b = static_cast<char*>(h->base);
  h->panel_col = reinterpret_cast<int32_t*>(b + o_pc);
  h->panel_nnz_dev = reinterpret_cast<int64_t*>(b + o_pn);
  h->row_scale = reinterpret_cast<float*>(b + o_rs);
  h->feat_dev = reinterpret_cast<float*>(b + o_ft);
  h->colrec = reinterpret_cast<int2*>(b + o_cr);
  h->nz = b + o_nz;
  if (rows) {
    h->rowptr = reinterpret_cast<int32_t*>(b + o_rowptr);
    h->rnz = b + o_rnz;
    for (int g = 0; g < 2; ++g) {
      h->segs[g].nat = reinterpret_cast<SegEntry*>(b + o_seg[3 * g]);
      h->segs[g].ord = dense ? reinterpret_cast<SegEntry*>(b + o_seg[3 * g + 1]) : nullptr;
      h->segs[g].lpt = reinterpret_cast<SegEntry*>(b + o_seg[3 * g + 2]);
    }
  }
  if (gather) {
    h->gu_start = reinterpret_cast<int32_t*>(b + o_gs);
    h->gu_k = reinterpret_cast<int32_t*>(b + o_gk);
    h->gnz = b + o_gnz;
  }
  if (dense) {
    h->tile_order_dev = reinterpret_cast<int32_t*>(b + o_to);
    h->panel_order_dev = reinterpret_cast<int32_t*>(b + o_po);
    h->dense_A = b + o_da;
  }
  if (staged > 0) {
    std::vector<char> stage(staged, 0);
    if (dense) {
      std::memcpy(stage.data() + o_to, h->tile_order.data(), (size_t)T * 4);
      std::memcpy(stage.data() + o_po, h->panel_order_host.data(), (size_t)P * 4);
    }
    // a pageable source is staged before the call returns
    if (cudaMemcpyAsync(b, stage.data(), staged, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return ROSKO_ERR_CUDA;
  }
  // the segment heads (16 bytes each; the entries' inline records are
  // filled on the device) go to stream-ordered scratch from the library's
  // pool (it keeps freed memory mapped: the default pool would map it anew
  // on every pack), released after the launch that expands them
  size_t n_heads = 0;
  for (int g = 0; g < 2; ++g) n_heads += nat[g].size() + ord[g].size() + lpt[g].size();
  std::vector<int4> heads;
  heads.reserve(n_heads);
  for (int g = 0; g < 2; ++g)
    for (const std::vector<int4>* v : {&nat[g], &ord[g], &lpt[g]}) heads.insert(heads.end(), v->begin(), v->end());
  struct Scratch {
    void* p = nullptr;
    cudaStream_t st;
    ~Scratch() {
      if (p) pool_free(p, st);
    }
  } heads_dev{nullptr, st};
  if (n_heads > 0) {
    if (pool_malloc(&heads_dev.p, n_heads * sizeof(int4), st) != cudaSuccess) {
      heads_dev.p = nullptr;
      return ROSKO_ERR_OOM;
    }
    if (cudaMemcpyAsync(heads_dev.p, heads.data(), n_heads * sizeof(int4), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
      return ROSKO_ERR_CUDA;
  }

  // ---- phase 2: writes ------------------------------------------------------
  if (quantize_rows) {
    if (M > 0 && cudaMemcpyAsync(h->row_scale, scale, (size_t)M * 4, cudaMemcpyDeviceToDevice,
                                 st) != cudaSuccess)
      return ROSKO_ERR_CUDA;
  } else if (h->dt == ROSKO_I8 && M > 0) {
    if (scale_in) {
      if (cudaMemcpyAsync(h->row_scale, scale_in, (size_t)M * 4, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess)
        return ROSKO_ERR_CUDA;
    } else {
      fill_kernel<<<(unsigned)std::min<int64_t>((M + 255) / 256, 1024), 256, 0, st>>>(
          h->row_scale, M, 1.0f);
      count_launches(1);
    }
  }
  WriteArgs w;
  std::memset(&w, 0, sizeof(w));
  w.cnt = cnt;
  w.colrec = h->colrec;
  w.nz = h->nz;
  w.panel_col = h->panel_col;
  w.panel_nnz = h->panel_nnz_dev;
  w.rcnt = rcnt;
  w.rowptr = h->rowptr;
  w.rnz = h->rnz;
  w.flag = flag;
  w.gu_start = h->gu_start;
  w.gu_k = h->gu_k;
  w.gnz = h->gnz;
  w.nnz = nnz;
  w.n_cols = n_cols;
  w.gu_total = h->gu_total;
  w.zero_panels = n == 0 ? 1 : 0;
  w.b_scatter = b_col;
  w.b_row = b_row;
  w.b_union = b_tile;
  if (dense && h->n_copy > 0) {
    w.tile_order = h->tile_order_dev;
    w.dense_A = reinterpret_cast<__nv_bfloat16*>(h->dense_A);
    w.dense_rows = h->n_copy * kDenseTileRows;
    w.Kpad = h->Kpad;
    w.gxd = (h->Kpad + kPackThreads - 1) / kPackThreads;
    w.ry = std::min<int64_t>(w.dense_rows, 2048);
    w.b_dense = w.gxd * w.ry;
  }
  pack_write_kernel<S, D>
      <<<(unsigned)(w.b_scatter + w.b_row + w.b_union + w.b_dense + 1), kPackThreads, 0, st>>>(
          A, geo, scale, w);
  count_launches(1);
  if (rows) {
    // the segments' inline records, once the row stream is written
    InlineLists il;
    std::memset(&il, 0, sizeof(il));
    int nl = 0;
    // heads are staged in the order nat, ord, lpt of list 0, then of list 1
    const int4* hp = static_cast<const int4*>(heads_dev.p);
    for (int g = 0; g < 2; ++g) {
      SegEntry* dst[3] = {h->segs[g].nat, h->segs[g].ord, h->segs[g].lpt};
      const std::vector<int4>* src[3] = {&nat[g], &ord[g], &lpt[g]};
      for (int k = 0; k < 3; ++k) {
        if (dst[k] && !src[k]->empty()) {
          il.list[nl] = dst[k];
          il.heads[nl] = hp;
          il.n[nl++] = (int64_t)src[k]->size();
        }
        hp += src[k]->size();
      }
    }
    il.first[0] = 0;
    for (int l = 0; l < 6; ++l) il.first[l + 1] = il.first[l] + (l < nl ? il.n[l] * 16 : 0);
    if (il.first[6] > 0) {
      seg_inline_kernel<<<(unsigned)((il.first[6] + 255) / 256), 256, 0, st>>>(
          il, static_cast<const uint32_t*>(h->rnz), (int)(rsz / 4));
      count_launches(1);
    }
  }
  // the scratch is released on return: wait for the writes that read it
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return ROSKO_ERR_CUDA;
  return ROSKO_OK;
}

// out[c][r] = in[r][c] for an R x C matrix of E-byte elements (row-major,
// leading dimensions ld_in / ld_out); 32 x 32 tiles through shared memory.
template <class E>
__global__ void transpose_kernel(const E* __restrict__ in, int64_t R, int64_t C, int64_t ld_in,
                                 E* __restrict__ out, int64_t ld_out) {
  __shared__ E tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int64_t r = r0 + j, c = c0 + threadIdx.x;
    if (r < R && c < C) tile[j][threadIdx.x] = in[r * ld_in + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int64_t c = c0 + j, r = r0 + threadIdx.x;
    if (r < R && c < C) out[c * ld_out + r] = tile[threadIdx.x][j];
  }
}

}  // namespace

// Dense K x M transpose of a row-major M x K matrix into `out` (ld = M).
rosko_status transpose_impl(const void* A, rosko_dtype dt, int64_t M, int64_t K, int64_t lda,
                            void* out, cudaStream_t st) {
  if (M == 0 || K == 0) return ROSKO_OK;
  const dim3 grid((unsigned)((K + 31) / 32), (unsigned)((M + 31) / 32));
  if (grid.y > 65535) return ROSKO_ERR_INVALID_ARG;
  const dim3 block(32, 8);
  const size_t es = dtype_size(dt);
  if (es == 4)
    transpose_kernel<uint32_t><<<grid, block, 0, st>>>(static_cast<const uint32_t*>(A), M, K, lda,
                                                       static_cast<uint32_t*>(out), M);
  else if (es == 2)
    transpose_kernel<uint16_t><<<grid, block, 0, st>>>(static_cast<const uint16_t*>(A), M, K, lda,
                                                       static_cast<uint16_t*>(out), M);
  else
    transpose_kernel<uint8_t><<<grid, block, 0, st>>>(static_cast<const uint8_t*>(A), M, K, lda,
                                                      static_cast<uint8_t*>(out), M);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
}

rosko_status pack_impl(const void* A, rosko_dtype a_dt, int64_t M, int64_t K, int64_t lda,
                       rosko_dtype p_dt, const float* row_scale_in, int32_t m_r,
                       int32_t dense_min_pm, cudaStream_t stream, rosko_packed_s** out) {
  rosko_packed_s* h = new (std::nothrow) rosko_packed_s();
  if (!h) return ROSKO_ERR_OOM;
  cudaGetDevice(&h->device);
  h->M = M;
  h->K = K;
  h->m_r = m_r;
  h->P = (M + m_r - 1) / m_r;
  h->dt = p_dt;
  rosko_status s = ROSKO_ERR_UNSUPPORTED;
  const int32_t dm = dense_min_pm;
  if (a_dt == ROSKO_F32 && p_dt == ROSKO_F32)
    s = pack_typed<float, float>((const float*)A, lda, nullptr, false, dm, h, stream);
  else if (a_dt == ROSKO_F32 && p_dt == ROSKO_BF16)
    s = pack_typed<float, __nv_bfloat16>((const float*)A, lda, nullptr, false, dm, h, stream);
  else if (a_dt == ROSKO_F32 && p_dt == ROSKO_F64)
    s = pack_typed<float, double>((const float*)A, lda, nullptr, false, dm, h, stream);
  else if (a_dt == ROSKO_F32 && p_dt == ROSKO_I8)
    s = pack_typed<float, int8_t>((const float*)A, lda, nullptr, true, dm, h, stream);
  else if (a_dt == ROSKO_BF16 && p_dt == ROSKO_BF16)
    s = pack_typed<__nv_bfloat16, __nv_bfloat16>((const __nv_bfloat16*)A, lda, nullptr, false, dm,
                                                 h, stream);
  else if (a_dt == ROSKO_I8 && p_dt == ROSKO_I8)
    s = pack_typed<int8_t, int8_t>((const int8_t*)A, lda, row_scale_in, false, dm, h, stream);
  if (s != ROSKO_OK) {
    pool_free(h->base, stream);
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
      unpack_kernel<float><<<g, 256, 0, st>>>(h->panel_col, h->colrec, h->nz, h->m_r, lda,
                                              (float*)A_out);
      break;
    case ROSKO_BF16:
      unpack_kernel<__nv_bfloat16><<<g, 256, 0, st>>>(h->panel_col, h->colrec, h->nz, h->m_r,
                                                      lda, (__nv_bfloat16*)A_out);
      break;
    case ROSKO_I8:
      unpack_kernel<int8_t><<<g, 256, 0, st>>>(h->panel_col, h->colrec, h->nz, h->m_r, lda,
                                               (int8_t*)A_out);
      break;
    case ROSKO_F64:
      unpack_kernel<double><<<g, 256, 0, st>>>(h->panel_col, h->colrec, h->nz, h->m_r, lda,
                                               (double*)A_out);
      break;
    default:
      return ROSKO_ERR_UNSUPPORTED;
  }
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
}

}  // namespace rosko
