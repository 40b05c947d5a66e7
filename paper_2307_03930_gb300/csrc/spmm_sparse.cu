// Sparse SpMM on CUDA cores: Alg. 2 (packed row-skipping outer product).
//
// Mapping of Alg. 2 and the tiling of Sec. 4.2 onto one SM:
//   * one warp owns one packed row panel (m_r = R rows) and keeps the
//     R x (32 V) C tile in registers (each lane: R rows x V columns) for the
//     whole K range (K-first schedule, Sec. 2.2 / 4.2);
//   * a CTA is W such warps (m_c = W R rows of C) plus one producer warp that
//     streams k_c x n_r slabs of B into shared memory with TMA, through a ring
//     of `stages` buffers guarded by full/empty mbarriers (the B block that
//     Sec. 4.2 broadcasts from L3 to the cores);
//   * for every packed column k of its panel inside the slab a warp loads the
//     B row segment once into registers ("load the B row", Alg. 2) and, for
//     each of the column's nonzeros, multiply-accumulates it into the C row
//     named by loc_m.  Registers cannot be indexed at run time, so the row is
//     resolved by a warp-uniform switch over the R register rows (all lanes
//     share the nonzero, so there is no divergence);
//   * C is written once at the end (or added with atomics when K is split
//     across CTAs).
#include <algorithm>

#include "handle.hpp"

namespace rosko {
namespace {

struct SparseParams {
  const int32_t* panel_col;
  const int32_t* col_ind;
  const int32_t* col_start;
  const void* vals;
  const uint8_t* rows;
  const float* row_scale;
  const float* col_scale;
  void* C;
  int64_t ldc, M, N, P;
  int W, KC, stages, split, slabs_total;
  int load_c_first, add_c_at_end, atomic_out, vec_ok;
  int* status;
};

template <class T> struct AccOf;
template <> struct AccOf<float> { using type = float; };
template <> struct AccOf<__nv_bfloat16> { using type = float; };
template <> struct AccOf<int8_t> { using type = int32_t; };
template <> struct AccOf<double> { using type = double; };

__device__ __forceinline__ float to_acc(float x, float) { return x; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 x, float) { return __bfloat162float(x); }
__device__ __forceinline__ int32_t to_acc(int8_t x, int32_t) { return (int32_t)x; }
__device__ __forceinline__ double to_acc(double x, double) { return x; }
__device__ __forceinline__ double to_acc(float x, double) { return (double)x; }

__device__ __forceinline__ float mac(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mac(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ int32_t mac(int32_t a, int32_t b, int32_t c) { return a * b + c; }

// V consecutive elements of a staged B row into accumulator-typed registers.
template <class TB, class TACC, int V>
__device__ __forceinline__ void load_b(const TB* __restrict__ src, TACC (&b)[V]) {
  constexpr int BYTES = V * (int)sizeof(TB);
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16 || BYTES == 32,
                "B segment must be 4, 8, 16 or 32 bytes");
  TB tmp[V];
  if constexpr (BYTES == 32) {
    reinterpret_cast<uint4*>(tmp)[0] = reinterpret_cast<const uint4*>(src)[0];
    reinterpret_cast<uint4*>(tmp)[1] = reinterpret_cast<const uint4*>(src)[1];
  } else if constexpr (BYTES == 16) {
    *reinterpret_cast<uint4*>(tmp) = *reinterpret_cast<const uint4*>(src);
  } else if constexpr (BYTES == 8) {
    *reinterpret_cast<uint2*>(tmp) = *reinterpret_cast<const uint2*>(src);
  } else {
    *reinterpret_cast<uint32_t*>(tmp) = *reinterpret_cast<const uint32_t*>(src);
  }
#pragma unroll
  for (int v = 0; v < V; ++v) b[v] = to_acc(tmp[v], TACC(0));
}

// acc[r][:] += a * b[:] for a run-time, warp-uniform row r < R.
template <int R, int V, class TACC>
__device__ __forceinline__ void row_mac(TACC (&acc)[R][V], int r, TACC a, const TACC (&b)[V]) {
#define ROSKO_ROW(j)                                              \
  case j:                                                         \
    if constexpr (j < R) {                                        \
      _Pragma("unroll") for (int v = 0; v < V; ++v) acc[j][v] =   \
          mac(a, b[v], acc[j][v]);                                \
    }                                                             \
    break;
  switch (r) {
    ROSKO_ROW(0) ROSKO_ROW(1) ROSKO_ROW(2) ROSKO_ROW(3) ROSKO_ROW(4) ROSKO_ROW(5)
    ROSKO_ROW(6) ROSKO_ROW(7) ROSKO_ROW(8) ROSKO_ROW(9) ROSKO_ROW(10) ROSKO_ROW(11)
    ROSKO_ROW(12) ROSKO_ROW(13) ROSKO_ROW(14) ROSKO_ROW(15) ROSKO_ROW(16) ROSKO_ROW(17)
    ROSKO_ROW(18) ROSKO_ROW(19) ROSKO_ROW(20) ROSKO_ROW(21) ROSKO_ROW(22) ROSKO_ROW(23)
    ROSKO_ROW(24) ROSKO_ROW(25) ROSKO_ROW(26) ROSKO_ROW(27) ROSKO_ROW(28) ROSKO_ROW(29)
    ROSKO_ROW(30) ROSKO_ROW(31)
    default:
      __builtin_unreachable();
  }
#undef ROSKO_ROW
}

template <class TC, class TACC>
__device__ __forceinline__ TC out_value(TACC acc, const SparseParams&, int64_t, int64_t) {
  return (TC)acc;
}
// INT8 x INT8 -> FP32: dequantise with the row scale of A and column scale of B.
template <>
__device__ __forceinline__ float out_value<float, int32_t>(int32_t acc, const SparseParams& p,
                                                           int64_t row, int64_t col) {
  return ((float)acc * p.row_scale[row]) * p.col_scale[col];
}

template <class TC>
__device__ __forceinline__ void atomic_add_out(TC* dst, TC v) {
  atomicAdd(dst, v);
}

template <class TA, class TB, class TC, int R, int V>
__global__ void __launch_bounds__(288, 1)
    sparse_spmm_kernel(const SparseParams p, const __grid_constant__ CUtensorMap tmB) {
  using TACC = typename AccOf<TA>::type;
  constexpr int NR = 32 * V;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + p.stages;
  TB* Bs = reinterpret_cast<TB*>(smem + 1024);
  const size_t stage_elems = (size_t)p.KC * NR;

  const int W = p.W;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n0 = (int64_t)blockIdx.y * NR;
  const int s_per = (p.slabs_total + p.split - 1) / p.split;
  const int s_begin = (int)blockIdx.z * s_per;
  const int nslabs = max(0, min(p.slabs_total, s_begin + s_per) - s_begin);

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], W);
    }
    fence_barrier_init();
  }
  __syncthreads();

  if (warp == W) {
    // ---------------- producer: TMA ring over the K slabs of this split -----
    if (lane == 0 && nslabs > 0) {
      prefetch_tensormap(&tmB);
      const uint32_t bytes = (uint32_t)(stage_elems * sizeof(TB));
      int i = 0;
      bool ok = true;
      for (; i < nslabs; ++i) {
        const int st = i % p.stages;
        const uint32_t ph = (uint32_t)(i / p.stages) & 1u;
        if (i >= p.stages && !mbar_wait_bounded(&empty[st], ph ^ 1u, p.status)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&full[st], bytes);
        tma_load_2d(Bs + st * stage_elems, &tmB, (int32_t)n0, (s_begin + i) * p.KC, &full[st]);
      }
      if (!ok) {
        // consumers gave up: wait (bounded) for our copies in flight to land
        for (int j = max(0, i - p.stages); j < i; ++j)
          mbar_wait_bounded(&full[j % p.stages], (uint32_t)(j / p.stages) & 1u, p.status);
      }
    }
    return;
  }

  // ---------------- consumers: one packed row panel per warp -----------------
  const int64_t panel = (int64_t)blockIdx.x * W + warp;
  const bool has_panel = panel < p.P;
  const int64_t row0 = panel * R;
  TACC acc[R][V];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int v = 0; v < V; ++v) acc[r][v] = TACC(0);

  TC* C = reinterpret_cast<TC*>(p.C);
  const int64_t col0 = n0 + lane * V;
  if (has_panel && p.load_c_first) {
    // Alg. 2 loads the C rows into registers before the outer products
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t row = row0 + r;
      if (row < p.M)
#pragma unroll
        for (int v = 0; v < V; ++v)
          if (col0 + v < p.N) acc[r][v] = (TACC)C[row * p.ldc + col0 + v];
    }
  }

  int c = 0, c_end = 0;
  if (has_panel) {
    c = __ldg(&p.panel_col[panel]);
    c_end = __ldg(&p.panel_col[panel + 1]);
    if (s_begin > 0) {  // first packed column of this split's K range
      const int kb = s_begin * p.KC;
      int lo = c, hi = c_end;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&p.col_ind[mid]) < kb) lo = mid + 1; else hi = mid;
      }
      c = lo;
    }
  }
  const TA* __restrict__ vals = reinterpret_cast<const TA*>(p.vals);
  const uint8_t* __restrict__ rows = p.rows;

  for (int i = 0; i < nslabs; ++i) {
    const int st = i % p.stages;
    const uint32_t ph = (uint32_t)(i / p.stages) & 1u;
    if (!mbar_wait_bounded(&full[st], ph, p.status)) return;
    const int kbase = (s_begin + i) * p.KC;
    const int kend = kbase + p.KC;
    const TB* bs = Bs + st * stage_elems + lane * V;
    while (c < c_end) {
      const int k = __ldg(&p.col_ind[c]);
      if (k >= kend) break;
      TACC b[V];
      load_b<TB, TACC, V>(bs + (size_t)(k - kbase) * NR, b);
      const int e1 = __ldg(&p.col_start[c + 1]);
      int e = __ldg(&p.col_start[c]);
      // one nonzero of look-ahead hides the load latency behind the switch
      TACC a_next = to_acc(vals[e], TACC(0));
      int r_next = rows[e];
      for (; e < e1; ++e) {
        const TACC a = a_next;
        const int r = r_next & (R - 1);
        if (e + 1 < e1) {
          a_next = to_acc(vals[e + 1], TACC(0));
          r_next = rows[e + 1];
        }
        row_mac<R, V, TACC>(acc, r, a, b);
      }
      ++c;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
  }
  if (!has_panel) return;

  // ---------------- epilogue: C written once ---------------------------------
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t row = row0 + r;
    if (row >= p.M) break;
    TC* crow = C + row * p.ldc;
    if (p.atomic_out) {
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (col0 + v < p.N) atomic_add_out(crow + col0 + v, out_value<TC, TACC>(acc[r][v], p, row, col0 + v));
      continue;
    }
    TC o[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      o[v] = (col0 + v < p.N) ? out_value<TC, TACC>(acc[r][v], p, row, col0 + v) : TC(0);
      if (p.add_c_at_end && col0 + v < p.N) o[v] = o[v] + crow[col0 + v];
    }
    constexpr int OB = V * (int)sizeof(TC);
    if (p.vec_ok && col0 + V <= p.N && (OB == 16 || OB == 8 || OB == 32)) {
      if constexpr (OB == 32) {
        reinterpret_cast<uint4*>(crow + col0)[0] = reinterpret_cast<uint4*>(o)[0];
        reinterpret_cast<uint4*>(crow + col0)[1] = reinterpret_cast<uint4*>(o)[1];
      } else if constexpr (OB == 16) {
        *reinterpret_cast<uint4*>(crow + col0) = *reinterpret_cast<uint4*>(o);
      } else if constexpr (OB == 8) {
        *reinterpret_cast<uint2*>(crow + col0) = *reinterpret_cast<uint2*>(o);
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (col0 + v < p.N) crow[col0 + v] = o[v];
    }
  }
}

using KernelFn = void (*)(const SparseParams, const CUtensorMap);

struct Entry {
  rosko_dtype a, b, c;
  int R, V;
  KernelFn fn;
  size_t smem_set;
};

#define ROSKO_ENTRY(TA, TB, TC, DA, DB, DC, R, V) \
  {DA, DB, DC, R, V, sparse_spmm_kernel<TA, TB, TC, R, V>, 0}

Entry g_table[] = {
    ROSKO_ENTRY(float, float, float, ROSKO_F32, ROSKO_F32, ROSKO_F32, 32, 4),
    ROSKO_ENTRY(float, float, float, ROSKO_F32, ROSKO_F32, ROSKO_F32, 16, 8),
    ROSKO_ENTRY(float, float, float, ROSKO_F32, ROSKO_F32, ROSKO_F32, 16, 4),
    ROSKO_ENTRY(float, float, float, ROSKO_F32, ROSKO_F32, ROSKO_F32, 8, 8),
    ROSKO_ENTRY(__nv_bfloat16, __nv_bfloat16, float, ROSKO_BF16, ROSKO_BF16, ROSKO_F32, 32, 4),
    ROSKO_ENTRY(__nv_bfloat16, __nv_bfloat16, float, ROSKO_BF16, ROSKO_BF16, ROSKO_F32, 16, 8),
    ROSKO_ENTRY(__nv_bfloat16, __nv_bfloat16, float, ROSKO_BF16, ROSKO_BF16, ROSKO_F32, 8, 8),
    ROSKO_ENTRY(int8_t, int8_t, int32_t, ROSKO_I8, ROSKO_I8, ROSKO_I32, 32, 4),
    ROSKO_ENTRY(int8_t, int8_t, int32_t, ROSKO_I8, ROSKO_I8, ROSKO_I32, 16, 8),
    ROSKO_ENTRY(int8_t, int8_t, int32_t, ROSKO_I8, ROSKO_I8, ROSKO_I32, 8, 8),
    ROSKO_ENTRY(int8_t, int8_t, float, ROSKO_I8, ROSKO_I8, ROSKO_F32, 32, 4),
    ROSKO_ENTRY(int8_t, int8_t, float, ROSKO_I8, ROSKO_I8, ROSKO_F32, 16, 8),
    ROSKO_ENTRY(int8_t, int8_t, float, ROSKO_I8, ROSKO_I8, ROSKO_F32, 8, 8),
    ROSKO_ENTRY(double, float, double, ROSKO_F64, ROSKO_F32, ROSKO_F64, 32, 2),
    ROSKO_ENTRY(double, float, double, ROSKO_F64, ROSKO_F32, ROSKO_F64, 16, 4),
    ROSKO_ENTRY(double, float, double, ROSKO_F64, ROSKO_F32, ROSKO_F64, 8, 4),
};

Entry* find_entry(rosko_dtype a, rosko_dtype b, rosko_dtype c, int R, int V) {
  for (auto& e : g_table)
    if (e.a == a && e.b == b && e.c == c && e.R == R && e.V == V) return &e;
  return nullptr;
}

CUtensorMapDataType tmap_dtype(rosko_dtype d) {
  switch (d) {
    case ROSKO_F32: return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    case ROSKO_BF16: return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    default: return CU_TENSOR_MAP_DATA_TYPE_UINT8;
  }
}

}  // namespace

bool sparse_config_supported(rosko_dtype p_dt, rosko_dtype b_dt, rosko_dtype c_dt, int R, int V) {
  return find_entry(p_dt, b_dt, c_dt, R, V) != nullptr;
}

int sparse_default_V(rosko_dtype p_dt, int R) {
  switch (p_dt) {
    case ROSKO_F64: return R == 32 ? 2 : 4;
    case ROSKO_F32: return R == 32 ? 4 : 8;
    default: return R == 32 ? 4 : 8;
  }
}

size_t sparse_smem_bytes(rosko_dtype b_dt, int V, int KC, int stages) {
  return 1024 + (size_t)stages * KC * 32 * V * dtype_size(b_dt);
}

rosko_status sparse_spmm_launch(rosko_packed_s* h, const void* B, rosko_dtype b_dt, int64_t N,
                                int64_t ldb, const float* col_scale, void* C, rosko_dtype c_dt,
                                int64_t ldc, int accumulate, const SparseLaunch& L,
                                cudaStream_t st) {
  Entry* e = find_entry(h->dt, b_dt, c_dt, L.R, L.V);
  if (!e) return ROSKO_ERR_UNSUPPORTED;
  const int NR = 32 * L.V;
  const size_t bsz = dtype_size(b_dt), csz = dtype_size(c_dt);
  const size_t smem = sparse_smem_bytes(b_dt, L.V, L.KC, L.stages);
  if (smem > e->smem_set) {
    if (cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return ROSKO_ERR_CUDA;
    e->smem_set = smem;
  }

  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)h->K};
  const cuuint64_t strides[1] = {(cuuint64_t)ldb * bsz};
  const cuuint32_t box[2] = {(cuuint32_t)NR, (cuuint32_t)L.KC};
  const cuuint32_t es[2] = {1, 1};
  CUresult r = encode_tiled(&map, tmap_dtype(b_dt), 2, const_cast<void*>(B), dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return ROSKO_ERR_INVALID_ARG;

  SparseParams p{};
  p.panel_col = h->panel_col;
  p.col_ind = h->col_ind;
  p.col_start = h->col_start;
  p.vals = h->vals;
  p.rows = h->rows;
  p.row_scale = h->row_scale;
  p.col_scale = col_scale;
  p.C = C;
  p.ldc = ldc;
  p.M = h->M;
  p.N = N;
  p.P = h->P;
  p.W = L.W;
  p.KC = L.KC;
  p.stages = L.stages;
  p.split = L.split;
  p.slabs_total = (int)((h->K + L.KC - 1) / L.KC);
  const bool dequant = (h->dt == ROSKO_I8 && c_dt == ROSKO_F32);
  p.atomic_out = L.split > 1;
  p.load_c_first = accumulate && !p.atomic_out && !dequant;
  p.add_c_at_end = accumulate && !p.atomic_out && dequant;
  p.vec_ok = ((reinterpret_cast<uintptr_t>(C) % 16) == 0) && ((ldc * csz) % 16 == 0);
  p.status = device_status_word();
  if (!p.status) return ROSKO_ERR_CUDA;

  if (p.atomic_out && !accumulate) {
    if (cudaMemset2DAsync(C, (size_t)ldc * csz, 0, (size_t)N * csz, (size_t)h->M, st) !=
        cudaSuccess)
      return ROSKO_ERR_CUDA;
  }
  const dim3 grid((unsigned)((h->P + L.W - 1) / L.W), (unsigned)((N + NR - 1) / NR),
                  (unsigned)L.split);
  e->fn<<<grid, (L.W + 1) * 32, smem, st>>>(p, map);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
}

}  // namespace rosko
