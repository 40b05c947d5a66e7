// Sparse SpMM on CUDA cores: Alg. 2 (packed row-skipping outer product).
//
// Mapping of Alg. 2 and the tiling of Sec. 4.2 onto one SM:
//   * one warp owns one packed row panel (m_r = R rows) and keeps an
//     R x (32 V) tile of C in registers (each lane: R rows x V columns) for
//     the whole K range of its CTA (K-first schedule, Sec. 2.2 / 4.2);
//   * a CTA is W such warps (m_c = W R rows of C) plus one producer warp that
//     streams k_c x n_r slabs of B into shared memory with TMA through a ring
//     of `stages` buffers guarded by full/empty mbarriers (the B block that
//     Sec. 4.2 broadcasts from L3 to the cores);
//   * for every packed column k of its panel inside the slab a warp loads the
//     B row segment once into registers ("load the B row", Alg. 2) and, for
//     each of the column's nonzeros, multiply-accumulates it into the C row
//     named by loc_m.  Registers cannot be indexed at run time, so the row is
//     resolved by a warp-uniform switch over the R register rows (all lanes
//     share the nonzero, so there is no divergence).  Each dispatch feeds V
//     FMAs per lane, so wide strips (V = 8..16) amortise it;
//   * a lane's V columns are V/CE chunks of CE = 16 bytes / sizeof(B) values
//     spaced 32 CE apart, so every shared-memory load of the warp reads one
//     contiguous 512-byte run (conflict free);
//   * C is written once at the end (or added with atomics when K is split
//     across CTAs).
#include <type_traits>
#include <algorithm>
#include <climits>
#include <cstring>
#include <cstdlib>

#include "handle.hpp"

namespace rosko {
namespace {

struct SparseParams {
  const int32_t* panel_list;  // panels to process (NULL: 0 .. n_list-1)
  int64_t n_list;
  const int32_t* panel_col;
  const int2* colrec;
  const void* nz;
  const int32_t* rowptr;  // row-slot stream
  const void* rnz;
  const int32_t* gu_start;  // gather stream (order 3)
  const int32_t* gu_k;
  const void* gnz;
  const float* row_scale;
  const float* col_scale;
  void* C;
  int64_t ldc, M, N, P;
  int W, KC, stages, split, slabs_total, boxes;
  int load_c_first, add_c_at_end, atomic_out, vec_ok;
  int* status;
};

template <class T> struct AccOf;
template <> struct AccOf<float> { using type = float; };
template <> struct AccOf<__nv_bfloat16> { using type = float; };
template <> struct AccOf<int8_t> { using type = int32_t; };
template <> struct AccOf<double> { using type = double; };

// Nonzero records (see handle.hpp) and their decoding.
template <class TA> struct Rec;
template <> struct Rec<float> {
  using T = uint2;
  __device__ static float a(T w) { return __uint_as_float(w.y); }
  __device__ static int r(T w) { return (int)w.x; }
};
template <> struct Rec<__nv_bfloat16> {
  using T = uint32_t;
  __device__ static float a(T w) { return __uint_as_float(w & 0xFFFF0000u); }
  __device__ static int r(T w) { return (int)(w & 0xFFFFu); }
};
template <> struct Rec<int8_t> {
  using T = uint32_t;
  __device__ static int32_t a(T w) { return (int32_t)(int8_t)(uint8_t)(w >> 16); }
  __device__ static int r(T w) { return (int)(w & 0xFFFFu); }
};
template <> struct Rec<double> {
  using T = RecF64;
  __device__ static double a(const T& w) { return w.a; }
  __device__ static int r(const T& w) { return w.r; }
};

// Row-slot records (value + column k, see handle.hpp) and their decoding.
template <class TA> struct RowRec;
template <> struct RowRec<float> {
  using T = uint2;
  __device__ static float a(T w) { return __uint_as_float(w.y); }
  __device__ static int k(T w) { return (int)w.x; }
};
template <> struct RowRec<__nv_bfloat16> {
  using T = uint32_t;
  __device__ static float a(T w) { return __uint_as_float(w & 0xFFFF0000u); }
  __device__ static int k(T w) { return (int)(w & 0xFFFFu); }
};
template <> struct RowRec<int8_t> {
  using T = uint32_t;
  __device__ static int32_t a(T w) { return (int32_t)(int8_t)(uint8_t)(w >> 16); }
  __device__ static int k(T w) { return (int)(w & 0xFFFFu); }
};
template <> struct RowRec<double> {
  using T = RecF64;
  __device__ static double a(const T& w) { return w.a; }
  __device__ static int k(const T& w) { return w.r; }
};

__device__ __forceinline__ float to_acc(float x, float) { return x; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 x, float) { return __bfloat162float(x); }
__device__ __forceinline__ int32_t to_acc(int8_t x, int32_t) { return (int32_t)x; }
__device__ __forceinline__ double to_acc(float x, double) { return (double)x; }

__device__ __forceinline__ float mac(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mac(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ int32_t mac(int32_t a, int32_t b, int32_t c) { return a * b + c; }

// CE consecutive B elements (CE * sizeof(TB) = 4, 8 or 16 bytes) into registers.
template <class TB, class TACC, int CE>
__device__ __forceinline__ void load_chunk(const TB* __restrict__ src, TACC* b) {
  constexpr int BYTES = CE * (int)sizeof(TB);
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "chunk must be 4, 8 or 16 bytes");
  TB tmp[CE];
  if constexpr (BYTES == 16) {
    *reinterpret_cast<uint4*>(tmp) = *reinterpret_cast<const uint4*>(src);
  } else if constexpr (BYTES == 8) {
    *reinterpret_cast<uint2*>(tmp) = *reinterpret_cast<const uint2*>(src);
  } else {
    *reinterpret_cast<uint32_t*>(tmp) = *reinterpret_cast<const uint32_t*>(src);
  }
#pragma unroll
  for (int v = 0; v < CE; ++v) b[v] = to_acc(tmp[v], TACC(0));
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

template <class TC, int CE>
__device__ __forceinline__ void store_chunk(TC* dst, const TC* o) {
  constexpr int OB = CE * (int)sizeof(TC);
  if constexpr (OB % 16 == 0) {
#pragma unroll
    for (int i = 0; i < OB / 16; ++i)
      reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(o)[i];
  } else if constexpr (OB == 8) {
    *reinterpret_cast<uint2*>(dst) = *reinterpret_cast<const uint2*>(o);
  } else {
#pragma unroll
    for (int i = 0; i < CE; ++i) dst[i] = o[i];
  }
}

template <class TA, class TB, class TC, int R, int V, int ORDER>
__global__ void __launch_bounds__(288, 1)
    sparse_spmm_kernel(const SparseParams p, const __grid_constant__ CUtensorMap tmB,
                       const __grid_constant__ CUtensorMap tmB1) {
  using TACC = typename AccOf<TA>::type;
  using RT = typename Rec<TA>::T;
  constexpr int NR = 32 * V;
  // a lane chunk is at most 16 bytes and at most 8 elements, so that the
  // warp's 32 chunks (<= 256 elements) never straddle a TMA box
  constexpr int G = (16 / (int)sizeof(TB)) < 8 ? (16 / (int)sizeof(TB)) : 8;
  constexpr int CE = V < G ? V : G;                // elements per lane chunk
  constexpr int J = V / CE;                        // chunks per lane
  constexpr int BOXW = NR > 256 ? 256 : NR;        // width of one TMA box
  static_assert(J * CE == V, "V must be a multiple of the chunk width");
  static_assert(BOXW % (32 * CE) == 0, "warp chunks must tile a box");
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + p.stages;
  TB* Bs = reinterpret_cast<TB*>(smem + 1024);
  const size_t stage_elems = (size_t)p.KC * NR;

  const int W = p.W;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n0 = (int64_t)blockIdx.y * NR;
  // order 3: this CTA is one 128-row tile and its slabs are slots of the
  // tile's touched-column list
  int64_t tile = 0;
  int ustart = 0, ulen = 0;
  int slabs_total = p.slabs_total;
  if constexpr (ORDER == 3) {
    tile = p.panel_list ? (int64_t)__ldg(&p.panel_list[blockIdx.x]) : (int64_t)blockIdx.x;
    ustart = __ldg(&p.gu_start[tile]);
    ulen = __ldg(&p.gu_start[tile + 1]) - ustart;
    slabs_total = (ulen + p.KC - 1) / p.KC;
  }
  const int s_per = (slabs_total + p.split - 1) / p.split;
  const int s_begin = (int)blockIdx.z * s_per;
  const int nslabs = max(0, min(slabs_total, s_begin + s_per) - s_begin);

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], W);
    }
    fence_barrier_init();
  }
  __syncthreads();

  if (ORDER == 3 && warp == W) {
    // ---------------- producer (order 3): gather the tile's touched B rows ---
    // slab i holds slots [(s_begin+i) k_c, +k_c) of the tile's column list;
    // the 32 lanes fetch their column indices and issue one row copy each
    if (nslabs > 0) {
      if (lane == 0) prefetch_tensormap(&tmB1);
      const int box_w = BOXW;
      int i = 0;
      bool ok = true;
      for (; i < nslabs; ++i) {
        const int st = i % p.stages;
        const uint32_t ph = (uint32_t)(i / p.stages) & 1u;
        if (i >= p.stages && !mbar_wait_bounded(&empty[st], ph ^ 1u, p.status)) {
          ok = false;
          break;
        }
        const int slot0 = (s_begin + i) * p.KC;
        const int rows = min(p.KC, ulen - slot0);
        if (lane == 0)
          mbar_arrive_expect_tx(&full[st], (uint32_t)(rows * NR * (int)sizeof(TB)));
        __syncwarp();
        for (int j = lane; j < rows; j += 32) {
          const int k = __ldg(&p.gu_k[ustart + slot0 + j]);
          for (int bx = 0; bx < p.boxes; ++bx)
            tma_load_2d(Bs + st * stage_elems + (size_t)bx * box_w * p.KC + (size_t)j * box_w,
                        &tmB1, (int32_t)(n0 + bx * box_w), k, &full[st]);
        }
      }
      if (!ok && lane == 0) {
        for (int j = max(0, i - p.stages); j < i; ++j)
          mbar_wait_bounded(&full[j % p.stages], (uint32_t)(j / p.stages) & 1u, p.status);
      }
    }
    return;
  }
  if (warp == W) {
    // ---------------- producer: TMA ring over the K slabs of this split -----
    if (lane == 0 && nslabs > 0) {
      prefetch_tensormap(&tmB);
      const uint32_t bytes = (uint32_t)(stage_elems * sizeof(TB));
      const int box_w = BOXW;
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
        for (int bx = 0; bx < p.boxes; ++bx)
          tma_load_2d(Bs + st * stage_elems + (size_t)bx * box_w * p.KC, &tmB,
                      (int32_t)(n0 + bx * box_w), (s_begin + i) * p.KC, &full[st]);
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
  int64_t panel = 0;
  bool has_panel = false;
  if constexpr (ORDER == 3) {
    panel = tile * W + warp;
    has_panel = panel < p.P;
  } else {
    const int64_t slot = (int64_t)blockIdx.x * W + warp;
    has_panel = slot < p.n_list;
    panel = !has_panel ? 0 : (p.panel_list ? (int64_t)__ldg(&p.panel_list[slot]) : slot);
  }
  const int64_t row0 = panel * R;
  TACC acc[R][V];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int v = 0; v < V; ++v) acc[r][v] = TACC(0);

  TC* C = reinterpret_cast<TC*>(p.C);
  if (has_panel && p.load_c_first) {
    // Alg. 2 loads the C rows into registers before the outer products
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t row = row0 + r;
      if (row < p.M)
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
          for (int v = 0; v < CE; ++v) {
            const int64_t col = n0 + j * 32 * CE + lane * CE + v;
            if (col < p.N) acc[r][j * CE + v] = (TACC)C[row * p.ldc + col];
          }
    }
  }

  if constexpr (ORDER == 1) {
    // ---- column order (Alg. 2): one B row per packed column, C row by switch
    int c = 0, c_end = 0;
    if (has_panel) {
      c = __ldg(&p.panel_col[panel]);
      c_end = __ldg(&p.panel_col[panel + 1]);
      if (s_begin > 0) {  // first packed column of this split's K range
        const int kb = s_begin * p.KC;
        int lo = c, hi = c_end;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (__ldg(&p.colrec[mid].x) < kb) lo = mid + 1; else hi = mid;
        }
        c = lo;
      }
    }
    const RT* __restrict__ nz = reinterpret_cast<const RT*>(p.nz);
    const int2* __restrict__ colrec = p.colrec;
    // current column record (k = INT_MAX once the panel is exhausted)
    int2 cur = (c < c_end) ? __ldg(&colrec[c]) : make_int2(INT_MAX, 0);

    for (int i = 0; i < nslabs; ++i) {
      const int st = i % p.stages;
      const uint32_t ph = (uint32_t)(i / p.stages) & 1u;
      if (!mbar_wait_bounded(&full[st], ph, p.status)) return;
      const int kbase = (s_begin + i) * p.KC;
      const int kend = kbase + p.KC;
      const TB* bs = Bs + st * stage_elems + lane * CE;
      while (cur.x < kend) {
        const int2 nxt = __ldg(&colrec[c + 1]);   // its start ends this column
        TACC b[V];
        // slab layout: [box][k_c rows][BOXW]
        const TB* brow = bs + (size_t)(cur.x - kbase) * BOXW;
#pragma unroll
        for (int j = 0; j < J; ++j)
          load_chunk<TB, TACC, CE>(brow + (size_t)((j * 32 * CE) / BOXW) * p.KC * BOXW +
                                       (j * 32 * CE) % BOXW,
                                   b + j * CE);
        int e = cur.y;
        const int e1 = nxt.y;
        RT w = nz[e];
        for (; e + 1 < e1; ++e) {
          const RT w2 = nz[e + 1];   // look-ahead hides the load behind the FMAs
          row_mac<R, V, TACC>(acc, Rec<TA>::r(w) & (R - 1), Rec<TA>::a(w), b);
          w = w2;
        }
        row_mac<R, V, TACC>(acc, Rec<TA>::r(w) & (R - 1), Rec<TA>::a(w), b);
        ++c;
        cur = (c < c_end) ? nxt : make_int2(INT_MAX, 0);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
  } else {
    // ---- row-slot order: register row r of C walks its own nonzeros (k
    // ascending) and reads each one's B row from the shared slab; no run-time
    // register indexing, rows are independent instruction streams
    using WT = typename RowRec<TA>::T;
    // order 3 reads the same records re-addressed by tile-list slot
    const WT* __restrict__ rnz = reinterpret_cast<const WT*>(ORDER == 3 ? p.gnz : p.rnz);
    int cur[R];
    WT nxt[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t row = row0 + r;
      int c0 = 0;
      if (has_panel && row < p.M) {
        c0 = __ldg(&p.rowptr[row]);
        if (s_begin > 0) {  // first nonzero of this split's K range
          const int kb = s_begin * p.KC;
          int lo = c0, hi = __ldg(&p.rowptr[row + 1]) - 1;   // last entry: sentinel
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (RowRec<TA>::k(rnz[mid]) < kb) lo = mid + 1; else hi = mid;
          }
          c0 = lo;
        }
        nxt[r] = rnz[c0];
      } else {
        // rows past M (or no panel): point at a sentinel of this handle
        c0 = __ldg(&p.rowptr[1]) - 1;
        nxt[r] = rnz[c0];
      }
      cur[r] = c0;
    }
    for (int i = 0; i < nslabs; ++i) {
      const int st = i % p.stages;
      const uint32_t ph = (uint32_t)(i / p.stages) & 1u;
      if (!mbar_wait_bounded(&full[st], ph, p.status)) return;
      const int kbase = (s_begin + i) * p.KC;
      const int kend = kbase + p.KC;
      const TB* bs = Bs + st * stage_elems + lane * CE;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        while (RowRec<TA>::k(nxt[r]) < kend) {
          const WT w = nxt[r];
          nxt[r] = rnz[++cur[r]];          // next record (the row ends on a sentinel)
          TACC b[V];
          const TB* brow = bs + (size_t)(RowRec<TA>::k(w) - kbase) * BOXW;
#pragma unroll
          for (int j = 0; j < J; ++j)
            load_chunk<TB, TACC, CE>(brow + (size_t)((j * 32 * CE) / BOXW) * p.KC * BOXW +
                                         (j * 32 * CE) % BOXW,
                                     b + j * CE);
          const TACC a = RowRec<TA>::a(w);
#pragma unroll
          for (int v = 0; v < V; ++v) acc[r][v] = mac(a, b[v], acc[r][v]);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
  }
  if (!has_panel) return;

  // ---------------- epilogue: C written once ---------------------------------
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t row = row0 + r;
    if (row >= p.M) break;
    TC* crow = C + row * p.ldc;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int64_t col0 = n0 + j * 32 * CE + lane * CE;
      if (col0 >= p.N) continue;
      if (p.atomic_out) {
#pragma unroll
        for (int v = 0; v < CE; ++v)
          if (col0 + v < p.N)
            atomicAdd(crow + col0 + v, out_value<TC, TACC>(acc[r][j * CE + v], p, row, col0 + v));
        continue;
      }
      TC o[CE];
#pragma unroll
      for (int v = 0; v < CE; ++v) {
        o[v] = (col0 + v < p.N) ? out_value<TC, TACC>(acc[r][j * CE + v], p, row, col0 + v)
                                : TC(0);
        if (p.add_c_at_end && col0 + v < p.N) o[v] = o[v] + crow[col0 + v];
      }
      if (p.vec_ok && col0 + CE <= p.N) {
        store_chunk<TC, CE>(crow + col0, o);
      } else {
#pragma unroll
        for (int v = 0; v < CE; ++v)
          if (col0 + v < p.N) crow[col0 + v] = o[v];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Order 4, row-direct: the row-slot traversal with B read straight from
// global memory (L2) instead of shared-memory slabs.  One warp owns one row
// of C over a 32 V-column strip and walks that row's nonzeros (k ascending,
// the same per-row order as the outer product of Alg. 2); each nonzero reads
// its B row segment once.  With very sparse A a B row staged for a panel is
// used by d*m_r << 1 rows of any panel whose C tile fits in registers, so a
// staged slab would cost shared-memory bandwidth without saving L2 reads;
// here every B byte read is used and all of B (resident in the 129 MB L2)
// serves every SM.
//
// The traversal is bound by L2 and HBM latency, not arithmetic, so the
// kernel is built to keep bytes in flight with few registers:
//   * a work segment names its record range directly ({row, e0, e_end,
//     cut}), so a warp reaches its B loads after two dependent loads (the
//     segment, then 32 records fetched one per lane, coalesced);
//   * records are broadcast by shuffles in groups of U; every lane copies its
//     own column slice of each record's B row segment into its own slots of
//     the warp's ring in shared memory (cp.async: the data in flight holds no
//     register), two groups in flight, and reads back only what it copied
//     (no barrier: each lane waits for its own copies);
//   * BF16 uses the mixed-precision FMA (BF16 x BF16 + FP32 -> FP32, one
//     rounding: the exact product added to the FP32 sum), which needs no
//     conversion instructions (measured on GB300: 58 against 35 MACs per
//     clock per SM for convert + FP32 FMA).
// Measured on the 512 x 4608 x 3136 layer (BF16): register-held batches of
// B loads reached 29 us at 99% sparsity (16 resident warps per SM, latency
// bound), this ring 19 us (24 warps per SM, twice the bytes in flight).
//
// One launch serves a batch: the problems travel in the kernel parameters
// and the items of problem q are [items0(q), items0(q+1)); an item is one
// segment x one strip, strips fastest so that neighbouring warps share the
// segment's records; a block is 8 items.
// Warp broadcast of one nonzero record from lane `src`.
__device__ __forceinline__ uint32_t shfl_rec(uint32_t w, int src) {
  return __shfl_sync(0xffffffffu, w, src);
}
__device__ __forceinline__ uint2 shfl_rec(uint2 w, int src) {
  return make_uint2(__shfl_sync(0xffffffffu, w.x, src), __shfl_sync(0xffffffffu, w.y, src));
}
__device__ __forceinline__ RecF64 shfl_rec(const RecF64& w, int src) {
  RecF64 o;
  o.a = __shfl_sync(0xffffffffu, w.a, src);
  o.r = __shfl_sync(0xffffffffu, w.r, src);
  o.pad = 0;
  return o;
}

// A register type of exactly B bytes (4, 8 or 16) for raw chunk loads.
template <int B> struct RawOf;
template <> struct RawOf<4> { using type = uint32_t; };
template <> struct RawOf<8> { using type = uint2; };
template <> struct RawOf<16> { using type = uint4; };

// c0 += a * lo(b), c1 += a * hi(b): a is the BF16 value in the high half of
// the record word, b two BF16 values of B; one rounding each.
__device__ __forceinline__ void fma_bf16x2(float& c0, float& c1, uint32_t rec, uint32_t b) {
  asm("{\n\t.reg .b16 al, ah, bl, bh;\n\t"
      "mov.b32 {al, ah}, %2;\n\t"
      "mov.b32 {bl, bh}, %3;\n\t"
      "fma.rn.f32.bf16 %0, ah, bl, %0;\n\t"
      "fma.rn.f32.bf16 %1, ah, bh, %1;\n\t}"
      : "+f"(c0), "+f"(c1)
      : "r"(rec), "r"(b));
}

struct DirectProb {
  const void* rnz;            // row stream: per-row k-ascending records + sentinel
  const SegEntry* segs;       // work segments: {row, e0, e_end, cut} + inline records
  const float* row_scale;     // INT8 dequantisation
  const float* col_scale;
  const void* B;
  void* C;
  int64_t n_segs, ldb, ldc, M, N;
  int64_t items0;             // first work item of this problem
  int strips, load_c_first, add_c_at_end, vec_ok;
};

template <int NP>
struct DirectTable {
  DirectProb p[NP];
  int64_t total;              // work items of all problems
  int count;
};

// Asynchronous copy of `bytes` (8 or 16) global -> shared, zero-filling
// past the first `src_bytes` (which may be 0: nothing is read).
template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t dst, const void* src, int src_bytes) {
  if constexpr (BYTES == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(dst), "l"(src), "n"(BYTES),
                 "r"(src_bytes)
                 : "memory");
  }
}
// Same, with an L2 eviction policy (createpolicy) for the line.
template <int BYTES>
__device__ __forceinline__ void cp_async_hint(uint32_t dst, const void* src, int src_bytes,
                                              uint64_t policy) {
  if constexpr (BYTES == 16) {
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2, %3;" ::"r"(dst),
                 "l"(src), "r"(src_bytes), "l"(policy)
                 : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], %2, %3, %4;" ::"r"(dst),
                 "l"(src), "n"(BYTES), "r"(src_bytes), "l"(policy)
                 : "memory");
  }
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// Loads of the handle's small arrays (segments, records) that should stay in
// L2 across launches while B streams through it.
__device__ __forceinline__ int4 ld_keep(const int4* p, uint64_t pol) {
  int4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint32_t ld_keep(const uint32_t* p, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint2 ld_keep(const uint2* p, uint64_t pol) {
  uint2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.b32 {%0, %1}, [%2], %3;"
               : "=r"(v.x), "=r"(v.y)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ RecF64 ld_keep(const RecF64* p, uint64_t) { return *p; }

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The warp's ring: two groups of U records; group g + 1 is in flight while
// group g is multiplied, then group g + 2 takes g's slots.  U = 8 records of
// 16 bytes per lane (4 when a lane's slice is 32 bytes, or with FP64
// accumulators): 8 KB of ring per warp, three 8-warp blocks per SM.
template <class TA, class TB, class TC, int V, int NP>
constexpr int async_batch() {
  return ((V * (int)sizeof(TB)) >= 32 || std::is_same<TA, double>::value) ? 4 : 8;
}
template <class TA, class TB, class TC, int V, int NP>
constexpr size_t async_smem_bytes() {
  return (size_t)8 * 2 * async_batch<TA, TB, TC, V, NP>() * 32 * V * sizeof(TB);
}

template <class TA, class TB, class TC, int V, int NP>
__global__ void __launch_bounds__(256, 3)
    rowdirect_kernel(const __grid_constant__ DirectTable<NP> T) {
  using TACC = typename AccOf<TA>::type;
  using WT = typename RowRec<TA>::T;
  constexpr int G = (16 / (int)sizeof(TB)) < 8 ? (16 / (int)sizeof(TB)) : 8;
  constexpr int CE = V < G ? V : G;   // elements per lane chunk (8 or 16 bytes)
  constexpr int J = V / CE;           // chunks per lane, 32 CE columns apart
  constexpr int CB = CE * (int)sizeof(TB);   // bytes per chunk
  constexpr int U = async_batch<TA, TB, TC, V, NP>();
  static_assert(J * CE == V, "V must be a multiple of the chunk width");
  static_assert(CB == 8 || CB == 16, "chunks of 8 or 16 bytes");
  static_assert(32 % U == 0, "groups must tile the 32 records of a fetch");
  constexpr bool kDp4a = std::is_same<TB, int8_t>::value && std::is_same<TACC, int32_t>::value &&
                         U % 4 == 0 && CE == 8 && J == 1;
  constexpr bool kMixed = std::is_same<TA, __nv_bfloat16>::value &&
                          std::is_same<TB, __nv_bfloat16>::value && CE % 2 == 0;
  using RawT = typename RawOf<CB>::type;
  extern __shared__ __align__(16) unsigned char ring_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // this launch may start while the previous one in the stream finishes
  // (programmatic dependent launch): wait before reading any global data
  pdl_wait();
  // the host launches at most 2^31 - 1 items
  const int it = (int)blockIdx.x * 8 + warp;
  if (it >= (int)T.total) return;
  const uint64_t keep = policy_evict_last(), stream = policy_evict_first();
  // this warp's ring: [2 groups][U records][J chunks][32 lanes] of CB bytes
  const uint32_t ring = smem_u32(ring_smem) + (uint32_t)(warp * 2 * U * J * 32 * CB);
  const unsigned char* ring_gen = ring_smem + (size_t)warp * 2 * U * J * 32 * CB;
  int q = 0;
  while (q + 1 < T.count && (int64_t)it >= T.p[q + 1].items0) ++q;
  const DirectProb& P = T.p[q];
  const int local = it - (int)P.items0;
  const int si = local / P.strips;
  const int strip = local - si * P.strips;
  // the segment entry (64 bytes, one coalesced load of 16 lanes): its head
  // and the piece's first records
  const uint32_t wv =
      lane < 16 ? ld_keep(reinterpret_cast<const uint32_t*>(&P.segs[si]) + lane, keep) : 0u;
  const int4 seg = make_int4((int)__shfl_sync(0xffffffffu, wv, 0),
                             (int)__shfl_sync(0xffffffffu, wv, 1),
                             (int)__shfl_sync(0xffffffffu, wv, 2),
                             (int)__shfl_sync(0xffffffffu, wv, 3));
  constexpr int RW = (int)sizeof(WT) / 4;   // words per record
  constexpr int NI = 12 / RW;               // records held inline
  WT inl;
  {
    uint32_t iw[RW];
#pragma unroll
    for (int j = 0; j < RW; ++j) iw[j] = __shfl_sync(0xffffffffu, wv, 4 + (lane % NI) * RW + j);
    memcpy(&inl, iw, sizeof(WT));
  }
  const int64_t row = seg.x;
  const int e0 = seg.y, e_end = seg.z;
  const bool cut = seg.w != 0;
  const int64_t n0 = (int64_t)strip * (32 * V);
  const int64_t N = P.N;
  TACC acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = TACC(0);
  TC* crow = reinterpret_cast<TC*>(P.C) + row * P.ldc;
  const WT* __restrict__ rnz = reinterpret_cast<const WT*>(P.rnz);
  // per lane chunk: the bytes inside N (0: past the end) and the chunk's
  // address in row 0 of B (column 0 when nothing is read), so that a
  // record's copy source is one multiply-add away
  int valid[J];
  const char* lane_ptr[J];
  const int64_t row_bytes = P.ldb * (int64_t)sizeof(TB);
#pragma unroll
  for (int jj = 0; jj < J; ++jj) {
    const int64_t col = n0 + jj * 32 * CE + lane * CE;
    const int64_t left = N - col;
    valid[jj] = left <= 0 ? 0 : (left >= CE ? CB : (int)left * (int)sizeof(TB));
    lane_ptr[jj] = static_cast<const char*>(P.B) + (valid[jj] ? col * (int64_t)sizeof(TB) : 0);
  }
  if (P.load_c_first && !cut) {
#pragma unroll
    for (int jj = 0; jj < J; ++jj)
#pragma unroll
      for (int v = 0; v < CE; ++v) {
        const int64_t col = n0 + jj * 32 * CE + lane * CE + v;
        if (col < N) acc[jj * CE + v] = (TACC)crow[col];
      }
  }
  auto slot_off = [&](int grp, int u, int jj) -> uint32_t {
    return (uint32_t)((((grp * U + u) * J + jj) * 32 + lane) * CB);
  };
  // issue group `grp` (records t .. t+U-1 of the fetch held in `m`); B rows
  // stream through L2 (evict first)
  auto issue = [&](WT m, int cnt, int t, int grp, WT (&wb)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) wb[u] = shfl_rec(m, t + u);
    const bool full = cnt - t >= U;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (full || t + u < cnt) {
        const int64_t off = (int64_t)(uint32_t)RowRec<TA>::k(wb[u]) * row_bytes;
#pragma unroll
        for (int jj = 0; jj < J; ++jj)
          cp_async_hint<CB>(ring + slot_off(grp, u, jj), lane_ptr[jj] + off, valid[jj], stream);
      }
    }
    cp_async_commit();
  };
  auto consume = [&](int cnt, int t, int grp, const WT (&wb)[U]) {
    RawT rb[U][J];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int jj = 0; jj < J; ++jj)
        rb[u][jj] = *reinterpret_cast<const RawT*>(ring_gen + slot_off(grp, u, jj));
    if constexpr (kDp4a) {
#pragma unroll
      for (int g4 = 0; g4 < U / 4; ++g4) {
        uint32_t ap = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          ap |= (t + 4 * g4 + u < cnt ? ((uint32_t)wb[4 * g4 + u] >> 16) & 0xFFu : 0u) << (8 * u);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t q0 = h ? rb[4 * g4 + 0][0].y : rb[4 * g4 + 0][0].x;
          const uint32_t q1 = h ? rb[4 * g4 + 1][0].y : rb[4 * g4 + 1][0].x;
          const uint32_t q2 = h ? rb[4 * g4 + 2][0].y : rb[4 * g4 + 2][0].x;
          const uint32_t q3 = h ? rb[4 * g4 + 3][0].y : rb[4 * g4 + 3][0].x;
          const uint32_t lo01 = __byte_perm(q0, q1, 0x5140);
          const uint32_t lo23 = __byte_perm(q2, q3, 0x5140);
          const uint32_t hi01 = __byte_perm(q0, q1, 0x7362);
          const uint32_t hi23 = __byte_perm(q2, q3, 0x7362);
          // a slot past the fetch holds stale bytes: its code in ap is 0
          acc[4 * h + 0] = __dp4a((int)__byte_perm(lo01, lo23, 0x5410), (int)ap, acc[4 * h + 0]);
          acc[4 * h + 1] = __dp4a((int)__byte_perm(lo01, lo23, 0x7632), (int)ap, acc[4 * h + 1]);
          acc[4 * h + 2] = __dp4a((int)__byte_perm(hi01, hi23, 0x5410), (int)ap, acc[4 * h + 2]);
          acc[4 * h + 3] = __dp4a((int)__byte_perm(hi01, hi23, 0x7632), (int)ap, acc[4 * h + 3]);
        }
      }
    } else {
      const bool full = cnt - t >= U;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (!full && t + u >= cnt) continue;
        if constexpr (kMixed) {
#pragma unroll
          for (int jj = 0; jj < J; ++jj) {
            const uint32_t* wds = reinterpret_cast<const uint32_t*>(&rb[u][jj]);
#pragma unroll
            for (int h = 0; h < CE / 2; ++h)
              fma_bf16x2(acc[jj * CE + 2 * h], acc[jj * CE + 2 * h + 1], (uint32_t)wb[u], wds[h]);
          }
        } else {
          const TACC a = RowRec<TA>::a(wb[u]);
#pragma unroll
          for (int jj = 0; jj < J; ++jj) {
            const TB* vals = reinterpret_cast<const TB*>(&rb[u][jj]);
#pragma unroll
            for (int v = 0; v < CE; ++v)
              acc[jj * CE + v] = mac(a, to_acc(vals[v], TACC(0)), acc[jj * CE + v]);
          }
        }
      }
    }
  };
  // 32 records per fetch (lane i holds record i; the next fetch of the row is
  // issued before this one is consumed); groups of U alternate between the
  // two halves of the ring
  // records stay in L2 across launches (evict last): e_end is the row's
  // sentinel or the next piece's first record, always inside the stream
  // a piece of at most NI records needs no record load at all
  WT mine = e_end - e0 <= NI ? inl : ld_keep(&rnz[lane < e_end - e0 ? e0 + lane : e_end], keep);
  for (int base = e0; base < e_end; base += 32) {
    const int cnt = min(32, e_end - base);
    WT nmine = mine;
    if (base + 32 < e_end)
      nmine = ld_keep(&rnz[base + 32 + lane < e_end ? base + 32 + lane : e_end], keep);
    WT wa[U], wbb[U];
    issue(mine, cnt, 0, 0, wa);
    for (int t = 0; t < cnt; t += 2 * U) {
      if (t + U < cnt) {
        issue(mine, cnt, t + U, 1, wbb);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      consume(cnt, t, 0, wa);
      if (t + U >= cnt) break;
      if (t + 2 * U < cnt) {
        issue(mine, cnt, t + 2 * U, 0, wa);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      consume(cnt, t + U, 1, wbb);
    }
    mine = nmine;
  }
  // the next launch in the stream may be scheduled as this CTA finishes
  pdl_trigger();
  // C written once (dequantisation needs the scales of this problem)
  SparseParams sp{};
  sp.row_scale = P.row_scale;
  sp.col_scale = P.col_scale;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int64_t col0 = n0 + j * 32 * CE + lane * CE;
    if (col0 >= N) continue;
    TC o[CE];
    if (cut) {
#pragma unroll
      for (int v = 0; v < CE; ++v)
        if (col0 + v < N)
          atomicAdd(crow + col0 + v, out_value<TC, TACC>(acc[j * CE + v], sp, row, col0 + v));
      continue;
    }
#pragma unroll
    for (int v = 0; v < CE; ++v) {
      o[v] = (col0 + v < N) ? out_value<TC, TACC>(acc[j * CE + v], sp, row, col0 + v) : TC(0);
      if (P.add_c_at_end && col0 + v < N) o[v] = o[v] + crow[col0 + v];
    }
    if (P.vec_ok && col0 + CE <= N) {
      store_chunk<TC, CE>(crow + col0, o);
    } else {
#pragma unroll
      for (int v = 0; v < CE; ++v)
        if (col0 + v < N) crow[col0 + v] = o[v];
    }
  }
}

using KernelFn = void (*)(const SparseParams, const CUtensorMap, const CUtensorMap);

struct Entry {
  rosko_dtype a, b, c;
  int R, V, order;
  KernelFn fn;
  size_t smem_set;
};

#define ROSKO_COL(TA, TB, TC, DA, DB, DC, R, V) \
  {DA, DB, DC, R, V, 1, sparse_spmm_kernel<TA, TB, TC, R, V, 1>, 0}
#define ROSKO_ROW(TA, TB, TC, DA, DB, DC, R, V) \
  {DA, DB, DC, R, V, 2, sparse_spmm_kernel<TA, TB, TC, R, V, 2>, 0}
#define ROSKO_GATHER(TA, TB, TC, DA, DB, DC, R, V) \
  {DA, DB, DC, R, V, 3, sparse_spmm_kernel<TA, TB, TC, R, V, 3>, 0}
// order 4 has its own kernel and signature (see DirectEntry)

// Column order: m_r x V = 128 accumulators per lane (wide strips amortise the
// row dispatch).  Row-slot order: 64 (its per-row cursors and look-ahead
// records need the rest of the register file), m_r <= 16.
Entry g_table[] = {
    ROSKO_COL(float, float, float, ROSKO_F32, ROSKO_F32, ROSKO_F32, 32, 4),
    ROSKO_COL(float, float, float, ROSKO_F32, ROSKO_F32, ROSKO_F32, 16, 8),
    ROSKO_COL(float, float, float, ROSKO_F32, ROSKO_F32, ROSKO_F32, 16, 4),
    ROSKO_COL(float, float, float, ROSKO_F32, ROSKO_F32, ROSKO_F32, 8, 16),
    ROSKO_COL(float, float, float, ROSKO_F32, ROSKO_F32, ROSKO_F32, 8, 8),
    ROSKO_COL(__nv_bfloat16, __nv_bfloat16, float, ROSKO_BF16, ROSKO_BF16, ROSKO_F32, 32, 4),
    ROSKO_COL(__nv_bfloat16, __nv_bfloat16, float, ROSKO_BF16, ROSKO_BF16, ROSKO_F32, 16, 8),
    ROSKO_COL(__nv_bfloat16, __nv_bfloat16, float, ROSKO_BF16, ROSKO_BF16, ROSKO_F32, 8, 16),
    ROSKO_COL(__nv_bfloat16, __nv_bfloat16, float, ROSKO_BF16, ROSKO_BF16, ROSKO_F32, 8, 8),
    ROSKO_COL(int8_t, int8_t, int32_t, ROSKO_I8, ROSKO_I8, ROSKO_I32, 32, 4),
    ROSKO_COL(int8_t, int8_t, int32_t, ROSKO_I8, ROSKO_I8, ROSKO_I32, 16, 8),
    ROSKO_COL(int8_t, int8_t, int32_t, ROSKO_I8, ROSKO_I8, ROSKO_I32, 8, 16),
    ROSKO_COL(int8_t, int8_t, float, ROSKO_I8, ROSKO_I8, ROSKO_F32, 32, 4),
    ROSKO_COL(int8_t, int8_t, float, ROSKO_I8, ROSKO_I8, ROSKO_F32, 16, 8),
    ROSKO_COL(int8_t, int8_t, float, ROSKO_I8, ROSKO_I8, ROSKO_F32, 8, 16),
    ROSKO_COL(double, float, double, ROSKO_F64, ROSKO_F32, ROSKO_F64, 32, 2),
    ROSKO_COL(double, float, double, ROSKO_F64, ROSKO_F32, ROSKO_F64, 16, 4),
    ROSKO_COL(double, float, double, ROSKO_F64, ROSKO_F32, ROSKO_F64, 8, 8),
    ROSKO_ROW(float, float, float, ROSKO_F32, ROSKO_F32, ROSKO_F32, 16, 4),
    ROSKO_ROW(float, float, float, ROSKO_F32, ROSKO_F32, ROSKO_F32, 8, 8),
    ROSKO_ROW(__nv_bfloat16, __nv_bfloat16, float, ROSKO_BF16, ROSKO_BF16, ROSKO_F32, 16, 4),
    ROSKO_ROW(__nv_bfloat16, __nv_bfloat16, float, ROSKO_BF16, ROSKO_BF16, ROSKO_F32, 8, 8),
    ROSKO_ROW(int8_t, int8_t, int32_t, ROSKO_I8, ROSKO_I8, ROSKO_I32, 16, 4),
    ROSKO_ROW(int8_t, int8_t, int32_t, ROSKO_I8, ROSKO_I8, ROSKO_I32, 8, 8),
    ROSKO_ROW(int8_t, int8_t, float, ROSKO_I8, ROSKO_I8, ROSKO_F32, 16, 4),
    ROSKO_ROW(int8_t, int8_t, float, ROSKO_I8, ROSKO_I8, ROSKO_F32, 8, 8),
    ROSKO_ROW(double, float, double, ROSKO_F64, ROSKO_F32, ROSKO_F64, 16, 2),
    ROSKO_ROW(double, float, double, ROSKO_F64, ROSKO_F32, ROSKO_F64, 8, 4),
    // row-slot with the touched-row gather: one 128-row tile (8 panels of 16)
    ROSKO_GATHER(float, float, float, ROSKO_F32, ROSKO_F32, ROSKO_F32, 16, 4),
    ROSKO_GATHER(__nv_bfloat16, __nv_bfloat16, float, ROSKO_BF16, ROSKO_BF16, ROSKO_F32, 16, 4),
    ROSKO_GATHER(int8_t, int8_t, int32_t, ROSKO_I8, ROSKO_I8, ROSKO_I32, 16, 4),
    ROSKO_GATHER(int8_t, int8_t, float, ROSKO_I8, ROSKO_I8, ROSKO_F32, 16, 4),
    ROSKO_GATHER(double, float, double, ROSKO_F64, ROSKO_F32, ROSKO_F64, 16, 2),
};

// Row-direct variants: V columns per lane (one 16-byte chunk for BF16 at
// V = 8), the shared-memory ring sized per variant.
struct DirectEntry {
  rosko_dtype a, b, c;
  int V;
  void (*one)(const DirectTable<1>);
  void (*many)(const DirectTable<64>);
  size_t smem;                   // dynamic shared memory (the warps' rings)
  mutable bool attr_set = false;
};

#define ROSKO_DIRECT(TA, TB, TC, DA, DB, DC, V)                                              \
  {DA, DB, DC, V, rowdirect_kernel<TA, TB, TC, V, 1>, rowdirect_kernel<TA, TB, TC, V, 64>, \
   async_smem_bytes<TA, TB, TC, V, 1>()}

const DirectEntry g_direct[] = {
    ROSKO_DIRECT(float, float, float, ROSKO_F32, ROSKO_F32, ROSKO_F32, 8),
    ROSKO_DIRECT(float, float, float, ROSKO_F32, ROSKO_F32, ROSKO_F32, 4),
    ROSKO_DIRECT(__nv_bfloat16, __nv_bfloat16, float, ROSKO_BF16, ROSKO_BF16, ROSKO_F32, 8),
    ROSKO_DIRECT(__nv_bfloat16, __nv_bfloat16, float, ROSKO_BF16, ROSKO_BF16, ROSKO_F32, 16),
    ROSKO_DIRECT(__nv_bfloat16, __nv_bfloat16, float, ROSKO_BF16, ROSKO_BF16, ROSKO_F32, 4),
    ROSKO_DIRECT(int8_t, int8_t, int32_t, ROSKO_I8, ROSKO_I8, ROSKO_I32, 8),
    ROSKO_DIRECT(int8_t, int8_t, float, ROSKO_I8, ROSKO_I8, ROSKO_F32, 8),
    ROSKO_DIRECT(double, float, double, ROSKO_F64, ROSKO_F32, ROSKO_F64, 4),
};

const DirectEntry* find_direct(rosko_dtype a, rosko_dtype b, rosko_dtype c, int V) {
  for (const auto& e : g_direct)
    if (e.a == a && e.b == b && e.c == c && e.V == V) return &e;
  return nullptr;
}

Entry* find_entry(rosko_dtype a, rosko_dtype b, rosko_dtype c, int R, int V, int order) {
  for (auto& e : g_table)
    if (e.a == a && e.b == b && e.c == c && e.R == R && e.V == V && e.order == order) return &e;
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

bool sparse_config_supported(rosko_dtype p_dt, rosko_dtype b_dt, rosko_dtype c_dt, int R, int V,
                             int order) {
  if (order == 4) return find_direct(p_dt, b_dt, c_dt, V) != nullptr;
  return find_entry(p_dt, b_dt, c_dt, R, V, order) != nullptr;
}

// Columns per lane: column order fills 128 accumulator registers, row-slot 64
// (FP64 accumulators take two registers each).
int sparse_default_V(rosko_dtype p_dt, int R, int order) {
  // order 4: 256-column strips, 16-byte lane loads (two per lane for FP32);
  // the wider loads keep more bytes in flight per warp, which this
  // latency-bound traversal needs (BF16 at 99.8% sparsity: 17.7 us against
  // 22.5 us for 128-column strips)
  if (order == 4) return p_dt == ROSKO_F64 ? 4 : 8;
  const int regs = (order >= 2 ? 64 : 128) / (p_dt == ROSKO_F64 ? 2 : 1);
  return std::max(2, regs / R);
}


// The work segments (list `which` of the handle, 0 = fine, 1 = coarse) of
// the listed panels (panel_list is NULL for all panels in order, or the
// handle's panel_order with n_panels its first entries); *n_segs receives
// their count, *cut whether one of those rows is cut into several pieces.
// NULL for a list of another kind.
const SegEntry* direct_segments(const rosko_packed_s* h, const int32_t* panel_list, int64_t n_panels,
                                int which, int64_t* n_segs, bool* cut) {
  if (cut) *cut = false;
  *n_segs = -1;
  const rosko_packed_s::SegList& L = h->segs[which & 1];
  if (!L.nat || n_panels < 0 || n_panels > h->P) return nullptr;
  const SegEntry* base;
  if (n_panels == h->P && L.lpt && (!panel_list || panel_list == h->panel_order_dev)) {
    // every panel runs sparse: any order of all segments covers them, and
    // the longest-first order balances the launch
    base = L.lpt;
  } else if (!panel_list) {
    // all panels in order (the prefix sums' last entry is the total in
    // either order)
    if (n_panels != h->P) return nullptr;
    base = L.nat;
  } else if (panel_list == h->panel_order_dev && L.ord) {
    base = L.ord;
  } else {
    return nullptr;
  }
  *n_segs = L.prefix[(size_t)n_panels];
  if (cut) *cut = L.split[(size_t)n_panels] > 0;
  return base;
}

// Granularity for a launch: the coarse list when it still gives every SM
// four waves of resident warps (24 per SM) over the column strips, else the
// fine list (more, shorter pieces; the cut rows are added atomically).
int direct_pick(const rosko_packed_s* h, const int32_t* panel_list, int64_t n_panels, int64_t N,
                int V) {
  int64_t ns = 0, ns_fine = 0;
  if (!direct_segments(h, panel_list, n_panels, 1, &ns, nullptr)) return 0;
  const int64_t strips = (N + 32 * V - 1) / (32 * V);
  if (ns * strips >= 4LL * 24 * num_sms()) return 1;
  // few work items: the fine list adds warps for long rows, but a cut row
  // costs a zero fill of C and atomic adds; when cutting adds under a
  // quarter more pieces (an even matrix with a few rows just past 64
  // records: 512x4608 at 99 %) the rows stay whole
  if (!direct_segments(h, panel_list, n_panels, 0, &ns_fine, nullptr)) return 1;
  return 4 * ns_fine >= 5 * ns ? 0 : 1;
}

// Fill one problem of a row-direct table; returns the problem's block count
// (< 0: invalid argument).
static int64_t direct_prob(const DirectJob& j, int V, int64_t items0, DirectProb* P) {
  const rosko_packed_s* h = j.h;
  const size_t bsz = dtype_size(j.b_dt), csz = dtype_size(j.c_dt);
  // 16-byte lane loads: B rows must start on 16-byte boundaries
  if (reinterpret_cast<uintptr_t>(j.B) % 16 != 0 || (j.ldb * (int64_t)bsz) % 16 != 0) return -1;
  int64_t n_segs = 0;
  const int which = direct_pick(h, j.panel_list, j.n_panels, j.N, V);
  const SegEntry* segs = direct_segments(h, j.panel_list, j.n_panels, which, &n_segs, nullptr);
  if (!segs) return -1;
  std::memset(P, 0, sizeof(*P));
  P->rnz = h->rnz;
  P->segs = segs;
  P->row_scale = h->row_scale;
  P->col_scale = j.col_scale;
  P->B = j.B;
  P->C = j.C;
  P->n_segs = n_segs;
  P->ldb = j.ldb;
  P->ldc = j.ldc;
  P->M = h->M;
  P->N = j.N;
  P->strips = (int)((j.N + 32 * V - 1) / (32 * V));
  const bool dequant = (h->dt == ROSKO_I8 && j.c_dt == ROSKO_F32);
  P->load_c_first = j.accumulate && !dequant;
  P->add_c_at_end = j.accumulate && dequant;
  P->vec_ok = ((reinterpret_cast<uintptr_t>(j.C) % 16) == 0) && ((j.ldc * (int64_t)csz) % 16 == 0);
  P->items0 = items0;
  return n_segs * P->strips;
}

rosko_status direct_batch_launch(const DirectJob* jobs, int count, int V, cudaStream_t st,
                                 bool pdl) {
  if (count <= 0) return ROSKO_OK;
  if (count > 64) return ROSKO_ERR_INVALID_ARG;
  const rosko_dtype a = jobs[0].h->dt, b = jobs[0].b_dt, c = jobs[0].c_dt;
  for (int i = 0; i < count; ++i) {
    if (jobs[i].h->dt != a || jobs[i].b_dt != b || jobs[i].c_dt != c) return ROSKO_ERR_INVALID_ARG;
    if (!jobs[i].h->rnz || !jobs[i].h->rowptr) return ROSKO_ERR_UNSUPPORTED;
  }
  const DirectEntry* e = find_direct(a, b, c, V);
  if (!e) return ROSKO_ERR_UNSUPPORTED;
  auto fill = [&](auto& T) -> int64_t {
    int64_t items = 0;
    int n = 0;
    for (int i = 0; i < count; ++i) {
      if (jobs[i].N <= 0 || jobs[i].n_panels <= 0) continue;
      const int64_t ni = direct_prob(jobs[i], V, items, &T.p[n]);
      if (ni < 0) return -1;
      if (ni == 0) continue;
      items += ni;
      ++n;
    }
    T.count = n;
    T.total = items;
    return items;
  };
  if (!e->attr_set) {
    if (cudaFuncSetAttribute(e->one, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e->smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(e->many, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e->smem) !=
            cudaSuccess)
      return ROSKO_ERR_CUDA;
    e->attr_set = true;
  }
  if (count == 1) {
    DirectTable<1> T;
    std::memset(static_cast<void*>(&T), 0, sizeof(T));
    const int64_t items = fill(T);
    if (items < 0 || items > INT_MAX) return ROSKO_ERR_UNSUPPORTED;   // 31-bit item index
    if (items == 0) return ROSKO_OK;
    if (pdl) {
      // a programmatic dependent of the launch before it (waits in-kernel)
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)((items + 7) / 8));
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = e->smem;
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (cudaLaunchKernelEx(&cfg, e->one, T) != cudaSuccess) return ROSKO_ERR_CUDA;
    } else {
      e->one<<<(unsigned)((items + 7) / 8), 256, e->smem, st>>>(T);
    }
  } else {
    DirectTable<64> T;
    std::memset(static_cast<void*>(&T), 0, sizeof(T));
    const int64_t items = fill(T);
    if (items < 0 || items > INT_MAX) return ROSKO_ERR_UNSUPPORTED;   // 31-bit item index
    if (items == 0) return ROSKO_OK;
    e->many<<<(unsigned)((items + 7) / 8), 256, e->smem, st>>>(T);
  }
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
}

rosko_status sparse_spmm_launch(rosko_packed_s* h, const void* B, rosko_dtype b_dt, int64_t N,
                                int64_t ldb, const float* col_scale, void* C, rosko_dtype c_dt,
                                int64_t ldc, int accumulate, const SparseLaunch& L,
                                const int32_t* panel_list, int64_t n_panels, bool c_zeroed,
                                cudaStream_t st) {
  if (n_panels <= 0) return ROSKO_OK;
  if (L.order == 4) {
    // one warp per C row, B from L2; no K split, C written (or added) directly
    DirectJob j{h, B, b_dt, N, ldb, col_scale, C, c_dt, ldc, accumulate, panel_list, n_panels};
    return direct_batch_launch(&j, 1, L.V, st, true);
  }
  if (L.order == 2 && !h->rnz) return ROSKO_ERR_UNSUPPORTED;
  if (L.order == 3 && (!h->gnz || L.R != 16 || L.W != 8)) return ROSKO_ERR_UNSUPPORTED;
  Entry* e = find_entry(h->dt, b_dt, c_dt, L.R, L.V, L.order);
  if (!e) return ROSKO_ERR_UNSUPPORTED;
  const int NR = 32 * L.V;
  const size_t bsz = dtype_size(b_dt), csz = dtype_size(c_dt);
  const size_t smem = 1024 + (size_t)L.stages * L.KC * NR * bsz;
  if (smem > e->smem_set) {
    if (cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return ROSKO_ERR_CUDA;
    e->smem_set = smem;
  }
  // a TMA box is at most 256 elements wide: wide strips take several boxes
  const int boxes = NR > 256 ? NR / 256 : 1;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)h->K};
  const cuuint64_t strides[1] = {(cuuint64_t)ldb * bsz};
  const cuuint32_t box[2] = {(cuuint32_t)(NR / boxes), (cuuint32_t)L.KC};
  const cuuint32_t es[2] = {1, 1};
  CUresult r = encode_tiled(&map, tmap_dtype(b_dt), 2, const_cast<void*>(B), dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return ROSKO_ERR_INVALID_ARG;
  // single-row boxes for the touched-row gather
  CUtensorMap map1 = map;
  if (L.order == 3) {
    const cuuint32_t box1[2] = {(cuuint32_t)(NR / boxes), 1u};
    if (encode_tiled(&map1, tmap_dtype(b_dt), 2, const_cast<void*>(B), dims, strides, box1, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return ROSKO_ERR_INVALID_ARG;
  }

  SparseParams p{};
  p.panel_list = panel_list;
  p.n_list = n_panels;
  p.panel_col = h->panel_col;
  p.colrec = h->colrec;
  p.nz = h->nz;
  p.rowptr = h->rowptr;
  p.rnz = h->rnz;
  p.gu_start = h->gu_start;
  p.gu_k = h->gu_k;
  p.gnz = h->gnz;
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
  p.boxes = boxes;
  p.slabs_total = (int)((h->K + L.KC - 1) / L.KC);
  const bool dequant = (h->dt == ROSKO_I8 && c_dt == ROSKO_F32);
  p.atomic_out = L.split > 1;
  p.load_c_first = accumulate && !p.atomic_out && !dequant;
  p.add_c_at_end = accumulate && !p.atomic_out && dequant;
  p.vec_ok = ((reinterpret_cast<uintptr_t>(C) % 16) == 0) && ((ldc * csz) % 16 == 0);
  p.status = device_status_word();
  if (!p.status) return ROSKO_ERR_CUDA;

  if (p.atomic_out && !accumulate && !c_zeroed) {
    if (cudaMemset2DAsync(C, (size_t)ldc * csz, 0, (size_t)N * csz, (size_t)h->M, st) !=
        cudaSuccess)
      return ROSKO_ERR_CUDA;
  }
  // order 3: panel_list holds 128-row tile ids and n_panels counts tiles
  const unsigned gx = L.order == 3 ? (unsigned)n_panels : (unsigned)((n_panels + L.W - 1) / L.W);
  const dim3 grid(gx, (unsigned)((N + NR - 1) / NR), (unsigned)L.split);
  e->fn<<<grid, (L.W + 1) * 32, smem, st>>>(p, map, map1);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
}

}  // namespace rosko
