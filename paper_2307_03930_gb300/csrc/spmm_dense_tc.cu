// Dense-panel path on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Row tiles of A (128 rows = several packed panels) whose density is high
// enough that a dense contraction beats row skipping on CUDA cores are kept
// as dense BF16 copies.  For such a tile the whole K-first schedule of
// Sec. 4.2 runs on the tensor core: the 128 x TN C tile lives in tensor memory
// (TMEM) for the full K range, K slabs of A (128 x 64, K-major) and B
// (64 x TN, N-major: B is row-major K x N) stream through a ring of shared
// memory stages filled by TMA, one elected thread issues tcgen05.mma
// (M = 128, N = TN, K = 16 per instruction) and C is written once.
//
// Warp roles (6 warps): 0 = TMA producer, 1 = MMA issuer (and TMEM owner),
// 2..5 = epilogue (warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31).
//
// Schedule: persistent stream-K.  The (tile, K slab) units of all dense tiles
// are cut into one equal contiguous share per SM, so small-M problems (few
// row tiles) still fill every SM in one wave.  A share covers the K ranges of
// one or two tiles; two TMEM accumulators alternate so that the epilogue of
// one range overlaps the MMAs of the next.  A tile whose K range is cut
// between CTAs is added into C with 16-byte atomics; a tile owned whole is
// stored.
#include <algorithm>
#include <vector>

#include "handle.hpp"
#include "tc_common.cuh"

namespace rosko {
namespace {

constexpr int kTM = 128;             // rows of a dense tile (MMA M)
constexpr int kTK = 64;              // K per stage: 64 BF16 = one 128-byte swizzle row
constexpr uint32_t kABytes = kTM * kTK * 2;   // 16 KB

struct DenseParams {
  const int32_t* tile_order;  // dense copy c holds rows tile_order[c]*128 ...
  float* C;
  int64_t ldc, M, N;
  int n_copy;        // 128-row tiles (dense copies) in the work
  int n_ntiles;      // TN-wide column tiles
  int slabs;         // K slabs of 64 per tile
  int64_t units;     // n_copy * n_ntiles * slabs
  int stages, accumulate, vec_ok;
  int* status;
};

// Stream-K split of the (tile, K slab) units: CTA b owns [b U / G, (b+1) U / G).
__device__ __forceinline__ int64_t unit_begin(int64_t U, int64_t b, int64_t G) {
  return U * b / G;
}

template <int TN>
__global__ void __launch_bounds__(192, 1)
    dense_panel_kernel(const DenseParams p, const __grid_constant__ CUtensorMap tmA,
                       const __grid_constant__ CUtensorMap tmB) {
  constexpr uint32_t kBBytes = (uint32_t)TN * kTK * 2;
  constexpr uint32_t kStageBytes = kABytes + kBBytes;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = p.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * kStageBytes);
  uint64_t* empty = full + S;
  uint64_t* acc_full = empty + S;    // [2] MMA -> epilogue: accumulator ready
  uint64_t* acc_empty = acc_full + 2;  // [2] epilogue -> MMA: accumulator drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t u0 = unit_begin(p.units, blockIdx.x, gridDim.x);
  const int64_t u1 = unit_begin(p.units, blockIdx.x + 1, gridDim.x);
  if (u0 >= u1) return;
  const int64_t per_tile = p.slabs;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    fence_barrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, 2 * TN);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer -----------------------------------------
    if (lane == 0) {
      prefetch_tensormap(&tmA);
      prefetch_tensormap(&tmB);
      int64_t i = 0;
      bool ok = true;
      for (int64_t u = u0; u < u1; ++u, ++i) {
        const int st = (int)(i % S);
        const uint32_t ph = (uint32_t)(i / S) & 1u;
        if (i >= S && !mbar_wait_bounded(&empty[st], ph ^ 1u, p.status)) {
          ok = false;
          break;
        }
        const int64_t tile = u / per_tile;
        const int slab = (int)(u % per_tile);
        const int copy = (int)(tile % p.n_copy);   // row tiles fastest: CTAs that
        const int nt = (int)(tile / p.n_copy);     // run together share B in L2
        uint8_t* a_dst = smem + (size_t)st * kStageBytes;
        uint8_t* b_dst = a_dst + kABytes;
        const int k0 = slab * kTK;
        mbar_arrive_expect_tx(&full[st], kStageBytes);
        tma_load_2d(a_dst, &tmA, k0, copy * kTM, &full[st]);
#pragma unroll
        for (int j = 0; j < TN / 64; ++j)
          tma_load_2d(b_dst + j * (kTK * 128), &tmB, nt * TN + 64 * j, k0, &full[st]);
      }
      if (!ok) {
        for (int64_t j = (i > S ? i - S : 0); j < i; ++j)
          mbar_wait_bounded(&full[j % S], (uint32_t)(j / S) & 1u, p.status);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (one thread) --------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(kTM, TN, false, true);
      int64_t i = 0;
      int seg = -1;
      bool ok = true;
      for (int64_t u = u0; u < u1 && ok; ++u, ++i) {
        const int slab = (int)(u % per_tile);
        const bool first = (u == u0) || slab == 0;
        const bool last = (u + 1 == u1) || slab + 1 == per_tile;
        if (first) {
          ++seg;
          const int b = seg & 1;
          // the epilogue must have drained this accumulator (segment seg - 2)
          if (seg >= 2 &&
              !mbar_wait_bounded(&acc_empty[b], (uint32_t)((seg >> 1) - 1) & 1u, p.status)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
        }
        const uint32_t d_tmem = tmem + (uint32_t)((seg & 1) * TN);
        const int st = (int)(i % S);
        const uint32_t ph = (uint32_t)(i / S) & 1u;
        if (!mbar_wait_bounded(&full[st], ph, p.status)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t a_base = smem_u32(smem + (size_t)st * kStageBytes);
        const uint32_t b_base = a_base + kABytes;
#pragma unroll
        for (int kk = 0; kk < kTK / 16; ++kk) {
          // A: K-major, 128-byte swizzle, 8-row groups 1024 B apart; a K step
          // of 16 BF16 is 32 bytes inside the swizzle row.
          const uint64_t ad = tc::smem_desc(a_base + kk * 32, 16, 1024, 2);
          // B: N-major (row k of B = 128 bytes of 64 N values), 128-byte
          // swizzle; 64-wide N chunks are 64 rows x 128 B = 8 KB apart (LBO),
          // 8-row K groups 1024 B apart (SBO); a K step of 16 rows = 2 KB.
          const uint64_t bd = tc::smem_desc(b_base + kk * 16 * 128, kTK * 128, 1024, 2);
          tc::mma_bf16(d_tmem, ad, bd, idesc, (!first || kk > 0) ? 1u : 0u);
        }
        tc::mma_commit(&empty[st]);                  // stage free once these MMAs finish
        if (last) tc::mma_commit(&acc_full[seg & 1]);  // accumulator complete
      }
      if (!ok) {
        // make the epilogue's waits end: release every accumulator it expects
        for (int b = 0; b < 2; ++b) tc::mma_commit(&acc_full[b]);
      }
    }
  } else {
    // ---------------- epilogue: TMEM -> registers -> C -----------------------
    const int quarter = warp & 3;
    int seg = -1;
    for (int64_t u = u0; u < u1; ++u) {
      const int slab = (int)(u % per_tile);
      const bool first = (u == u0) || slab == 0;
      if (!first) continue;
      ++seg;
      // segment [u, ue): slabs of one tile
      int64_t ue = u - slab + per_tile;
      if (ue > u1) ue = u1;
      const bool whole = (slab == 0) && (ue - u == per_tile);
      const int64_t tile = u / per_tile;
      const int copy = (int)(tile % p.n_copy);
      const int nt = (int)(tile / p.n_copy);
      const int b = seg & 1;
      const bool ok = mbar_wait_bounded(&acc_full[b], (uint32_t)(seg >> 1) & 1u, p.status);
      tc::fence_after_sync();
      const int64_t row = (int64_t)__ldg(&p.tile_order[copy]) * kTM + quarter * 32 + lane;
      const int64_t n0 = (int64_t)nt * TN;
#pragma unroll 1
      for (int c = 0; c < TN / 32; ++c) {
        uint32_t r[32];
        tc::tmem_ld_32x32b_x32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * TN + c * 32),
                               r);
        tc::tmem_ld_wait();
        const int64_t col0 = n0 + c * 32;
        if (!ok || row >= p.M || col0 >= p.N) continue;
        float* dst = p.C + row * p.ldc + col0;
        const bool vec = p.vec_ok && col0 + 32 <= p.N;
        if (!whole) {
          // a K range of a split tile: add into C (zeroed beforehand unless
          // the call accumulates)
          if (vec) {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
              atomicAdd(reinterpret_cast<float4*>(dst + j),
                        make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                    __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3])));
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (col0 + j < p.N) atomicAdd(dst + j, __uint_as_float(r[j]));
          }
        } else if (vec) {
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            float4 v = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                   __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
            if (p.accumulate) {
              const float4 o = *reinterpret_cast<const float4*>(dst + j);
              v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
            }
            *reinterpret_cast<float4*>(dst + j) = v;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (col0 + j < p.N) dst[j] = __uint_as_float(r[j]) + (p.accumulate ? dst[j] : 0.0f);
        }
      }
      // accumulator drained: hand it back to the MMA issuer
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 1) tc::tmem_dealloc(tmem, 2 * TN);
}

template <int TN>
size_t dense_smem_bytes(int stages) {
  return 1024 + (size_t)stages * (kABytes + (size_t)TN * kTK * 2) + 256;
}

}  // namespace

// True when the stream-K split leaves some tile with more than one K range
// (those tiles are accumulated with atomics into a zeroed C).
int64_t dense_grid(int64_t n_tiles, int64_t N, int64_t K, int TN, int ctas) {
  const int64_t slabs = (K + kTK - 1) / kTK;
  const int64_t units = n_tiles * ((N + TN - 1) / TN) * slabs;
  return std::max<int64_t>(1, std::min<int64_t>(ctas, units));
}

bool dense_needs_zero(int64_t n_tiles, int64_t N, int64_t K, int TN, int ctas) {
  const int64_t slabs = (K + kTK - 1) / kTK;
  const int64_t units = n_tiles * ((N + TN - 1) / TN) * slabs;
  const int64_t G = dense_grid(n_tiles, N, K, TN, ctas);
  for (int64_t b = 0; b <= G; ++b) {
    const int64_t u = units * b / G;
    if (u % slabs != 0 && u != units) return true;
  }
  return false;
}

rosko_status dense_spmm_launch(const void* dense_A, int64_t dense_rows, int64_t Kpad,
                               const int32_t* tile_order_dev, int64_t n_tiles, int64_t K,
                               const void* B, int64_t N, int64_t ldb, float* C, int64_t ldc,
                               int64_t M, int accumulate, int TN, int ctas, bool c_zeroed,
                               cudaStream_t st) {
  if (n_tiles <= 0 || N <= 0) return ROSKO_OK;
  if (ctas <= 0) ctas = num_sms();
  if (TN != 128 && TN != 256) return ROSKO_ERR_INVALID_ARG;
  const int stages = (TN == 256) ? 4 : 6;
  const size_t smem = TN == 256 ? dense_smem_bytes<256>(stages) : dense_smem_bytes<128>(stages);
  static size_t set128 = 0, set256 = 0;
  size_t& set = TN == 256 ? set256 : set128;
  auto fn = TN == 256 ? dense_panel_kernel<256> : dense_panel_kernel<128>;
  if (smem > set) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return ROSKO_ERR_CUDA;
    set = smem;
  }
  CUtensorMap mapA, mapB;
  {
    const cuuint64_t dims[2] = {(cuuint64_t)Kpad, (cuuint64_t)dense_rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Kpad * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kTK, (cuuint32_t)kTM};
    const cuuint32_t es[2] = {1, 1};
    if (encode_tiled(&mapA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(dense_A), dims,
                     strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return ROSKO_ERR_INVALID_ARG;
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)K};
    const cuuint64_t strides[1] = {(cuuint64_t)ldb * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)kTK};
    const cuuint32_t es[2] = {1, 1};
    if (encode_tiled(&mapB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(B), dims,
                     strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return ROSKO_ERR_INVALID_ARG;
  }
  DenseParams p{};
  p.tile_order = tile_order_dev;
  p.C = C;
  p.ldc = ldc;
  p.M = M;
  p.N = N;
  p.n_copy = (int)n_tiles;
  p.n_ntiles = (int)((N + TN - 1) / TN);
  p.slabs = (int)((K + kTK - 1) / kTK);
  p.units = (int64_t)p.n_copy * p.n_ntiles * p.slabs;
  p.stages = stages;
  p.accumulate = accumulate;
  p.vec_ok = ((reinterpret_cast<uintptr_t>(C) % 16) == 0) && ((ldc * 4) % 16 == 0);
  p.status = device_status_word();
  if (!p.status) return ROSKO_ERR_CUDA;
  const int64_t G = dense_grid(n_tiles, N, K, TN, ctas);
  if (!accumulate && !c_zeroed && dense_needs_zero(n_tiles, N, K, TN, ctas)) {
    // zero the C rows of every dense tile (tiles are disjoint row blocks)
    std::vector<int32_t> order((size_t)n_tiles);
    if (cudaMemcpyAsync(order.data(), tile_order_dev, order.size() * 4, cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return ROSKO_ERR_CUDA;
    for (int32_t t : order) {
      const int64_t r0 = (int64_t)t * kTM;
      const int64_t rows = std::min<int64_t>(kTM, M - r0);
      if (rows > 0 &&
          cudaMemset2DAsync(C + r0 * ldc, (size_t)ldc * 4, 0, (size_t)N * 4, (size_t)rows, st) !=
              cudaSuccess)
        return ROSKO_ERR_CUDA;
    }
  }
  fn<<<(unsigned)G, 192, smem, st>>>(p, mapA, mapB);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
}

}  // namespace rosko
