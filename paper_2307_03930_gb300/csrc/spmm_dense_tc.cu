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
#include <algorithm>

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
  int slabs_total, split, stages;
  int atomic_out, accumulate, vec_ok;
  int* status;
};

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
  uint64_t* done = empty + S;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int copy = blockIdx.x;
  const int n0 = blockIdx.y * TN;
  const int s_per = (p.slabs_total + p.split - 1) / p.split;
  const int s_begin = (int)blockIdx.z * s_per;
  const int nslabs = max(0, min(p.slabs_total, s_begin + s_per) - s_begin);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    fence_barrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, TN);
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
      int i = 0;
      bool ok = true;
      for (; i < nslabs; ++i) {
        const int st = i % S;
        const uint32_t ph = (uint32_t)(i / S) & 1u;
        if (i >= S && !mbar_wait_bounded(&empty[st], ph ^ 1u, p.status)) {
          ok = false;
          break;
        }
        uint8_t* a_dst = smem + (size_t)st * kStageBytes;
        uint8_t* b_dst = a_dst + kABytes;
        const int k0 = (s_begin + i) * kTK;
        mbar_arrive_expect_tx(&full[st], kStageBytes);
        tma_load_2d(a_dst, &tmA, k0, copy * kTM, &full[st]);
#pragma unroll
        for (int j = 0; j < TN / 64; ++j)
          tma_load_2d(b_dst + j * (kTK * 128), &tmB, n0 + 64 * j, k0, &full[st]);
      }
      if (!ok) {
        for (int j = max(0, i - S); j < i; ++j)
          mbar_wait_bounded(&full[j % S], (uint32_t)(j / S) & 1u, p.status);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (one thread) --------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(kTM, TN, false, true);
      for (int i = 0; i < nslabs; ++i) {
        const int st = i % S;
        const uint32_t ph = (uint32_t)(i / S) & 1u;
        if (!mbar_wait_bounded(&full[st], ph, p.status)) break;
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
          tc::mma_bf16(tmem, ad, bd, idesc, (i > 0 || kk > 0) ? 1u : 0u);
        }
        tc::mma_commit(&empty[st]);  // frees the stage once these MMAs finish
      }
      tc::mma_commit(done);
    }
  } else {
    // ---------------- epilogue: TMEM -> registers -> C -----------------------
    const int quarter = warp & 3;
    const bool ok = mbar_wait_bounded(done, 0, p.status);
    tc::fence_after_sync();
    const int64_t row = (int64_t)__ldg(&p.tile_order[copy]) * kTM + quarter * 32 + lane;
    if (ok && nslabs > 0) {
#pragma unroll 1
      for (int c = 0; c < TN / 32; ++c) {
        uint32_t r[32];
        tc::tmem_ld_32x32b_x32(tmem + ((uint32_t)(quarter * 32) << 16) + c * 32, r);
        tc::tmem_ld_wait();
        const int64_t col0 = n0 + c * 32;
        if (row >= p.M || col0 >= p.N) continue;
        float* dst = p.C + row * p.ldc + col0;
        if (p.atomic_out) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (col0 + j < p.N) atomicAdd(dst + j, __uint_as_float(r[j]));
        } else if (p.vec_ok && col0 + 32 <= p.N) {
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
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 1) tc::tmem_dealloc(tmem, TN);
}

template <int TN>
size_t dense_smem_bytes(int stages) {
  return 1024 + (size_t)stages * (kABytes + (size_t)TN * kTK * 2) + 256;
}

}  // namespace

rosko_status dense_spmm_launch(const void* dense_A, int64_t dense_rows, int64_t Kpad,
                               const int32_t* tile_order_dev, int64_t n_tiles, int64_t K,
                               const void* B, int64_t N, int64_t ldb, float* C, int64_t ldc,
                               int64_t M, int accumulate, int TN, int split, cudaStream_t st) {
  if (n_tiles <= 0 || N <= 0) return ROSKO_OK;
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
  p.slabs_total = (int)((K + kTK - 1) / kTK);
  p.split = std::max(1, std::min(split, p.slabs_total));
  p.stages = stages;
  p.atomic_out = p.split > 1;
  p.accumulate = accumulate;
  p.vec_ok = ((reinterpret_cast<uintptr_t>(C) % 16) == 0) && ((ldc * 4) % 16 == 0);
  p.status = device_status_word();
  if (!p.status) return ROSKO_ERR_CUDA;
  const dim3 grid((unsigned)n_tiles, (unsigned)((N + TN - 1) / TN), (unsigned)p.split);
  fn<<<grid, 192, smem, st>>>(p, mapA, mapB);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
}

}  // namespace rosko
