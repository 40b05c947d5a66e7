// Shared device/host helpers of the GB300 row-skipping SpMM library.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rosko.h"

namespace rosko {

// ---------------------------------------------------------------------------
// Device status bits (per-device word, see rosko_device_status).
constexpr int kStatusTimeout = 1;   // a bounded wait gave up
constexpr int kStatusCorrupt = 2;   // packed stream inconsistent with the handle

// Bounded waits give up after this many nanoseconds of %globaltimer, unless
// the per-device wait limit (rosko_set_wait_limit: the 64-bit word that
// follows the status word, 0 = this default) says otherwise.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;
// Byte offset of the wait limit in the per-device status allocation.
constexpr int kWaitLimitOffset = 8;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Programmatic dependent launch.  pdl_wait: block until the grids this launch
// depends on have completed and their writes are visible (at once when the
// launch has no such dependency).  pdl_trigger: let the next launch in the
// stream start (it waits in its own pdl_wait before touching data).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------------------
// mbarrier (shared::cta) helpers.
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// The wait limit of the device whose status word is `status`.
__device__ __forceinline__ unsigned long long wait_limit_ns(const int* status) {
  if (!status) return kWaitLimitNs;
  const unsigned long long v = *reinterpret_cast<const volatile unsigned long long*>(
      reinterpret_cast<const char*>(status) + kWaitLimitOffset);
  return v ? v : kWaitLimitNs;
}

// Wait for the phase with the given parity to complete.  Gives up after the
// device's wait limit, records kStatusTimeout in *status and returns false.
// The clock and the limit (a global load) are first read after 256 polls,
// so a wait that ends soon touches no memory: a pipeline stage that is
// waited on every iteration must not pay an L2 round trip each time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  unsigned long long t0 = 0, limit = 0;
  for (uint32_t spin = 1;; ++spin) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((spin & 255u) == 0) {
      const unsigned long long now = global_ns();
      if (t0 == 0) {
        t0 = now;
        limit = wait_limit_ns(status);
      } else if (now - t0 > limit) {
        if (status) atomicOr(status, kStatusTimeout);
        return false;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// TMA: 2D tiled bulk tensor load global -> shared, completion on an mbarrier.
// x (innermost coordinate) times the element size must be a multiple of 16 B.
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map, int32_t x,
                                            int32_t y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared -> global tile copies, tracked per thread as bulk async-groups.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int32_t x, int32_t y,
                                             const void* smem_src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];"
               ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(smem_src))
               : "memory");
}
// Same, adding into global memory (element-wise atomic add in L2).
__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap* map, int32_t x, int32_t y,
                                                  const void* smem_src) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];"
      ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(smem_src))
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until at most N of this thread's bulk groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// Wait until all of this thread's bulk groups have completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void tma_load_3d(void* smem_dst, const CUtensorMap* map, int32_t x,
                                            int32_t y, int32_t z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---------------------------------------------------------------------------
// Element traits.
template <class T> struct Elem;
template <> struct Elem<float> { static constexpr rosko_dtype dt = ROSKO_F32; };
template <> struct Elem<__nv_bfloat16> { static constexpr rosko_dtype dt = ROSKO_BF16; };
template <> struct Elem<int8_t> { static constexpr rosko_dtype dt = ROSKO_I8; };
template <> struct Elem<double> { static constexpr rosko_dtype dt = ROSKO_F64; };
template <> struct Elem<int32_t> { static constexpr rosko_dtype dt = ROSKO_I32; };

inline size_t dtype_size(rosko_dtype d) {
  switch (d) {
    case ROSKO_F32: return 4;
    case ROSKO_BF16: return 2;
    case ROSKO_I8: return 1;
    case ROSKO_F64: return 8;
    case ROSKO_I32: return 4;
  }
  return 0;
}

inline bool dtype_valid(int d) { return d >= ROSKO_F32 && d <= ROSKO_I32; }

__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }

}  // namespace rosko

// ---------------------------------------------------------------------------
// Host-side helpers implemented in api.cu.
namespace rosko {
// Per-device status word (device memory), allocated once per device.
int* device_status_word();
// Device allocation with the test-only failure hook (ROSKO_FAIL_ALLOC=n makes
// the n-th allocation of the process fail).
cudaError_t dev_malloc(void** p, size_t bytes);
// cuTensorMapEncodeTiled obtained through the runtime (no libcuda link).
CUresult encode_tiled(CUtensorMap* map, CUtensorMapDataType dt, cuuint32_t rank, void* gaddr,
                      const cuuint64_t* dims, const cuuint64_t* strides, const cuuint32_t* box,
                      const cuuint32_t* estrides, CUtensorMapInterleave il, CUtensorMapSwizzle sw,
                      CUtensorMapL2promotion l2, CUtensorMapFloatOOBfill oob);
int num_sms();
// Count of kernels launched by the library (rosko_kernel_launches).
void count_launches(int n);
}  // namespace rosko
