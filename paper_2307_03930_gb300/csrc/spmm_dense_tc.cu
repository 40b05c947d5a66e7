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
// Warp roles: 0 = TMA producer, 1 = MMA issuer (and TMEM owner), 2.. =
// epilogue (warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31; with 8
// epilogue warps two share a lane quarter and split its columns).  The
// producer and MMA warps wait as whole warps (converged) and one lane
// issues.  Each ring step costs such a warp a few hundred cycles (measured:
// a wait on a completed mbarrier, an arrive or a commit, and the wake-up of
// the other side), about the 512 tensor-pipe cycles of the four MMAs of a
// 128-row K slab, so with 128-row tiles both warps move two stages per step
// (the producer's two lanes issue their stages' copies side by side).
//
// Schedule: persistent stream-K.  The (tile, K slab) units of all dense tiles
// are cut into one equal contiguous share per SM, so small-M problems (few
// row tiles) still fill every SM in one wave.  A share covers the K ranges of
// one or two tiles; two TMEM accumulators alternate so that the epilogue of
// one range overlaps the MMAs of the next.  A tile whose K range is cut
// between CTAs is added into C; a tile owned whole is stored.  C is then
// zero-filled by a small kernel launched just before this one, of which this
// launch is a programmatic dependent: the ring fills and MMAs start at once
// and only the epilogue waits (griddepcontrol.wait) for the fill, which thus
// runs under the MMAs.  The first ring fill is issued by thread 0 before the
// TMEM allocation and the block barrier, overlapping its cold DRAM latency.
//
// Epilogue: each epilogue warp moves its 32 TMEM lanes (C rows) 32 columns
// at a time into a 32 x 32 FP32 staging tile in shared memory (128-byte
// swizzle, so the row-per-lane writes are bank-conflict free) and one lane
// hands the tile to TMA: a tensor store for a whole tile, a tensor
// reduce-add (element-wise add in L2) for a cut tile or C += A.B.  Two
// staging tiles per warp let the next chunk's TMEM load overlap the copy.
// C whose rows are not 16-byte aligned falls back to direct stores and
// 16-byte atomics.
#include <algorithm>
#include <cstring>
#include <vector>

#include "handle.hpp"
#include "tc_common.cuh"

namespace rosko {
namespace {

constexpr int kTM = 128;             // rows of a dense tile (MMA M)
constexpr int kTK = 64;              // K per stage: 64 BF16 = one 128-byte swizzle row
constexpr uint32_t kABytes = kTM * kTK * 2;   // 16 KB
constexpr uint32_t kStageC = 32 * 32 * 4;      // one 32 x 32 FP32 staging tile
// Epilogue warps: 4 (one per TMEM lane quarter, two staging tiles each) or
// 8 (two per quarter, each writing half of the columns, one staging tile
// each); the staging space is the same 32 KB either way.  Measured on GB300
// the two run the epilogue in the same time (it is bound by the TMA stores
// and L2 reductions, not by the warps), so the smaller block is kept.
constexpr int kEpiWarps = 4;
constexpr int kStagePerWarp = 8 / kEpiWarps;
constexpr uint32_t kEpiBytes = 8 * kStageC;
constexpr int kThreads = 64 + 32 * kEpiWarps;

// One problem of the batch (a single SpMM is a batch of one).
struct DenseProb {
  const int32_t* tile_order;  // dense copy c holds rows tile_order[c]*128 ...
  float* C;
  int64_t ldc, M, N;
  int64_t unit0;     // first unit of this problem in the batch's unit space
  int n_copy;        // 128-row tiles (dense copies) in the work
  int n_ntiles;      // TN-wide column tiles
  int slabs;         // K slabs of 64 per tile
  int accumulate, vec_ok;
  int tma_c;         // C tensor map usable (16-byte aligned rows)
  int b3d;           // B tensor map is 3-D (64 columns x K x N / 64 chunks)
};

// The whole batch travels in the kernel parameters (no device allocation):
// per problem its A and B tensor maps and its scalars.
template <int NP>
struct DenseTable {
  CUtensorMap tmA[NP];
  CUtensorMap tmB[NP];
  CUtensorMap tmC[NP];   // FP32 C, 32 x 32 boxes, 128-byte swizzle
  DenseProb p[NP];
  int count;
  int64_t units;
  int stages;
  int aligned;   // CTA ranges start and end on tile boundaries (no tile is cut)
  // INT8 codes through the BF16 pipe: accumulator segments end every
  // `kchunk` K slabs (0: only at tile ends), so that every FP32 partial sum
  // stays an exact integer, and C is INT32 (partials converted and added)
  int kchunk;
  int out_i32;
  int* status;
};

// Stream-K split of the (tile, K slab) units: CTA b owns [b U / G, (b+1) U / G).
// U < 2^31 and b <= G < 2^16 (checked on the host), so floor(U b / G) is
// (U / G) b + ((U % G) b) / G in 32-bit unsigned divisions (a 64-bit
// division is a long software sequence that every CTA would pay at start).
__device__ __forceinline__ int64_t unit_begin(int64_t U, int64_t b, int64_t G) {
  const uint32_t u = (uint32_t)U, g = (uint32_t)G, bb = (uint32_t)b;
  const uint32_t q = u / g, r = u - q * g;
  return (int64_t)q * bb + (int64_t)((r * bb) / g);
}

// Advance the problem index q (monotone in u) so that u belongs to problem q.
template <int NP>
__device__ __forceinline__ void advance_problem(const DenseTable<NP>& T, int64_t u, int& q) {
  while (q + 1 < T.count && u >= T.p[q + 1].unit0) ++q;
}

// First tile boundary at or after unit x (tile = `slabs` consecutive units).
template <int NP>
__device__ __forceinline__ int64_t tile_boundary(const DenseTable<NP>& T, int64_t x) {
  if (x >= T.units) return T.units;
  int q = 0;
  advance_problem(T, x, q);
  const uint32_t slabs = (uint32_t)T.p[q].slabs;
  const uint32_t r = (uint32_t)(x - T.p[q].unit0) % slabs;
  return r ? x + (slabs - r) : x;
}

// Position of a unit inside the batch: problem q, row-tile group mt, column
// tile nt, K slab (unit = (nt * mtiles + mt) * slabs + slab within problem q).
// Set once per role with divisions, then advanced by increments only.
struct Cursor {
  int q, mt, nt, slab;
  int mtiles, ntiles, slabs;
  int b3d;   // problem q's B tensor map is 3-D (kept in a register: the
             // parameter table is indexed by q, a run-time value)
};

template <int NP, int MH>
__device__ __forceinline__ void cursor_load(const DenseTable<NP>& T, Cursor& c) {
  const DenseProb& P = T.p[c.q];
  c.mtiles = (P.n_copy + MH - 1) / MH;
  c.ntiles = P.n_ntiles;
  c.slabs = P.slabs;
  c.b3d = P.b3d;
}

template <int NP, int MH>
__device__ __forceinline__ Cursor cursor_at(const DenseTable<NP>& T, int64_t u) {
  Cursor c;
  c.q = 0;
  advance_problem(T, u, c.q);
  cursor_load<NP, MH>(T, c);
  const uint32_t lu = (uint32_t)(u - T.p[c.q].unit0);
  const uint32_t tile = lu / (uint32_t)c.slabs;
  c.slab = (int)(lu - tile * (uint32_t)c.slabs);
  c.nt = (int)(tile / (uint32_t)c.mtiles);
  c.mt = (int)(tile - (uint32_t)c.nt * (uint32_t)c.mtiles);
  return c;
}

// Move to the first slab of the next tile (next problem after its last tile).
template <int NP, int MH>
__device__ __forceinline__ void cursor_next_tile(const DenseTable<NP>& T, Cursor& c) {
  c.slab = 0;
  if (++c.mt == c.mtiles) {
    c.mt = 0;
    if (++c.nt == c.ntiles) {
      c.nt = 0;
      if (c.q + 1 < T.count) {
        ++c.q;
        cursor_load<NP, MH>(T, c);
      }
    }
  }
}

template <int NP, int MH>
__device__ __forceinline__ void cursor_next(const DenseTable<NP>& T, Cursor& c) {
  if (++c.slab == c.slabs) cursor_next_tile<NP, MH>(T, c);
}

// MH = 128-row halves per CTA tile (1: 128 x TN, 2: 256 x TN sharing each B
// stage between two MMAs, which halves B's shared-memory bytes per flop).
template <int TN, int NP, int MH>
__global__ void __launch_bounds__(kThreads, 1)
    dense_panel_kernel(const __grid_constant__ DenseTable<NP> T) {
  constexpr uint32_t kBBytes = (uint32_t)TN * kTK * 2;
  constexpr uint32_t kStageBytes = MH * kABytes + kBBytes;
  constexpr int NBUF = (MH * TN * 2 <= 512) ? 2 : 1;   // TMEM accumulator sets
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = T.stages;
  uint8_t* stage_c = smem + (size_t)S * kStageBytes;   // 1024-aligned: stages are 1 KB multiples
  uint64_t* full = reinterpret_cast<uint64_t*>(stage_c + kEpiBytes);
  uint64_t* empty = full + S;
  uint64_t* acc_full = empty + S;    // [2] MMA -> epilogue: accumulator ready
  uint64_t* acc_empty = acc_full + 2;  // [2] epilogue -> MMA: accumulator drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // one thread fills ring stage sj with unit cj: A (MH x 128 rows; rows past
  // the last copy are zero-filled) and TN / 64 chunks of 64 B columns, one
  // 3-D box when N is a multiple of 64 (x = column in chunk, y = k,
  // z = chunk), else one 2-D box each
  auto issue_stage = [&](const Cursor& cj, int sj) {
    uint8_t* a_dst = smem + (size_t)sj * kStageBytes;
    uint8_t* b_dst = a_dst + MH * kABytes;
    const int k0 = cj.slab * kTK;
    mbar_arrive_expect_tx(&full[sj], kStageBytes);
    tma_load_2d(a_dst, &T.tmA[cj.q], k0, cj.mt * MH * kTM, &full[sj]);
    if (cj.b3d) {
      tma_load_3d(b_dst, &T.tmB[cj.q], 0, k0, cj.nt * (TN / 64), &full[sj]);
    } else {
#pragma unroll
      for (int jj = 0; jj < TN / 64; ++jj)
        tma_load_2d(b_dst + jj * (kTK * 128), &T.tmB[cj.q], cj.nt * TN + 64 * jj, k0, &full[sj]);
    }
  };
  int64_t u0 = unit_begin(T.units, blockIdx.x, gridDim.x);
  int64_t u1 = unit_begin(T.units, blockIdx.x + 1, gridDim.x);
  if (T.aligned) {
    // many tiles: whole tiles per CTA (no zero fill, no reductions into C)
    u0 = tile_boundary(T, u0);
    u1 = tile_boundary(T, u1);
  }
  if (u0 >= u1) return;

  if (threadIdx.x == 32) {
    // descriptor fetches overlap the barrier and TMEM set-up
    int q0 = 0;
    advance_problem(T, u0, q0);
    prefetch_tensormap(&T.tmA[q0]);
    prefetch_tensormap(&T.tmB[q0]);
    if (T.p[q0].tma_c) prefetch_tensormap(&T.tmC[q0]);
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiWarps);
    }
    fence_barrier_init();
    // (a programmatic dependent only of a zero fill of C, whose start means
    // that every launch before it has completed: A and B are final here)
    // the first ring fill goes out now: its (cold, DRAM) latency overlaps
    // the TMEM allocation and the block barrier
    Cursor c = cursor_at<NP, MH>(T, u0);
    for (int64_t u = u0; u < u1 && u < u0 + S; ++u) {
      issue_stage(c, (int)(u - u0));
      cursor_next<NP, MH>(T, c);
    }
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, NBUF * MH * TN);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer -----------------------------------------
    // The whole warp walks the ring (waits are warp-wide, so the warp stays
    // converged); lane 0 issues the copies.
    // the first min(S, units) stages were filled at start
    const int64_t pre = std::min<int64_t>(S, u1 - u0);
    int64_t i = pre;
    int st = (int)(pre % S);
    uint32_t ph = pre == S ? 1u : 0u;   // ring stage and its phase parity
    bool ok = true;
    Cursor c = cursor_at<NP, MH>(T, u0 + pre < u1 ? u0 + pre : u0);
    // two stages per iteration (the MMA warp takes them in pairs too): each
    // ring step costs this warp a few hundred cycles
    constexpr int kPair = MH == 1 ? 2 : 1;
    for (int64_t u = u0 + pre; u < u1;) {
      const int n = (kPair == 2 && u + 1 < u1) ? 2 : 1;
      const int st2 = st + 1 == S ? 0 : st + 1;
      const uint32_t ph2 = st + 1 == S ? ph ^ 1u : ph;
      bool got = i < S || mbar_wait_bounded(&empty[st], ph ^ 1u, T.status);
      if (n == 2 && i + 1 >= S) got = got && mbar_wait_bounded(&empty[st2], ph2 ^ 1u, T.status);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      // lane j fills stage j of the pair: the two stages' copies are issued
      // by one instruction stream, side by side
      Cursor c1 = c;
      cursor_next<NP, MH>(T, c1);
      if (lane < n) issue_stage(lane ? c1 : c, lane ? st2 : st);
      // row tiles fastest: CTAs that run together share B in L2
      if (n == 2) {
        c = c1;
        cursor_next<NP, MH>(T, c);
      } else {
        c = c1;
      }
      __syncwarp();
      for (int j = 0; j < n; ++j) {
        if (++st == S) {
          st = 0;
          ph ^= 1u;
        }
      }
      u += n;
      i += n;
    }
    if (!ok && lane == 0) {
      // consumers gave up: wait (bounded) for our copies in flight to land
      for (int64_t j = (i > S ? i - S : 0); j < i; ++j)
        mbar_wait_bounded(&full[j % S], (uint32_t)(j / S) & 1u, T.status);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer --------------------------------------------
    // The warp waits together; lane 0 issues the MMAs and the commits.  The
    // smem descriptors of stage 0 are built once; stage s, K step kk and
    // half hh only move the start address (a 14-bit field in 16-byte units:
    // shared memory is below 256 KB, so the sum never carries out of it).
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTM, TN, false, true);
    const uint32_t sbase = smem_u32(smem);
    // A: K-major, 128-byte swizzle, 8-row groups 1024 B apart; a K step of
    // 16 BF16 is 32 bytes inside the swizzle row.  B: N-major (row k of B =
    // 128 bytes of 64 N values), 128-byte swizzle; 64-wide N chunks are
    // 64 rows x 128 B = 8 KB apart (LBO), 8-row K groups 1024 B apart (SBO);
    // a K step of 16 rows = 2 KB.
    const uint64_t a_desc0 = tc::smem_desc(sbase, 16, 1024, 2);
    const uint64_t b_desc0 = tc::smem_desc(sbase + MH * kABytes, kTK * 128, 1024, 2);
    int seg = -1;
    int st = 0;
    uint32_t ph = 0;
    bool ok = true;
    Cursor c = cursor_at<NP, MH>(T, u0);
    int bsel = NBUF - 1;      // accumulator set of the current segment
    uint32_t bph = 1;         // its acc_empty parity (flips each reuse)
    const int kc = T.kchunk;
    // 128-row tiles: two K slabs per iteration when both belong to the same
    // accumulator segment.  Every ring step (a wait on a full stage, a
    // commit) costs this warp a few hundred cycles, about what the four MMAs
    // of one 128-row slab take on the tensor pipe.  (A 256-row stage already
    // holds eight MMAs; pairing its three stages would leave the ring too
    // shallow to cover the commit -> producer -> consumer round trip.)
    constexpr int kPair = MH == 1 ? 2 : 1;
    auto seg_end_after = [&](int64_t uu, int sl) {
      return (uu + 1 == u1) || sl + 1 == c.slabs || (kc && (sl + 1) % kc == 0);
    };
    for (int64_t u = u0; u < u1;) {
      const int slab = c.slab;
      const bool first = (u == u0) || slab == 0 || (kc && slab % kc == 0);
      const bool end1 = seg_end_after(u, slab);
      const int n = (end1 || kPair == 1) ? 1 : 2;   // slabs this iteration
      const bool last = n == 1 ? end1 : seg_end_after(u + 1, slab + 1);
      if (first) {
        ++seg;
        if (++bsel == NBUF) {
          bsel = 0;
          bph ^= 1u;
        }
        // the epilogue must have drained this accumulator (segment seg - NBUF)
        if (seg >= NBUF &&
            !__all_sync(0xffffffffu, mbar_wait_bounded(&acc_empty[bsel], bph ^ 1u, T.status))) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
      }
      const int st2 = st + 1 == S ? 0 : st + 1;
      const uint32_t ph2 = st + 1 == S ? ph ^ 1u : ph;
      bool got = mbar_wait_bounded(&full[st], ph, T.status);
      if (n == 2) got = got && mbar_wait_bounded(&full[st2], ph2, T.status);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      if (lane == 0) {
        const uint32_t d_tmem = tmem + (uint32_t)(bsel * MH * TN);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          if (j == n) break;
          const int sj = j ? st2 : st;
          const uint64_t so = (uint64_t)((sj * kStageBytes) >> 4);
#pragma unroll
          for (int kk = 0; kk < kTK / 16; ++kk) {
            const uint64_t bd = b_desc0 + so + (uint64_t)((kk * 16 * 128) >> 4);
#pragma unroll
            for (int hh = 0; hh < MH; ++hh) {
              const uint64_t ad = a_desc0 + so + (uint64_t)((hh * kABytes + kk * 32) >> 4);
              tc::mma_bf16(d_tmem + hh * TN, ad, bd, idesc, (!first || j > 0 || kk > 0) ? 1u : 0u);
            }
          }
          tc::mma_commit(&empty[sj]);               // stage free once these MMAs finish
        }
        if (last) tc::mma_commit(&acc_full[bsel]);  // accumulator complete
      }
      __syncwarp();
      for (int j = 0; j < n; ++j) {
        cursor_next<NP, MH>(T, c);
        if (++st == S) {
          st = 0;
          ph ^= 1u;
        }
      }
      u += n;
    }
    if (!ok && lane == 0) {
      // make the epilogue's waits end: release every accumulator it expects
      for (int b = 0; b < NBUF; ++b) tc::mma_commit(&acc_full[b]);
    }
    // every MMA is issued: the next launch in the stream may start its
    // prologue during this CTA's epilogue
    if (lane == 0) pdl_trigger();
  } else {
    // ---------------- epilogue: TMEM -> registers -> C -----------------------
    // C may still be being zero-filled by the kernel this launch depends on
    // (programmatic dependent launch): wait for it before any write to C.
    // Without such a dependency the wait returns at once.
    pdl_wait();
    const int quarter = warp & 3;                  // TMEM lanes 32 quarter .. + 31
    const int part = (warp - 2) >> 2;              // column part of this warp
    constexpr int kParts = kEpiWarps / 4;
    uint8_t* my_stage = stage_c + (size_t)(warp - 2) * kStagePerWarp * kStageC;
    int chunk = 0;   // staging tiles alternate per chunk
    Cursor c = cursor_at<NP, MH>(T, u0);
    int b = NBUF - 1;
    uint32_t bph = 1;
    // one iteration per segment: the slabs of one tile inside [u0, u1)
    for (int64_t u = u0; u < u1;) {
      const DenseProb& P = T.p[c.q];
      const int q = c.q;
      // the segment ends at the tile's end, the K chunk's end or the range's
      const int seg_end = T.kchunk ? min(c.slabs, (c.slab / T.kchunk + 1) * T.kchunk) : c.slabs;
      int64_t ue = u + (seg_end - c.slab);
      if (ue > u1) ue = u1;
      const bool whole = (c.slab == 0) && (ue - u == c.slabs);
      const int mt = c.mt, nt = c.nt;
      if (++b == NBUF) {
        b = 0;
        bph ^= 1u;
      }
      // the tiles' C rows, fetched while the MMAs run
      int32_t trow[MH];
#pragma unroll
      for (int hh = 0; hh < MH; ++hh) {
        const int copy = mt * MH + hh;
        trow[hh] = copy < P.n_copy ? __ldg(&P.tile_order[copy]) : 0;
      }
      // the problem's scalars in registers for the chunk loop
      const int64_t PM = P.M, PN = P.N;
      const int n_copy = P.n_copy, tma_c = P.tma_c, out_i32 = T.out_i32;
      const bool add = !whole || P.accumulate;
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&acc_full[b], bph, T.status));
      tc::fence_after_sync();
      const int64_t n0 = (int64_t)nt * TN;
#pragma unroll
      for (int hh = 0; hh < MH; ++hh) {
        const int copy = mt * MH + hh;
        if (copy >= n_copy) break;   // warp-uniform
        const int64_t row0 = (int64_t)trow[hh] * kTM + quarter * 32;
#pragma unroll 1
        for (int cc = part * (TN / 32 / kParts); cc < (part + 1) * (TN / 32 / kParts); ++cc) {
          uint32_t r[32];
          tc::tmem_ld_32x32b_x32(tmem + ((uint32_t)(quarter * 32) << 16) +
                                     (uint32_t)(b * MH * TN + hh * TN + cc * 32),
                                 r);
          tc::tmem_ld_wait();
          const int64_t col0 = n0 + cc * 32;
          if (!ok || row0 >= PM || col0 >= PN) continue;   // warp-uniform
          if (out_i32) {
            // an exact integer in FP32 (|partial| < 2^24): convert to INT32
#pragma unroll
            for (int j = 0; j < 32; ++j) r[j] = (uint32_t)__float2int_rn(__uint_as_float(r[j]));
          }
          if (tma_c) {
            // staging tile (chunk & 1) is free once the copy issued two
            // chunks ago has read it
            uint8_t* buf = my_stage + (size_t)(chunk % kStagePerWarp) * kStageC;
            if (lane == 0) bulk_wait_read<kStagePerWarp - 1>();
            __syncwarp();
            // row `lane`, 16-byte chunk j at (j ^ (lane % 8)): the 128-byte swizzle
#pragma unroll
            for (int j = 0; j < 8; ++j)
              *reinterpret_cast<uint4*>(buf + lane * 128 + ((j ^ (lane & 7)) << 4)) =
                  make_uint4(r[4 * j], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
              // rows past M and columns past N are clipped by the tensor map
              if (add) tma_reduce_add_2d(&T.tmC[q], (int32_t)col0, (int32_t)row0, buf);
              else tma_store_2d(&T.tmC[q], (int32_t)col0, (int32_t)row0, buf);
              bulk_commit();
            }
            ++chunk;
            continue;
          }
          // C rows not 16-byte aligned (no tensor map): transpose the 32 x 32
          // chunk through this warp's staging tile (rotated rows, no bank
          // conflicts) so that each store instruction writes 32 consecutive
          // columns of one row
          float* tr = reinterpret_cast<float*>(my_stage);
          // the staging tiles may still be read by this warp's TMA stores of
          // an earlier problem of the batch (one with aligned C rows): wait
          // until those reads are done before reusing the space
          if (lane == 0) bulk_wait_read<0>();
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 32; ++j) tr[lane * 32 + ((j + lane) & 31)] = __uint_as_float(r[j]);
          __syncwarp();
          const int64_t col = col0 + lane;
          const int rows = (int)(PM - row0 < 32 ? PM - row0 : 32);
          if (col < PN) {
#pragma unroll 4
            for (int rr = 0; rr < rows; ++rr) {
              const float v = tr[rr * 32 + ((lane + rr) & 31)];
              float* dst = P.C + (row0 + rr) * P.ldc + col;
              if (out_i32) {
                int* di = reinterpret_cast<int*>(dst);
                const int iv = (int)__float_as_uint(v);   // already converted
                if (add) atomicAdd(di, iv);
                else *di = iv;
              } else if (add) {
                atomicAdd(dst, v);   // a cut tile, or C += A.B
              } else {
                *dst = v;
              }
            }
          }
        }
      }
      // accumulator drained: hand it back to the MMA issuer
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
      const int adv = (int)(ue - u);
      u = ue;
      if (c.slab + adv >= c.slabs) cursor_next_tile<NP, MH>(T, c);
      else c.slab += adv;   // the next K chunk of the same tile
    }
    // the staging tiles must not be released (CTA exit) while TMA reads
    // them, and C must be complete when the kernel ends
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 1) tc::tmem_dealloc(tmem, NBUF * MH * TN);
}

template <int TN, int MH>
size_t dense_smem_bytes(int stages) {
  return 1024 + (size_t)stages * (MH * kABytes + (size_t)TN * kTK * 2) + kEpiBytes + 256;
}

template <int TN, int MH>
constexpr int dense_stages() {
  return (200 * 1024) / (MH * kABytes + TN * kTK * 2) > 6 ? 6
                                                         : (200 * 1024) / (MH * kABytes + TN * kTK * 2);
}

int64_t slabs_of(int64_t K) { return (K + kTK - 1) / kTK; }

template <int TN, int NP, int MH>
rosko_status launch_table(DenseTable<NP>& T, int64_t grid, bool pdl, cudaStream_t st) {
  const size_t smem = dense_smem_bytes<TN, MH>(T.stages);
  static size_t set = 0;
  auto fn = dense_panel_kernel<TN, NP, MH>;
  if (smem > set) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return ROSKO_ERR_CUDA;
    set = smem;
  }
  if (pdl) {
    // starts while the preceding zero fill runs; its epilogue waits for it
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, fn, T) != cudaSuccess) return ROSKO_ERR_CUDA;
  } else {
    fn<<<(unsigned)grid, kThreads, smem, st>>>(T);
  }
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
}

rosko_status encode_dense_maps(const DenseJob& j, int MH, CUtensorMap* mA, CUtensorMap* mB,
                               CUtensorMap* mC, bool c_ok, int TN, bool* b3d) {
  if (c_ok) {
    const cuuint64_t dims[2] = {(cuuint64_t)j.N, (cuuint64_t)j.M};
    const cuuint64_t strides[1] = {(cuuint64_t)j.ldc * 4};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t es[2] = {1, 1};
    if (encode_tiled(mC, j.out_i32 ? CU_TENSOR_MAP_DATA_TYPE_INT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                     2, j.C, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return ROSKO_ERR_INVALID_ARG;
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)j.Kpad, (cuuint64_t)j.dense_rows};
    const cuuint64_t strides[1] = {(cuuint64_t)j.Kpad * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kTK, (cuuint32_t)(kTM * MH)};
    const cuuint32_t es[2] = {1, 1};
    if (encode_tiled(mA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(j.dense_A), dims,
                     strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return ROSKO_ERR_INVALID_ARG;
  }
  *b3d = false;
  if (j.N % 64 == 0) {
    // B viewed as [N / 64][K][64]: chunk z starts 128 bytes after chunk z-1
    const cuuint64_t dims[3] = {64, (cuuint64_t)j.K, (cuuint64_t)(j.N / 64)};
    const cuuint64_t strides[2] = {(cuuint64_t)j.ldb * 2, 128};
    const cuuint32_t box[3] = {64, (cuuint32_t)kTK, (cuuint32_t)(TN / 64)};
    const cuuint32_t es[3] = {1, 1, 1};
    *b3d = encode_tiled(mB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(j.B), dims,
                        strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  if (!*b3d) {
    const cuuint64_t dims[2] = {(cuuint64_t)j.N, (cuuint64_t)j.K};
    const cuuint64_t strides[1] = {(cuuint64_t)j.ldb * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)kTK};
    const cuuint32_t es[2] = {1, 1};
    if (encode_tiled(mB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(j.B), dims,
                     strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return ROSKO_ERR_INVALID_ARG;
  }
  return ROSKO_OK;
}

// Tile-granular split when there are at least two tiles per CTA: the
// stream-K balance is then not needed and uncut tiles need no zero fill of C
// and no reductions.
static bool use_aligned(int64_t tiles, int64_t G) { return tiles >= 2 * G; }

// Stream-K pieces shorter than this many K slabs cost more in reductions
// (every piece adds its partial tile into C) than they gain in balance.
constexpr int64_t kMinUnitsPerCta = 8;

// CTAs of a launch over `units` (tile, slab) units in `tiles` tiles: one per
// SM at most, and no stream-K piece shorter than kMinUnitsPerCta slabs.
static int64_t grid_for(int64_t units, int64_t tiles, int ctas) {
  // (the kernel's 32-bit split arithmetic wants G < 2^16)
  int64_t G = std::min<int64_t>(std::min(ctas, 65535), units);
  if (!use_aligned(tiles, G)) G = std::min<int64_t>(G, std::max(tiles, units / kMinUnitsPerCta));
  return std::max<int64_t>(1, G);
}

template <int TN, int NP, int MH>
rosko_status run_jobs(const DenseJob* jobs, int count, int ctas, cudaStream_t st) {
  static_assert(sizeof(DenseTable<NP>) <= 32 * 1024 - 256, "kernel parameter table too large");
  DenseTable<NP> T;
  std::memset(static_cast<void*>(&T), 0, sizeof(T));
  int64_t units = 0;
  int n = 0;
  for (int i = 0; i < count; ++i) {
    const DenseJob& j = jobs[i];
    if (j.n_tiles <= 0 || j.N <= 0) continue;
    const bool c_ok = ((reinterpret_cast<uintptr_t>(j.C) % 16) == 0) && ((j.ldc * 4) % 16 == 0);
    bool b3d = false;
    rosko_status s = encode_dense_maps(j, MH, &T.tmA[n], &T.tmB[n], &T.tmC[n], c_ok, TN, &b3d);
    if (s != ROSKO_OK) return s;
    DenseProb& P = T.p[n];
    P.tma_c = c_ok ? 1 : 0;
    P.b3d = b3d ? 1 : 0;
    P.tile_order = j.tile_order_dev;
    P.C = j.C;
    P.ldc = j.ldc;
    P.M = j.M;
    P.N = j.N;
    P.unit0 = units;
    P.n_copy = (int)j.n_tiles;
    P.n_ntiles = (int)((j.N + TN - 1) / TN);
    P.slabs = (int)slabs_of(j.K);
    P.accumulate = j.accumulate;
    P.vec_ok = ((reinterpret_cast<uintptr_t>(j.C) % 16) == 0) && ((j.ldc * 4) % 16 == 0);
    units += (int64_t)((P.n_copy + MH - 1) / MH) * P.n_ntiles * P.slabs;
    ++n;
  }
  if (n == 0) return ROSKO_OK;
  // the kernel splits and walks units in 32-bit arithmetic
  if (units >= (int64_t(1) << 31)) return ROSKO_ERR_UNSUPPORTED;
  T.count = n;
  T.units = units;
  int64_t tiles = 0;
  for (int i = 0; i < n; ++i) tiles += (int64_t)((T.p[i].n_copy + MH - 1) / MH) * T.p[i].n_ntiles;
  const int64_t grid = grid_for(units, tiles, ctas);
  T.aligned = use_aligned(tiles, grid) ? 1 : 0;
  T.kchunk = jobs[0].kchunk;
  T.out_i32 = jobs[0].out_i32;
  T.stages = dense_stages<TN, MH>();
  T.status = device_status_word();
  if (!T.status) return ROSKO_ERR_CUDA;
  return launch_table<TN, NP, MH>(T, grid, jobs[0].pdl != 0, st);
}

}  // namespace

static int64_t job_units(int64_t n_tiles, int64_t N, int64_t K, int TN, int MH) {
  return ((n_tiles + MH - 1) / MH) * ((N + TN - 1) / TN) * slabs_of(K);
}

int64_t dense_grid(int64_t n_tiles, int64_t N, int64_t K, int TN, int ctas, int MH) {
  const int64_t units = job_units(n_tiles, N, K, TN, MH);
  return grid_for(units, units / slabs_of(K), ctas);
}

// True when the stream-K split of `units` over `ctas` CTAs cuts some tile of
// `slabs` units (those tiles are accumulated with atomics into a zeroed C).
static bool split_cuts_tile(int64_t units_before, int64_t units, int64_t total, int64_t slabs,
                            int64_t G) {
  for (int64_t b = 0; b <= G; ++b) {
    const int64_t u = total * b / G;
    if (u <= units_before || u >= units_before + units) continue;
    if ((u - units_before) % slabs != 0) return true;
  }
  return false;
}

bool dense_needs_zero(int64_t n_tiles, int64_t N, int64_t K, int TN, int ctas, int MH) {
  const int64_t units = job_units(n_tiles, N, K, TN, MH);
  const int64_t G = dense_grid(n_tiles, N, K, TN, ctas, MH);
  if (use_aligned(units / slabs_of(K), G)) return false;
  return split_cuts_tile(0, units, units, slabs_of(K), G);
}

// For a batch: which jobs have a tile cut between CTAs (job order as given).
void dense_batch_needs_zero(const DenseJob* jobs, int count, int TN, int ctas, int MH,
                            bool* out) {
  int64_t total = 0;
  for (int i = 0; i < count; ++i)
    if (jobs[i].n_tiles > 0 && jobs[i].N > 0)
      total += job_units(jobs[i].n_tiles, jobs[i].N, jobs[i].K, TN, MH);
  int64_t tiles = 0;
  for (int i = 0; i < count; ++i)
    if (jobs[i].n_tiles > 0 && jobs[i].N > 0)
      tiles += job_units(jobs[i].n_tiles, jobs[i].N, jobs[i].K, TN, MH) / slabs_of(jobs[i].K);
  const int64_t G = grid_for(total, tiles, ctas);
  const bool aligned = use_aligned(tiles, G);
  int64_t before = 0;
  for (int i = 0; i < count; ++i) {
    out[i] = false;
    if (aligned) continue;
    if (jobs[i].n_tiles <= 0 || jobs[i].N <= 0) continue;
    const int64_t units = job_units(jobs[i].n_tiles, jobs[i].N, jobs[i].K, TN, MH);
    out[i] = split_cuts_tile(before, units, total, slabs_of(jobs[i].K), G);
    before += units;
  }
}

template <int NP>
static rosko_status dispatch_jobs(const DenseJob* jobs, int count, int TN, int MH, int ctas,
                                  cudaStream_t st) {
  if (TN == 256 && MH == 2) return run_jobs<256, NP, 2>(jobs, count, ctas, st);
  if (TN == 256) return run_jobs<256, NP, 1>(jobs, count, ctas, st);
  if (MH == 2) return run_jobs<128, NP, 2>(jobs, count, ctas, st);
  return run_jobs<128, NP, 1>(jobs, count, ctas, st);
}

rosko_status dense_batch_launch(const DenseJob* jobs, int count, int TN, int ctas, int MH,
                                cudaStream_t st) {
  if (count <= 0) return ROSKO_OK;
  if ((TN != 128 && TN != 256) || (MH != 1 && MH != 2)) return ROSKO_ERR_INVALID_ARG;
  if (ctas <= 0) ctas = num_sms();
  if (count == 1) return dispatch_jobs<1>(jobs, 1, TN, MH, ctas, st);
  if (count <= 64) return dispatch_jobs<64>(jobs, count, TN, MH, ctas, st);
  return ROSKO_ERR_INVALID_ARG;
}

namespace {
// Zero rows x row_bytes of C (pitch bytes apart), one CTA per row at a time.
// Dependents may launch at once: they wait (griddepcontrol.wait) before
// touching C.
__global__ void zero_fill_kernel(char* __restrict__ C, int64_t pitch, int64_t row_bytes,
                                 int64_t rows, int vec16) {
  pdl_trigger();   // the tensor-core launch after it starts at once
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    char* row = C + r * pitch;
    if (vec16) {
      uint4* p = reinterpret_cast<uint4*>(row);
      for (int64_t i = threadIdx.x; i < row_bytes / 16; i += blockDim.x) p[i] = make_uint4(0, 0, 0, 0);
    } else {
      uint32_t* p = reinterpret_cast<uint32_t*>(row);
      for (int64_t i = threadIdx.x; i < row_bytes / 4; i += blockDim.x) p[i] = 0u;
    }
  }
}

// INT8 -> BF16 (exact: |code| <= 127), K rows of N, into rows of ldo.
__global__ void i8_to_bf16_kernel(const int8_t* __restrict__ B, int64_t K, int64_t N, int64_t ldb,
                                  __nv_bfloat16* __restrict__ out, int64_t ldo) {
  const int64_t cols = (ldo + 3) / 4;   // four values per thread
  const int64_t n = K * cols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / cols, c0 = (i - k * cols) * 4;
    __nv_bfloat16 v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t c = c0 + j;
      v[j] = __float2bfloat16_rn(c < N ? (float)B[k * ldb + c] : 0.0f);
      if (c < ldo) out[k * ldo + c] = v[j];
    }
  }
}
}  // namespace

rosko_status zero_fill_launch(const ZeroFill& z, cudaStream_t st) {
  if (z.rows <= 0 || z.row_bytes <= 0) return ROSKO_OK;
  // every C element type is a multiple of 4 bytes
  if ((reinterpret_cast<uintptr_t>(z.C) % 4) != 0 || z.pitch % 4 != 0 || z.row_bytes % 4 != 0)
    return ROSKO_ERR_INVALID_ARG;
  const int vec16 = (reinterpret_cast<uintptr_t>(z.C) % 16 == 0 && z.pitch % 16 == 0 &&
                     z.row_bytes % 16 == 0)
                        ? 1
                        : 0;
  // a grid that is resident at once, so that every CTA has signalled its
  // dependents before the tensor-core launch needs an SM
  const int64_t grid = std::min<int64_t>(z.rows, (int64_t)num_sms() * 4);
  // an ordinary launch: when it starts, every launch before it has completed,
  // so its programmatic dependent (the tensor-core kernel) may read A and B
  // at once; only that kernel's writes of C wait for the fill
  zero_fill_kernel<<<(unsigned)grid, 256, 0, st>>>(static_cast<char*>(z.C), z.pitch, z.row_bytes,
                                                   z.rows, vec16);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
}

// K slabs of 64 per exact chunk: 16 slabs = 1024 products of magnitude
// <= 127^2, so a partial sum stays below 1024 * 16129 < 2^24 and is exact in
// the FP32 accumulator.
constexpr int kI8ChunkSlabs = 16;

rosko_status dense_spmm_i8_launch(const rosko_packed_s* h, int64_t n_tiles, const int8_t* B,
                                  int64_t N, int64_t ldb, int32_t* C, int64_t ldc, int TN,
                                  int ctas, int MH, const ZeroFill* zf, cudaStream_t st) {
  if (n_tiles <= 0 || N <= 0) return ROSKO_OK;
  if (TN != 128 && TN != 256) return ROSKO_ERR_INVALID_ARG;
  if (ctas <= 0) ctas = num_sms();
  const int64_t K = h->K;
  const int64_t ldo = (N + 7) / 8 * 8;   // 16-byte rows for the tensor map
  void* scratch = nullptr;
  // stream-ordered (and capturable) from the library's pool, which keeps
  // freed memory mapped: released after the launch that reads it
  if (pool_malloc(&scratch, (size_t)std::max<int64_t>(K * ldo, 1) * 2, st) != cudaSuccess)
    return ROSKO_ERR_OOM;
  const int64_t work = K * ((ldo + 3) / 4);
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 4096));
  i8_to_bf16_kernel<<<blocks, 256, 0, st>>>(B, K, N, ldb, static_cast<__nv_bfloat16*>(scratch),
                                            ldo);
  count_launches(1);
  rosko_status s = cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
  // the zero fill of C (after the conversion, so that B is complete when the
  // dependent tensor-core launch starts)
  if (s == ROSKO_OK && zf) s = zero_fill_launch(*zf, st);
  if (s == ROSKO_OK) {
    DenseJob j;
    j.dense_A = h->dense_A;
    j.dense_rows = h->n_copy * kTM;
    j.Kpad = h->Kpad;
    j.tile_order_dev = h->tile_order_dev;
    j.n_tiles = n_tiles;
    j.K = K;
    j.B = scratch;
    j.N = N;
    j.ldb = ldo;
    j.C = reinterpret_cast<float*>(C);
    j.ldc = ldc;
    j.M = h->M;
    j.accumulate = 1;   // every chunk adds into the zeroed (or accumulated) C
    j.kchunk = kI8ChunkSlabs;
    j.out_i32 = 1;
    j.pdl = zf ? 1 : 0;
    s = dense_batch_launch(&j, 1, TN, ctas, MH, st);
  }
  pool_free(scratch, st);
  return s;
}

rosko_status dense_spmm_launch(const void* dense_A, int64_t dense_rows, int64_t Kpad,
                               const int32_t* tile_order_dev, int64_t n_tiles, int64_t K,
                               const void* B, int64_t N, int64_t ldb, float* C, int64_t ldc,
                               int64_t M, int accumulate, int TN, int ctas, int MH,
                               bool c_zeroed, const ZeroFill* zf, cudaStream_t st) {
  if (n_tiles <= 0 || N <= 0) return ROSKO_OK;
  if (TN != 128 && TN != 256) return ROSKO_ERR_INVALID_ARG;
  if (ctas <= 0) ctas = num_sms();
  if (zf) {
    rosko_status s = zero_fill_launch(*zf, st);
    if (s != ROSKO_OK) return s;
  } else if (!accumulate && !c_zeroed && dense_needs_zero(n_tiles, N, K, TN, ctas, MH)) {
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
  DenseJob j;
  j.dense_A = dense_A;
  j.dense_rows = dense_rows;
  j.Kpad = Kpad;
  j.tile_order_dev = tile_order_dev;
  j.n_tiles = n_tiles;
  j.K = K;
  j.B = B;
  j.N = N;
  j.ldb = ldb;
  j.C = C;
  j.ldc = ldc;
  j.M = M;
  j.accumulate = accumulate;
  // a programmatic dependent of its zero fill only (it reads A and B before
  // any wait, which is safe only after a launch that started after every
  // earlier one had completed)
  j.pdl = zf ? 1 : 0;
  return dense_batch_launch(&j, 1, TN, ctas, MH, st);
}

}  // namespace rosko
