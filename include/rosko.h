/*
 * rosko.h - C ABI of the GB300 (sm_103a) row-skipping outer-product SpMM.
 *
 * Method (Rosko, arXiv 2307.03930): C = A.B with A an unstructured sparse
 * weight matrix (M x K) and B a dense activation matrix (K x N).  Sec. 3: the
 * outer product of column k of A with row k of B only touches the result rows
 * m with A[m,k] != 0, so the other rows are skipped.  Sec. 4.1 / Alg. 1: A is
 * packed per row panel into the nonzero values of each non-empty column (A_p),
 * their panel-relative rows (loc_m), the column indices (col_ind) and the
 * per-column counts (nnz).  Alg. 2 streams the packed columns, loads the
 * matching row of B once and multiply-accumulates it into the register-
 * resident C rows named by loc_m.
 *
 * Conventions shared by every call
 *   - Pointers named *_dev are CUDA device pointers (or managed memory) on the
 *     current device; *_host are host pointers.  The caller owns A, B, C and
 *     the stream.  The library owns a packed handle until rosko_free.
 *   - Matrices are row-major with an explicit leading dimension in ELEMENTS:
 *     A[m*lda + k], B[k*ldb + n], C[m*ldc + n] (Alg. 1 indexes A as A[k + mK]).
 *   - Every call is ordered on the given stream (NULL = legacy default stream)
 *     and returns without synchronising, except where stated.
 *   - Arguments are validated on the host before any launch; an invalid
 *     argument returns ROSKO_ERR_INVALID_ARG and launches nothing.  Calls never
 *     abort the process.  A kernel that detects an internal error (a bounded
 *     wait that ran out, a corrupt packed stream) sets a bit in a per-device
 *     status word read by rosko_device_status.
 *   - Sizes are int64; the total nonzero count and the total number of packed
 *     columns of one handle must stay below 2^31.
 */
#ifndef ROSKO_H_
#define ROSKO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ROSKO_OK = 0,
  ROSKO_ERR_INVALID_ARG = 1,  /* bad size, pointer, dtype, alignment or tile   */
  ROSKO_ERR_UNSUPPORTED = 2,  /* valid request the library does not implement */
  ROSKO_ERR_OOM = 3,          /* a device allocation failed                    */
  ROSKO_ERR_CUDA = 4,         /* a CUDA runtime/driver call failed             */
  ROSKO_ERR_TIMEOUT = 5,      /* a bounded device wait ran out                 */
  ROSKO_ERR_BAD_HANDLE = 6,   /* NULL, freed or corrupt packed handle          */
  ROSKO_ERR_DEVICE = 7        /* a kernel reported an internal error           */
} rosko_status;

typedef enum {
  ROSKO_F32 = 0,
  ROSKO_BF16 = 1,
  ROSKO_I8 = 2,
  ROSKO_F64 = 3,  /* check mode only: FP64 accumulation of FP32-exact inputs */
  ROSKO_I32 = 4
} rosko_dtype;

/* Opaque handle to a packed A (device buffers owned by the library). */
typedef struct rosko_packed_s* rosko_packed_t;
/* A cudaStream_t passed as an untyped pointer (NULL = legacy default stream). */
typedef void* rosko_stream_t;

typedef enum {
  ROSKO_SCHED_ANALYTIC = 0,  /* closed-form tile rule (Sec. 4.2 re-derived)  */
  ROSKO_SCHED_AUTOTUNE = 1,  /* per-shape timed search, cached               */
  ROSKO_SCHED_LEARNED = 2,   /* MLP selector over problem features           */
  ROSKO_SCHED_FORCED = 3     /* use the tile exactly as given                */
} rosko_sched_mode;

/*
 * Tile parameters (Sec. 4.2 and Sec. 6 expose m_c, k_c, m_r, n_r).
 *   m_r   rows per packed panel = C rows one warp holds in registers
 *         (8, 16 or 32); fixed when A is packed.
 *   n_r   C columns per CTA tile (32 lanes x columns per lane).
 *   k_c   rows of B staged in shared memory per pipeline slab.
 *   m_c   C rows per CTA = warps per CTA x m_r.
 *   split_k  number of K ranges reduced into C with atomics (>= 1).
 *   dense_split_pm  BF16, and INT8 with an INT32 result: 128-row tiles of A
 *         whose density in per mille (nonzeros per 1000 entries) is >= this
 *         value run on the tensor-core dense-panel path, the others on the
 *         sparse path; >= 1001 = never.  At pack time the same field is the
 *         minimum density for which a dense copy is kept.
 *   dense_n_r      C columns per tensor-core CTA tile (128 or 256).
 *   dense_split_k  CTAs over which the stream-K tensor-core path divides its
 *         (tile, K slab) work (default: one per SM); a tile whose K range
 *         is divided is added into C with atomics.
 *   order traversal of a panel inside a B slab by the CUDA-core path:
 *         1 = column order, Alg. 2 as printed (one B row per packed column,
 *         the C row picked by a run-time switch over loc_m);
 *         2 = row-slot order (each register row of C walks its own
 *         nonzeros and reads their B rows from the shared slab; needs
 *         K < 65280);
 *         3 = row-slot order over a gather of only the B rows the CTA's
 *         128-row tile touches (the tile's col_ind); needs m_r = 16,
 *         m_c = 128.
 *   mode  a rosko_sched_mode.
 *   dense_m_c  C rows per tensor-core CTA tile: 128 (one MMA per K step) or
 *         256 (two 128-row MMAs sharing each staged B slab).
 * A field <= 0 means "library chooses" (except in ROSKO_SCHED_FORCED, where
 * the sparse fields must be set and dense fields <= 0 still mean default).
 */
typedef struct {
  int32_t m_r;
  int32_t n_r;
  int32_t k_c;
  int32_t m_c;
  int32_t split_k;
  int32_t dense_split_pm;
  int32_t dense_n_r;
  int32_t dense_split_k;
  int32_t order;
  int32_t mode;
  int32_t dense_m_c;
} rosko_tile;

/* Human-readable name of a status code (static string, never NULL). */
const char* rosko_status_string(rosko_status s);

/*
 * rosko_pack - Alg. 1 on the device, per row panel of m_r rows.
 *
 * A_dev   dense row-major M x K matrix of type a_dtype, leading dim lda >= K.
 * a_dtype ROSKO_F32, ROSKO_BF16 or ROSKO_I8.
 * packed_dtype  storage type of the nonzeros:
 *           F32  from F32 (copy);   BF16 from F32 (round to nearest even) or BF16;
 *           I8   from F32 (per-row symmetric scale s_i = max_k|a_ik|/127,
 *                q = clamp(rint(a/s_i), -127, 127), mask = q != 0) or from I8
 *                (row_scale_dev gives the scales, NULL = all 1);
 *           F64  from F32 (exact widening; FP64 check mode).
 * Limits: at most 65535 panels (M <= 65535 * m_r) and M * K < 2^31.
 * row_scale_dev  I8-from-I8 only: M FP32 row scales (device), else NULL.
 * tile    only tile->m_r and, for BF16 and INT8, tile->dense_split_pm
 *         (minimum tile density, per mille, for keeping a dense BF16 copy of
 *         the tile - the values, or the INT8 codes; <= 0: 1 per mille for
 *         BF16, 10 for INT8) are read.
 *         m_r <= 0: 16.
 * out     receives the new handle (set to NULL on error).
 * Zero test: IEEE a != 0, so -0.0 is dropped and NaN/Inf are kept.
 * Synchronises `stream` twice: once to size the packed buffers, and once
 * before returning, so that the handle is ready for use on any stream.  Device
 * memory (scratch and the handle) comes from the library's stream-ordered pool
 * (see rosko_free).  M or K may be 0.
 */
rosko_status rosko_pack(const void* A_dev, rosko_dtype a_dtype, int64_t M, int64_t K,
                        int64_t lda, rosko_dtype packed_dtype, const float* row_scale_dev,
                        const rosko_tile* tile, rosko_stream_t stream, rosko_packed_t* out);

/*
 * rosko_pack_transposed - rosko_pack of the K x M transpose of the dense
 * row-major M x K matrix A_dev, for the other SpMM of a pruned layer's
 * training step (the input gradient W^T . dO of Sec. 5.4's CNN training).  Same
 * rules as rosko_pack with the roles of M and K exchanged (I8-from-I8 row
 * scales are per row of the transpose, i.e. per column of A).  A K x M
 * scratch copy is allocated for the transpose and freed before returning;
 * synchronises `stream`.
 */
rosko_status rosko_pack_transposed(const void* A_dev, rosko_dtype a_dtype, int64_t M, int64_t K,
                                   int64_t lda, rosko_dtype packed_dtype,
                                   const float* row_scale_dev, const rosko_tile* tile,
                                   rosko_stream_t stream, rosko_packed_t* out);

/*
 * rosko_spmm - C = A.B (accumulate = 0) or C += A.B (accumulate = 1, the
 * in-place accumulation of Alg. 2, which loads C first).
 *
 * A       packed handle.  B_dev: K x N row-major of type b_dtype, leading dim
 *         ldb >= N; B_dev and ldb * sizeof(b_dtype) must be 16-byte aligned
 *         (B slabs are moved by TMA).  C_dev: M x N row-major, ldc >= N.
 * Supported (packed, b_dtype -> c_dtype):
 *         (F32, F32 -> F32), (BF16, BF16 -> F32), (I8, I8 -> I32),
 *         (I8, I8 -> F32: C = s_i * t_j * sum q_a q_b with col_scale_dev = t),
 *         (F64, F32 -> F64, check mode).
 * col_scale_dev  N FP32 column scales of B for (I8, I8 -> F32), else NULL.
 * tile    NULL = analytic rule; otherwise see rosko_tile.
 * Accumulation: FP32 (FP64 in check mode, INT32 exact for I8) in registers.
 * With split_k > 1 partial sums are added with atomics, so FP results may
 * differ run to run in the last bits.  N may be 0 (no-op).
 * Dense-panel tiles (BF16) multiply their explicit zeros too, so there a
 * non-finite B value meets 0 * Inf = NaN, while skipped rows never see it.
 * INT8 packs with an INT32 result run their dense-enough tiles on the same
 * tensor-core path, exactly: the codes are integers exact in BF16, every K
 * chunk of at most 1024 sums below 2^24 in magnitude (exact in the FP32
 * accumulator) and is added into C as INT32, so the result is bit-identical
 * to the integer sum; the call converts B to BF16 in stream-ordered scratch
 * (K x N x 2 bytes from the library's device memory pool on `stream`,
 * released in stream order).  The FP32 (dequantised) INT8 result stays on
 * the CUDA-core path.
 * Stream order: when C must be zero-filled first (tiles or rows cut along K
 * and added), the fill is a small kernel ahead of a tensor-core launch, else
 * a memset.  The tensor-core kernel is launched as a programmatic dependent
 * of that fill (it reads A and B at once and writes C only after the fill),
 * and the row-direct kernel as a programmatic dependent of whatever kernel
 * precedes it on `stream` (it reads nothing before that kernel has
 * completed).  Both keep ordinary stream-order semantics for the caller;
 * they only let the launch overlap its predecessor's tail.
 * The row-direct traversal numbers its work items (row pieces x column
 * strips of n_r columns) with 31 bits; beyond that it returns
 * ROSKO_ERR_UNSUPPORTED.
 */
rosko_status rosko_spmm(rosko_packed_t A, const void* B_dev, rosko_dtype b_dtype, int64_t N,
                        int64_t ldb, const float* col_scale_dev, void* C_dev,
                        rosko_dtype c_dtype, int64_t ldc, int accumulate,
                        const rosko_tile* tile, rosko_stream_t stream);

/* The work split one rosko_spmm call runs (see rosko_spmm_plan). */
typedef struct {
  int64_t dense_tiles;    /* 128-row tiles on the tensor-core path            */
  int64_t sparse_panels;  /* m_r-row panels on the CUDA-core path             */
  int32_t order;          /* CUDA-core traversal (1..4), 0 when no panel      */
  int32_t zero_fill;      /* 1 when C is zero-filled before the kernels       */
  rosko_tile tile;        /* the schedule resolved for the call               */
} rosko_plan;

/*
 * rosko_spmm_plan - what rosko_spmm with the same arguments would run,
 * without running it: the split between the tensor-core and CUDA-core
 * paths, the traversal and the resolved tile.  Arguments are validated as in
 * rosko_spmm; nothing is written to C.  In ROSKO_SCHED_LEARNED mode without
 * a cached choice the selector's feature kernels run (and synchronise), in
 * ROSKO_SCHED_AUTOTUNE mode without a cached choice the autotuner runs (and
 * writes C); both cache their choice on the handle as rosko_spmm does.
 */
rosko_status rosko_spmm_plan(rosko_packed_t A, const void* B_dev, rosko_dtype b_dtype, int64_t N,
                             int64_t ldb, const float* col_scale_dev, void* C_dev,
                             rosko_dtype c_dtype, int64_t ldc, int accumulate,
                             const rosko_tile* tile, rosko_plan* out, rosko_stream_t stream);

/*
 * rosko_spmm_batched - C_i = A_i . B_i (or C_i += ...) for `count` <= 64
 * independent problems (pruned layers of different shapes).  The dense-panel
 * tiles of all problems run in one persistent tensor-core launch per CTA-tile
 * shape (at most four: 128 or 256 columns x 128 or 256 rows, each problem
 * taking the shape its tile or the analytic rule gives it), whose work list
 * (per-problem TMA descriptors and sizes) is passed in the kernel
 * parameters; the row-direct sparse remainders share one launch, other
 * remainders run one launch per problem.  Per-problem arrays: A, B (device),
 * N, ldb, C (device), ldc; all problems share b_dtype and c_dtype.  tiles:
 * NULL (analytic rule) or `count` tiles (e.g. from rosko_autotune).  No
 * device memory is allocated
 * and nothing synchronises, so the call can be captured in a CUDA graph and
 * replayed (capture after a first, uncaptured call on the same handles).
 */
rosko_status rosko_spmm_batched(int32_t count, const rosko_packed_t* A, const void* const* B,
                                const int64_t* N, const int64_t* ldb, void* const* C,
                                const int64_t* ldc, rosko_dtype b_dtype, rosko_dtype c_dtype,
                                int accumulate, const rosko_tile* tiles, rosko_stream_t stream);

/*
 * Release a packed handle and its device buffers.  Waits for the handle's
 * device to finish queued work (which may still read the handle), then
 * returns the buffers to the library's memory pool on that device; the pool
 * keeps up to 256 MiB of freed memory mapped for later packs.  NULL-safe.
 */
void rosko_free(rosko_packed_t A);

/*
 * rosko_unpack - inverse of Alg. 1: writes the dense M x K matrix (packed
 * dtype; I8 codes for I8) to A_dev_out with leading dim lda, zeros elsewhere.
 */
rosko_status rosko_unpack(rosko_packed_t A, void* A_dev_out, int64_t lda, rosko_stream_t stream);

/*
 * rosko_packed_info - sizes of a handle (any output pointer may be NULL):
 * nnz, exact bytes of the device format the SpMM reads (nonzero records,
 * column records, panel offsets), number of
 * B rows touched (distinct non-empty columns over all panels), number of
 * panels, panel height m_r, packed dtype.  Synchronous (host data only,
 * except touched_k which is computed at pack time).
 */
rosko_status rosko_packed_info(rosko_packed_t A, int64_t* nnz, int64_t* bytes,
                               int64_t* touched_k, int64_t* n_panels, int32_t* m_r,
                               int32_t* packed_dtype, int64_t* n_cols);

/*
 * rosko_packed_shape - M and K of the packed matrix and the handle's whole
 * device footprint in bytes: every layout the pack builds (column records,
 * row stream and work segments, touched-row gather, dense BF16 tile copies,
 * scales, bookkeeping) in its single device allocation; rosko_packed_info's
 * `bytes` counts only the Rosko column format.  Any pointer may be NULL.
 * Host data only.
 */
rosko_status rosko_packed_shape(rosko_packed_t A, int64_t* M, int64_t* K, int64_t* device_bytes);

/*
 * rosko_packed_export - copy the canonical Alg. 1 arrays to host buffers,
 * concatenated over panels in panel order (synchronous):
 *   A_p_host   nnz values (packed dtype)       loc_m_host  nnz uint8 rows
 *   col_ind_host  n_cols int32                 nnz_host    n_cols int32 counts
 *   panel_cols_host  n_panels + 1 int64 offsets into col_ind / nnz
 * Any pointer may be NULL to skip that array.
 */
rosko_status rosko_packed_export(rosko_packed_t A, void* A_p_host, uint8_t* loc_m_host,
                                 int32_t* col_ind_host, int32_t* nnz_host,
                                 int64_t* panel_cols_host);

/*
 * rosko_pack_save - write a packed handle to a host byte image, so that a
 * pre-packed weight (Sec. 4.1: weights of an inference layer are packed once
 * and stored) can be restored by rosko_pack_load without re-packing.
 * buf_host  destination (host memory), or NULL to query the size only.
 * capacity  bytes available at buf_host (ignored for a size query).
 * bytes     receives the image size (always set on ROSKO_OK).
 * Image: little-endian; a versioned header (magic "ROSKOKP1", format 1), the
 * handle's host bookkeeping, its device allocation byte for byte, and an
 * FNV-1a 64-bit checksum of all of it.  It records the packed dtype, m_r and
 * the dense-copy threshold the pack used.  Synchronous (one device-to-host
 * copy).  Errors: ROSKO_ERR_BAD_HANDLE, ROSKO_ERR_INVALID_ARG (capacity too
 * small), ROSKO_ERR_CUDA.
 */
rosko_status rosko_pack_save(rosko_packed_t A, void* buf_host, int64_t capacity, int64_t* bytes);

/*
 * rosko_pack_load - a new handle on the current device from an image written
 * by rosko_pack_save (any device, any process).  The image is checked before
 * any device work: a wrong magic, a bad checksum, a truncated image or
 * inconsistent sizes give ROSKO_ERR_INVALID_ARG, another format version
 * ROSKO_ERR_UNSUPPORTED; *out is NULL on error.  The restored handle is
 * identical to the saved one (same bytes on the device), so every SpMM gives
 * bit-identical results.  Device memory comes from the library's pool.
 * Synchronises `stream`.
 */
rosko_status rosko_pack_load(const void* buf_host, int64_t bytes, rosko_stream_t stream,
                             rosko_packed_t* out);

/*
 * rosko_schedule_analytic - the closed-form tile rule (host only, no GPU
 * needed): Eq. 1-3 of Sec. 4.2 re-derived for the GB300 register file,
 * shared memory, L2 and 152 SMs.  Fills *tile for an M x K x N problem with
 * nnz nonzeros whose packed panels have height m_r (<= 0: choose), values
 * of type packed_dtype.
 */
rosko_status rosko_schedule_analytic(int64_t M, int64_t K, int64_t N, int64_t nnz,
                                     int32_t m_r, rosko_dtype packed_dtype, rosko_tile* tile);

/*
 * rosko_num_candidates - size of the fixed candidate schedule set searched by
 * the autotuner and predicted by the learned selector (host only).
 */
int32_t rosko_num_candidates(void);

/*
 * rosko_candidate - candidate schedule `index` for handle A and width N, as a
 * ROSKO_SCHED_FORCED tile.  Returns ROSKO_ERR_UNSUPPORTED when the candidate
 * does not apply to this handle (e.g. a dense split on a non-BF16 pack).
 */
rosko_status rosko_candidate(rosko_packed_t A, int64_t N, int32_t index, rosko_tile* out);
/* Index of the candidate with the schedule of `tile` (e.g. the analytic
 * rule's, from rosko_schedule_analytic; tile->m_r = the handle's panel
 * height) for handles of packed_dtype, or -1 if no candidate has it.  Host
 * only.  ROSKO_SCHED_LEARNED keeps the analytic rule unless the network's
 * logit for its pick exceeds this candidate's by ln 2. */
int32_t rosko_candidate_index(const rosko_tile* tile, rosko_dtype packed_dtype);

/*
 * rosko_autotune - per-shape search (Sec. 6: the tile parameters are exposed
 * for auto-tuning).  Times every applicable candidate on (A, B, C) with CUDA
 * events on `stream` (one untimed launch, then `reps` timed launches), writes
 * the fastest to *best and caches it for (A, N): a later rosko_spmm with
 * tile->mode = ROSKO_SCHED_AUTOTUNE uses it.  C is used as scratch output.
 * times_ms (optional, rosko_num_candidates() floats) receives each
 * candidate's mean time in ms, -1 where it does not apply.  Synchronises.
 */
rosko_status rosko_autotune(rosko_packed_t A, const void* B_dev, rosko_dtype b_dtype, int64_t N,
                            int64_t ldb, const float* col_scale_dev, void* C_dev,
                            rosko_dtype c_dtype, int64_t ldc, int32_t reps, rosko_tile* best,
                            float* times_ms, rosko_stream_t stream);

/*
 * rosko_time_tile - mean device time in ms of rosko_spmm(A, B, C) with `tile`
 * (NULL = analytic rule): `reps` launches, each after an L2 flush, captured
 * as one CUDA graph (host launch overhead excluded), minus the flushes.
 * C is overwritten.  Synchronises.
 */
rosko_status rosko_time_tile(rosko_packed_t A, const void* B_dev, rosko_dtype b_dtype, int64_t N,
                             int64_t ldb, const float* col_scale_dev, void* C_dev,
                             rosko_dtype c_dtype, int64_t ldc, const rosko_tile* tile,
                             int32_t reps, float* ms, rosko_stream_t stream);

/*
 * Learned schedule selector.  Features (16, double) of a packed A and a
 * width N: log2 M, log2 K, log2 N, density, log2(1+nnz), log2(1+mean row
 * nnz), row-nnz coefficient of variation, log2(1+max row nnz) - log2(1+mean),
 * fractions of rows in four row-density bins (100 r < K, 20 r < K <= 100 r,
 * 5 r < K <= 20 r, K <= 5 r for row nnz r), mean fraction of non-empty
 * columns per panel, panel-nnz coefficient of variation, log2(1 + nnz per
 * packed column), fraction of empty panels.  Synchronises.  The handle's
 * device must be current (else ROSKO_ERR_INVALID_ARG, nothing launched).
 */
rosko_status rosko_features(rosko_packed_t A, int64_t N, double* features16, rosko_stream_t stream);

/*
 * rosko_features_static - the same 16 features, computed in FP32 on the
 * device, for callers that must not allocate device memory (fixed memory
 * pools, latency-critical serving).  The paper has no counterpart: it is a
 * variant of rosko_features whose scratch is a static device array of this
 * library instead of a per-call cudaMalloc.
 *
 * features16_dev  16 floats of device memory (4-byte aligned), written in
 *         stream order; the caller owns it.
 * Allocates no device memory and does not synchronise.  Limits and races:
 *   - A->M must be <= 1048576 (the static array's rows), else
 *     ROSKO_ERR_INVALID_ARG before anything is enqueued;
 *   - the handle's device must be current (else ROSKO_ERR_INVALID_ARG);
 *   - every call outside a stream capture looks up the array's device
 *     address on the current device (cudaGetSymbolAddress); a call inside a
 *     capture uses the address found by that device's last uncaptured call,
 *     so make one call on each device before capturing (and again after a
 *     cudaDeviceReset, which invalidates the address);
 *   - the features are FP32 arithmetic on exact integer counts: they agree
 *     with rosko_features to FP32 rounding (a relative 1e-5 or better);
 *   - every call shares the one array per device and clears it first, so
 *     calls that can overlap on the GPU (different streams, or several host
 *     threads) race and may return wrong features: serialise them.
 * Errors: ROSKO_ERR_BAD_HANDLE, ROSKO_ERR_INVALID_ARG (NULL or misaligned
 * output, N < 1, M too large), ROSKO_ERR_CUDA (a launch or memset failed).
 */
rosko_status rosko_features_static(rosko_packed_t A, int64_t N, float* features16_dev,
                                   rosko_stream_t stream);

/*
 * The selector network: n_in -> 64 -> 64 -> 64 -> n_out, ReLU on the hidden
 * layers, FP32.  Parameters are one flat device array, per layer the weight
 * matrix [out][in] row-major followed by the bias [out].
 */
int64_t rosko_mlp_param_count(int32_t n_in, int32_t n_out);
/* Workspace (floats) rosko_mlp_loss_grad needs for `batch` samples. */
int64_t rosko_mlp_workspace_floats(int64_t batch, int32_t n_out);
/* logits_dev[batch x n_out] = MLP(X_dev[batch x n_in]); acts_dev holds
 * 3 x batch x 64 floats of hidden activations (device, caller-owned). */
rosko_status rosko_mlp_forward(const float* params_dev, const float* X_dev, int64_t batch,
                               int32_t n_in, int32_t n_out, float* acts_dev, float* logits_dev,
                               rosko_stream_t stream);
/* Mean softmax cross-entropy of the batch against target rows Y_dev
 * [batch x n_out] (one-hot or soft) into *loss_dev, and its gradient with
 * respect to every parameter into grads_dev (same layout as params). */
rosko_status rosko_mlp_loss_grad(const float* params_dev, const float* X_dev, const float* Y_dev,
                                 int64_t batch, int32_t n_in, int32_t n_out, float* grads_dev,
                                 float* loss_dev, float* workspace_dev, rosko_stream_t stream);
/* One Adam step (bias-corrected, step >= 1) on n parameters in place, of
 * the objective L + (weight_decay / 2) |params|^2 (the step uses the
 * gradient grads + weight_decay * params). */
rosko_status rosko_mlp_adam(float* params_dev, const float* grads_dev, float* m_dev, float* v_dev,
                            int64_t n, int32_t step, float lr, float beta1, float beta2,
                            float eps, float weight_decay, rosko_stream_t stream);
/* Install trained selector weights (host array, n_in = 16, n_out =
 * rosko_num_candidates()) with the feature standardisation (mean, std) and
 * the training range [lo, hi] per feature; ROSKO_SCHED_LEARNED then picks the
 * candidate with the largest logit, or the analytic rule for features
 * outside the range. */
rosko_status rosko_selector_set(const float* params_host, int64_t n_params, const double* mean16,
                                const double* std16, const double* lo16, const double* hi16);

/*
 * rosko_device_status - read (and with clear != 0, reset) the current
 * device's kernel error bits: 1 = bounded wait ran out, 2 = corrupt packed
 * stream.  Synchronises the device.
 */
rosko_status rosko_device_status(int32_t* bits, int clear);

/*
 * rosko_set_wait_limit - the time after which every bounded wait of this
 * library's kernels on the current device gives up (sets status bit 1, see
 * rosko_device_status, and lets its kernel return).  ns > 0 sets it, ns = 0
 * restores the default of 2 s; ns < 0 is ROSKO_ERR_INVALID_ARG.  Synchronous;
 * launches already queued read the new value when their waits start.
 */
rosko_status rosko_set_wait_limit(int64_t ns);

/*
 * rosko_probe_bounded_wait - diagnostic launch of the failure-detection
 * path: one CTA waits on an mbarrier that nothing completes, with the same
 * bounded wait every pipelined kernel of the library uses; after the current
 * device's wait limit it sets status bit 1 and returns, leaving the context
 * usable.  Ordered on `stream`, does not synchronise.  With the default limit
 * the launch takes about 2 s: set a short limit first.
 */
rosko_status rosko_probe_bounded_wait(rosko_stream_t stream);

/*
 * rosko_kernel_launches - number of CUDA kernels this library has launched
 * in the calling process since it was loaded (all devices, all streams).
 * Host-only; used to count the library's launches inside a timed region.
 */
int64_t rosko_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* ROSKO_H_ */
