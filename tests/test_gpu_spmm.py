"""Sparse SpMM (Alg. 2 on CUDA cores) against the FP64/int64 oracle.  GPU only.

Bars: INT8 -> INT32 bit-exact; FP32 and BF16-in/FP32-accumulate within 1e-5
of the normalised error max|C - C_ref| / sum_k |a||b| (BF16 against the oracle
on the BF16-rounded inputs; within 1e-2 against the unrounded inputs); FP64
check mode within 1e-13."""
import numpy as np
import pytest
import torch

from tests._lib import built
from oracle.spmm import spmm, spmm_int, normalized_error
from oracle.quant import bf16_round, quantize_rows_int8, quantize_cols_int8
from paper_2307_03930_gb300 import inputs as gen

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "bf16": 1e-5, "f64": 1e-13, "i8f": 1e-5}


def _problem(M, K, N, s, seed, pattern="uniform", relu_b=False):
    rng = gen.rng_for(seed, M, K, N)
    A = gen.sparse_weight(M, K, s, rng, pattern)
    B = gen.relu_normal((K, N), rng) if relu_b else gen.normal((K, N), rng)
    return A, B


def _ldpad(X, elem):
    """Device copy of X with a leading dimension rounded up to 16 bytes."""
    K, N = X.shape
    per = 16 // elem
    ld = max(per, -(-N // per) * per)
    buf = torch.zeros((K, ld), dtype=X.dtype, device="cuda")
    buf[:, :N] = X.cuda()
    return buf[:, :N]


def run(rosko, A, B, mode, m_r=32, tile=None, accumulate=False, C0=None, rows=None):
    """Run the library on (A, B) in `mode` and return (C_gpu[rows], C_ref, D)."""
    M, K = A.shape
    N = B.shape[1]
    if mode == "f32":
        h = rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.F32, m_r=m_r)
        Bd = _ldpad(torch.from_numpy(B), 4)
        C = torch.zeros((M, N), dtype=torch.float32, device="cuda")
        Ar, Br = A, B
    elif mode == "bf16":
        h = rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.BF16, m_r=m_r)
        Bd = _ldpad(torch.from_numpy(B).to(torch.bfloat16), 2)
        C = torch.zeros((M, N), dtype=torch.float32, device="cuda")
        Ar, Br = bf16_round(A), bf16_round(B)
    elif mode == "f64":
        h = rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.F64, m_r=m_r)
        Bd = _ldpad(torch.from_numpy(B), 4)
        C = torch.zeros((M, N), dtype=torch.float64, device="cuda")
        Ar, Br = A, B
    elif mode in ("i8", "i8f"):
        qa, sa = quantize_rows_int8(A)
        qb, sb = quantize_cols_int8(B)
        h = rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.I8, m_r=m_r)
        Bd = _ldpad(torch.from_numpy(qb), 1)
        C = torch.zeros((M, N), dtype=torch.int32 if mode == "i8" else torch.float32,
                        device="cuda")
    if C0 is not None:
        C.copy_(torch.from_numpy(C0).to(C.dtype))
    else:
        # C = A.B overwrites C: an element no kernel writes fails the check
        C.fill_(2**31 - 1 if C.dtype == torch.int32 else float("nan"))
    col_scale = torch.from_numpy(sb).cuda() if mode == "i8f" else None
    rosko.rosko_spmm(h, Bd, C, col_scale=col_scale, accumulate=accumulate, tile=tile)
    torch.cuda.synchronize()
    assert rosko.rosko_device_status(clear=True) == 0
    Cg = C.cpu().numpy()
    rows = np.arange(M) if rows is None else np.asarray(rows)
    Cg = Cg[rows]
    if mode == "i8":
        ref = spmm_int(qa, qb, rows=rows, C0=C0.astype(np.int64) if C0 is not None else None)
        return Cg, ref, None
    if mode == "i8f":
        ci = spmm_int(qa, qb, rows=rows).astype(np.float64)
        ref = ci * sa[rows, None].astype(np.float64) * sb[None, :].astype(np.float64)
        D = np.abs(qa[rows]).astype(np.float64) @ np.abs(qb).astype(np.float64)
        D = D * sa[rows, None] * sb[None, :]
        if C0 is not None:
            ref = ref + C0[rows]
            D = D + np.abs(C0[rows])
        return Cg, ref, D
    ref, D = spmm(Ar, Br, rows=rows, C0=C0)
    if C0 is not None:
        D = D + np.abs(C0[rows].astype(np.float64))
    return Cg, ref, D


def check(mode, Cg, ref, D):
    if mode == "i8":
        assert np.array_equal(Cg.astype(np.int64), ref)
        return 0.0
    err = normalized_error(Cg, ref, D)
    assert err <= TOL[mode], err
    return err


SHAPES = [(1, 1, 1, 0.0), (33, 17, 65, 0.5), (70, 300, 129, 0.9), (200, 1000, 300, 0.99),
          (64, 96, 40, 1.0), (130, 77, 257, 0.0)]


@pytest.mark.parametrize("mode", ["f32", "bf16", "i8", "i8f", "f64"])
@pytest.mark.parametrize("M,K,N,s", SHAPES)
@pytest.mark.parametrize("m_r", [0, 32])
def test_small_ragged(mode, M, K, N, s, m_r):
    # m_r = 0: the library's density-based panel height (8 or 16)
    rosko = built()
    A, B = _problem(M, K, N, s, seed=0)
    if mode == "f64" and m_r == 32:
        m_r = 16
    check(mode, *run(rosko, A, B, mode, m_r=m_r))


# every compiled (order, m_r, V) variant with several CTA heights, slabs and K
# splits; order 1 = column order (Alg. 2), order 2 = row-slot order,
# order 3 = row-slot over the tile's touched rows, order 4 = row-direct (B
# from L2, no slabs: k_c and the split do not apply)
VARIANTS = {"f32": [(1, 32, 4), (1, 16, 8), (1, 16, 4), (1, 8, 16), (1, 8, 8), (2, 16, 4),
                    (2, 8, 8), (3, 16, 4), (4, 16, 4), (4, 8, 8), (4, 32, 4)],
            "bf16": [(1, 32, 4), (1, 16, 8), (1, 8, 16), (1, 8, 8), (2, 16, 4), (2, 8, 8),
                     (3, 16, 4), (4, 16, 8), (4, 8, 4), (4, 32, 8)],
            "i8": [(1, 32, 4), (1, 16, 8), (1, 8, 16), (2, 16, 4), (2, 8, 8), (3, 16, 4),
                   (4, 16, 8)],
            "i8f": [(1, 32, 4), (1, 16, 8), (1, 8, 16), (2, 16, 4), (2, 8, 8), (3, 16, 4),
                    (4, 8, 8)],
            "f64": [(1, 32, 2), (1, 16, 4), (1, 8, 8), (2, 16, 2), (2, 8, 4), (3, 16, 2),
                    (4, 16, 4)]}


@pytest.mark.parametrize("mode", list(VARIANTS))
@pytest.mark.parametrize("W,KC,split", [(1, 8, 1), (3, 32, 3), (8, 64, 2), (4, 256, 1)])
def test_forced_tiles(mode, W, KC, split):
    rosko = built()
    A, B = _problem(150, 700, 300, 0.8, seed=1)
    esz = {"f32": 4, "bf16": 2, "i8": 1, "i8f": 1, "f64": 4}[mode]
    for order, R, V in VARIANTS[mode]:
        m_c = 128 if order == 3 else W * R   # order 3: one CTA per 128-row tile
        t = rosko.make_tile(m_r=R, n_r=32 * V, k_c=KC, m_c=m_c, split_k=split, order=order,
                            mode=rosko.SCHED_FORCED)
        if order != 4 and 2 * KC * 32 * V * esz > 200 * 1024:
            # a two-slab ring would not fit in shared memory: rejected on the host
            with pytest.raises(rosko.RoskoError) as ei:
                run(rosko, A, B, mode, m_r=R, tile=t)
            assert ei.value.status == 1
            continue
        check(mode, *run(rosko, A, B, mode, m_r=R, tile=t))


@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("s", [0.0, 0.99, 0.999])
def test_orders_agree_bitwise_int8(order, s):
    # integer accumulation is exact: both traversals give the same INT32 C
    rosko = built()
    A, B = _problem(96, 333, 150, s, seed=21)
    t = rosko.make_tile(order=order)
    check("i8", *run(rosko, A, B, "i8", m_r=16, tile=t))


@pytest.mark.parametrize("mode", ["f32", "bf16", "i8", "i8f", "f64"])
@pytest.mark.parametrize("split", [1, 4])
def test_accumulate_in_place(mode, split):
    # Alg. 2 loads C first: C += A.B
    rosko = built()
    A, B = _problem(90, 500, 200, 0.9, seed=2)
    rng = np.random.default_rng(5)
    if mode == "i8":
        C0 = rng.integers(-1000, 1000, size=(90, 200)).astype(np.int32)
    else:
        C0 = rng.standard_normal((90, 200)).astype(np.float64 if mode == "f64" else np.float32)
    for order, m_r in ((1, 16 if mode == "f64" else 32), (2, 16), (3, 16), (4, 16)):
        t = rosko.make_tile(split_k=split, order=order)
        check(mode, *run(rosko, A, B, mode, m_r=m_r, tile=t, accumulate=True, C0=C0))


def test_identity_and_zero():
    rosko = built()
    rng = np.random.default_rng(0)
    B = rng.standard_normal((64, 100)).astype(np.float32)
    Cg, ref, D = run(rosko, np.eye(64, dtype=np.float32), B, "f32")
    assert np.array_equal(Cg, B)
    Cg, ref, D = run(rosko, np.zeros((64, 64), np.float32), B, "f32")
    assert np.all(Cg == 0)
    Bb = bf16_round(B)
    Cg, _, _ = run(rosko, np.eye(64, dtype=np.float32), Bb, "bf16")
    assert np.array_equal(Cg, Bb)


def test_bf16_against_unrounded_inputs():
    rosko = built()
    A, B = _problem(256, 2048, 512, 0.9, seed=3, pattern="magnitude", relu_b=True)
    Cg, ref, D = run(rosko, A, B, "bf16")
    assert normalized_error(Cg, ref, D) <= 1e-5
    ref_u, D_u = spmm(A, B)
    assert normalized_error(Cg, ref_u, D_u) <= 1e-2


def test_c1_full_size_fp32():
    # 1024 x 1024 at 90% uniform sparsity times a 1024 x 1024 N(0,1) B, seed 0
    rosko = built()
    rng = gen.rng_for(0)
    A = gen.sparse_weight(1024, 1024, 0.9, rng, "uniform")
    B = gen.normal((1024, 1024), rng)
    check("f32", *run(rosko, A, B, "f32"))


@pytest.mark.parametrize("s", [0.5, 0.7, 0.9, 0.95, 0.99, 0.998])
@pytest.mark.parametrize("mode", ["f32", "bf16"])
def test_c2_full_size_sampled(s, mode):
    # conv-layer shape: A 512 x 4608 magnitude-pruned, B 4608 x 3136 post-ReLU,
    # seed 1; the analytic schedule the bench uses; 48 sampled rows vs oracle
    rosko = built()
    rng = gen.rng_for(1, int(round(s * 1000)))
    A = gen.magnitude_prune(gen.normal((512, 4608), rng), s)
    B = gen.relu_normal((4608, 3136), rng)
    rows = np.random.default_rng(int(s * 1000)).choice(512, 48, replace=False)
    check(mode, *run(rosko, A, B, mode, rows=rows))


@pytest.mark.parametrize("mode", ["f32", "bf16", "i8"])
@pytest.mark.parametrize("order", [3, 4])
def test_gather_empty_tiles_and_ragged(mode, order):
    # tiles whose rows are all zero have an empty touched-column list; the
    # last tile is ragged (M = 300); N = 130 leaves a partial lane chunk
    rosko = built()
    A, B = _problem(300, 777, 130, 0.995, seed=31)
    A[0:128] = 0                       # tile 0: nothing touched
    A[256:300, :5] = 1.0               # ragged tile 2: a few dense columns
    t = rosko.make_tile(order=order)
    check(mode, *run(rosko, A, B, mode, m_r=16, tile=t))


@pytest.mark.parametrize("M,K", [(11008, 4096), (4096, 11008)])
@pytest.mark.parametrize("s", [0.7, 0.9, 0.95])
def test_c3_full_size_sampled(M, K, s):
    # transformer-FFN shapes, seed 2: A magnitude-pruned N(0,1), B K x 2048
    # N(0,1); BF16 in / FP32 accumulate (analytic schedule: the tensor-core
    # path) and INT8 -> INT32 (row-direct), 40 sampled rows against the oracle
    rosko = built()
    rng = gen.rng_for(2, M, int(round(s * 100)))
    A = gen.magnitude_prune(gen.normal((M, K), rng), s)
    B = gen.normal((K, 2048), rng)
    rows = np.random.default_rng(M + int(s * 100)).choice(M, 40, replace=False)
    check("bf16", *run(rosko, A, B, "bf16", m_r=0, rows=rows))
    check("i8", *run(rosko, A, B, "i8", m_r=0, rows=rows))


@pytest.mark.parametrize("mode", ["f32", "bf16", "i8", "i8f", "f64"])
@pytest.mark.parametrize("accumulate", [False, True])
def test_row_direct_cuts_long_rows(mode, accumulate):
    # power-law rows plus two full rows: rows longer than one work segment
    # (64 nonzeros) are cut into pieces whose sums are added into C
    rosko = built()
    M, K, N = 150, 700, 300
    A = gen.sparse_weight(M, K, 0.97, gen.rng_for(61), "powerlaw")
    rng = np.random.default_rng(62)
    A[3] = rng.standard_normal(K).astype(np.float32)
    A[149, :300] = rng.standard_normal(300).astype(np.float32)
    B = gen.normal((K, N), gen.rng_for(63))
    C0 = None
    if accumulate:
        C0 = (rng.integers(-1000, 1000, size=(M, N)).astype(np.int32) if mode == "i8" else
              rng.standard_normal((M, N)).astype(np.float64 if mode == "f64" else np.float32))
    t = rosko.make_tile(order=4, dense_split_pm=1001)
    check(mode, *run(rosko, A, B, mode, m_r=16, tile=t, accumulate=accumulate, C0=C0))


@pytest.mark.parametrize("mode", ["f32", "bf16", "i8"])
def test_k_beyond_the_row_stream(mode):
    # K >= 65280 does not fit the 16-bit k of the row stream: the pack builds
    # no row stream and the library runs Alg. 2's column order (and, for
    # BF16, the tensor-core path for dense-enough tiles)
    rosko = built()
    A, B = _problem(40, 70000, 33, 0.999, seed=95)
    A[5, 65000:65100] = 1.5          # nonzeros past k = 65535
    check(mode, *run(rosko, A, B, mode, m_r=0))
    # forcing a row-stream traversal is refused, not silently wrong
    t = rosko.make_tile(order=4, dense_split_pm=1001)
    with pytest.raises(rosko.RoskoError):
        run(rosko, A, B, mode, m_r=0, tile=t)
