"""Device packer (Alg. 1) against the oracle's packer: byte-exact arrays,
unpack round trip and handle sizes.  GPU only."""
import numpy as np
import pytest
import torch

from tests._lib import built
from paper_2307_03930_gb300 import inputs as gen
from oracle.pack import pack_panels
from oracle.quant import bf16_bits, bf16_round, quantize_rows_int8

pytestmark = pytest.mark.gpu


def _matrix(M, K, s, seed, special=False):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, K)).astype(np.float32)
    A[rng.random((M, K)) < s] = 0
    if special and M * K >= 4:
        A.flat[0] = -0.0
        A.flat[1] = np.inf
        A.flat[2] = -np.inf
        A.flat[3] = np.nan
    return A


def _expected(A, a_dt, p_dt, m_r):
    """Oracle view of what the device should pack: (packed values as raw
    comparable array, PackedPanels)."""
    if p_dt == "f32":
        pk = pack_panels(A, m_r)
        return pk.A_p.view(np.uint32), pk
    if p_dt == "f64":
        pk = pack_panels(A, m_r)
        return pk.A_p.astype(np.float64).view(np.uint64), pk
    if p_dt == "bf16":
        src = bf16_round(A) if a_dt == "bf16" else A
        pk = pack_panels(src, m_r)
        return bf16_bits(pk.A_p), pk
    if p_dt == "i8":
        q = A if a_dt == "i8" else quantize_rows_int8(A)[0]
        pk = pack_panels(q, m_r)
        return pk.A_p, pk
    raise ValueError(p_dt)


CODES = {"f32": 0, "bf16": 1, "i8": 2, "f64": 3}
PAIRS = [("f32", "f32"), ("f32", "bf16"), ("f32", "i8"), ("f32", "f64"), ("bf16", "bf16"),
         ("i8", "i8")]


@pytest.mark.parametrize("a_dt,p_dt", PAIRS)
@pytest.mark.parametrize("M,K,s,m_r", [(1, 1, 0.0, 8), (37, 53, 0.5, 8), (70, 300, 0.9, 32),
                                       (200, 129, 0.99, 16), (64, 64, 1.0, 32),
                                       (33, 1000, 0.0, 32)])
def test_pack_matches_oracle(a_dt, p_dt, M, K, s, m_r):
    rosko = built()
    special = a_dt == "f32" and p_dt in ("f32", "f64", "bf16")
    A = _matrix(M, K, s, seed=M * 7 + K, special=special)
    if a_dt == "bf16":
        At = torch.from_numpy(A).to(torch.bfloat16).cuda()
    elif a_dt == "i8":
        Ai = np.clip(np.rint(A * 40), -127, 127).astype(np.int8)
        A = Ai
        At = torch.from_numpy(Ai).cuda()
    else:
        At = torch.from_numpy(A).cuda()
    h = rosko.rosko_pack(At, CODES[p_dt], m_r=m_r)
    got = rosko.rosko_packed_export(h)
    want_vals, pk = _expected(A, a_dt, p_dt, m_r)
    raw = got["A_p"].view({"f32": np.uint32, "f64": np.uint64, "bf16": np.uint16,
                           "i8": np.int8}[p_dt])
    if p_dt == "bf16":
        # NaN has many encodings: the positions must agree, the payload is free
        nan_got = (raw & 0x7FFF) > 0x7F80
        nan_want = (want_vals & 0x7FFF) > 0x7F80
        assert np.array_equal(nan_got, nan_want)
        raw, want_vals = raw[~nan_got], want_vals[~nan_want]
    assert np.array_equal(raw, want_vals)
    assert np.array_equal(got["loc_m"].astype(np.int64), pk.loc_m)
    assert np.array_equal(got["col_ind"].astype(np.int64), pk.col_ind)
    assert np.array_equal(got["nnz"].astype(np.int64), pk.nnz)
    assert np.array_equal(got["panel_cols"], pk.panel_cols)
    info = h.info()
    assert info["nnz"] == pk.A_p.size and info["n_cols"] == pk.col_ind.size
    assert info["n_panels"] == (M + m_r - 1) // m_r and info["m_r"] == m_r
    src = A if p_dt != "i8" or a_dt == "i8" else quantize_rows_int8(A)[0]
    assert info["touched_k"] == int(np.count_nonzero((src != 0).any(axis=0)))
    # unpack round trip (inverse of Alg. 1) in the packed dtype
    out = torch.full((M, K), 7, dtype={"f32": torch.float32, "f64": torch.float64,
                                        "bf16": torch.bfloat16, "i8": torch.int8}[p_dt],
                     device="cuda")
    rosko.rosko_unpack(h, out)
    torch.cuda.synchronize()
    back = out.cpu()
    if p_dt == "bf16":
        ref = bf16_bits(np.where(A != 0, A, 0).astype(np.float32) if a_dt == "f32" else bf16_round(A))
        ref = np.where(A != 0, ref, 0)
        gb = back.view(torch.int16).numpy().view(np.uint16)
        ref = ref.astype(np.uint16)
        nan = (ref & 0x7FFF) > 0x7F80
        assert np.array_equal((gb & 0x7FFF) > 0x7F80, nan)
        assert np.array_equal(gb[~nan], ref[~nan])
    elif p_dt == "i8":
        assert np.array_equal(back.numpy(), src)
    else:
        exp = np.where(A != 0, A, 0).astype(back.numpy().dtype)
        assert np.array_equal(back.numpy().view(np.uint8), exp.view(np.uint8))


def test_pack_empty_shapes():
    rosko = built()
    for M, K in [(0, 5), (5, 0), (0, 0)]:
        A = torch.zeros((M, K), dtype=torch.float32, device="cuda")
        h = rosko.rosko_pack(A, 0)
        info = h.info()
        assert info["nnz"] == 0 and info["n_cols"] == 0 and info["touched_k"] == 0


def test_alloc_failure_is_reported(monkeypatch):
    # host-side fault injection: each of the packer's three device
    # allocations (pass-1 scratch, the handle, the segment-head scratch)
    # fails in turn and is reported as ROSKO_ERR_OOM; there is no fourth
    rosko = built()
    A = torch.randn(40, 40, device="cuda")
    for n in ("1", "2", "3"):
        monkeypatch.setenv("ROSKO_FAIL_ALLOC", n)
        with pytest.raises(rosko.RoskoError) as ei:
            rosko.rosko_pack(A, 0)
        assert ei.value.status == 3
    for dt in (rosko.F32, rosko.BF16):
        monkeypatch.setenv("ROSKO_FAIL_ALLOC", "4" if dt == rosko.F32 else "5")
        h = rosko.rosko_pack(A, dt)
        assert h.info()["nnz"] == int((A != 0).sum())
    monkeypatch.delenv("ROSKO_FAIL_ALLOC")
    h = rosko.rosko_pack(A, 0)
    assert h.info()["nnz"] == int((A != 0).sum())


@pytest.mark.parametrize("dt", ["f32", "bf16", "i8"])
@pytest.mark.parametrize("M,K", [(300, 177), (1, 64), (129, 1)])
def test_pack_transposed_is_the_pack_of_the_transpose(dt, M, K):
    # the backward SpMM of a pruned layer uses W^T: packing A transposed
    # equals packing the transpose (byte-exact export), and the SpMM with it
    # matches the oracle on A^T
    rosko = built()
    from tests.test_gpu_spmm import run, check
    A = gen.sparse_weight(M, K, 0.8, gen.rng_for(91, M, K), "uniform")
    code = {"f32": rosko.F32, "bf16": rosko.BF16, "i8": rosko.I8}[dt]
    h1 = rosko.rosko_pack_transposed(torch.from_numpy(A).cuda(), code)
    h2 = rosko.rosko_pack(torch.from_numpy(np.ascontiguousarray(A.T)).cuda(), code)
    e1, e2 = rosko.rosko_packed_export(h1), rosko.rosko_packed_export(h2)
    for k in e2:
        assert np.array_equal(np.asarray(e1[k]), np.asarray(e2[k])), k
    assert h1.info() == h2.info()
    B = gen.normal((M, 70), gen.rng_for(92, M))
    check(dt, *run(rosko, np.ascontiguousarray(A.T), B, dt, m_r=0))


@pytest.mark.parametrize("a_dt,p_dt", PAIRS)
def test_pack_launch_count(a_dt, p_dt):
    # the independent passes of each phase share one launch: counting (panel
    # columns, rows, tile columns), the three launches of the fused scans,
    # the size summary, then writing (column records, row and gather streams,
    # union lists, dense copies, terminating entries), then the work
    # segments' inline records; INT8 adds its row scales (quantisation from
    # FP32, or the all-ones default)
    rosko = built()
    A = _matrix(300, 500, 0.9, seed=5)
    if a_dt == "bf16":
        At = torch.from_numpy(A).to(torch.bfloat16).cuda()
    elif a_dt == "i8":
        At = torch.from_numpy(np.clip(np.rint(A * 40), -127, 127).astype(np.int8)).cuda()
    else:
        At = torch.from_numpy(A).cuda()
    torch.cuda.synchronize()
    l0 = rosko.rosko_kernel_launches()
    h = rosko.rosko_pack(At, CODES[p_dt])
    assert rosko.rosko_kernel_launches() - l0 == 7 + (p_dt == "i8")
    nnz = int((At != 0).sum())
    # quantisation from FP32 also drops the values whose code rounds to 0
    assert h.info()["nnz"] == nnz if a_dt == p_dt or p_dt != "i8" else h.info()["nnz"] <= nnz
