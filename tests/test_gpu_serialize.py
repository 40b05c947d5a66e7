"""Serialisation of packed handles (pre-packed inference weights, Sec. 4.1):
rosko_pack_save / rosko_pack_load round trips restore the same device bytes,
so INT8 results are reproduced bit for bit and FP results up to the rounding
order of atomic partial sums, and damaged or foreign images are refused
before any device work."""
import ctypes
import struct

import numpy as np
import pytest
import torch

from tests._lib import built
from oracle.spmm import spmm, spmm_int, normalized_error
from oracle.quant import bf16_round, quantize_rows_int8, quantize_cols_int8
from paper_2307_03930_gb300 import inputs as gen


def _fnv1a(b: bytes) -> int:
    h = 1469598103934665603
    for x in b:
        h = ((h ^ x) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def test_load_refuses_garbage_on_host():
    rosko = built()
    L = rosko.lib()
    out = ctypes.c_void_p(123)
    for blob in (b"", b"x" * 7, b"ROSKOKP1" + b"\0" * 400, bytes(range(256)) * 4):
        buf = ctypes.create_string_buffer(blob, max(len(blob), 1))
        st = L.rosko_pack_load(buf if blob else None, len(blob), None, ctypes.byref(out))
        assert rosko.STATUS_NAMES[st] == "ROSKO_ERR_INVALID_ARG"
        assert out.value is None
    assert rosko.STATUS_NAMES[L.rosko_pack_save(None, None, 0, None)] == "ROSKO_ERR_BAD_HANDLE"


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["int8", "bf16_dense", "fp32", "bf16_powerlaw_m32"])
def test_round_trip_restores_the_handle(kind):
    rosko = built()
    M, K, N = 700, 1500, 300
    pat = "powerlaw" if "powerlaw" in kind else "uniform"
    A = gen.sparse_weight(M, K, 0.9 if kind != "bf16_dense" else 0.6, gen.rng_for(91, M), pat)
    B = gen.relu_normal((K, N), gen.rng_for(92, K))
    Ad = torch.from_numpy(A).cuda()
    m_r = 32 if "m32" in kind else 0
    if kind == "int8":
        h = rosko.rosko_pack(Ad, rosko.I8, m_r=m_r)
        qb, _ = quantize_cols_int8(B)
        Bd = torch.zeros((K, 304), dtype=torch.int8, device="cuda")
        Bd[:, :N] = torch.from_numpy(qb).cuda()
        Bd = Bd[:, :N]
        mk = lambda: torch.empty((M, N), dtype=torch.int32, device="cuda")
    elif kind == "fp32":
        h = rosko.rosko_pack(Ad, rosko.F32, m_r=m_r)
        Bd = torch.from_numpy(B).cuda()
        mk = lambda: torch.empty((M, N), device="cuda")
    else:
        h = rosko.rosko_pack(Ad, rosko.BF16, m_r=m_r)
        Bd = torch.zeros((K, 304), dtype=torch.bfloat16, device="cuda")
        Bd[:, :N] = torch.from_numpy(B).cuda().to(torch.bfloat16)
        Bd = Bd[:, :N]
        mk = lambda: torch.empty((M, N), device="cuda")
    img = rosko.rosko_pack_save(h)
    assert img[:8] == b"ROSKOKP1"
    info = h.info()
    assert info["device_bytes"] >= info["bytes"] > 0
    h2 = rosko.rosko_pack_load(img)
    info2 = h2.info()
    assert info2 == info
    assert rosko.rosko_pack_save(h2) == img           # the same bytes again
    tiles = [None, rosko.make_tile(order=4, dense_split_pm=1001)]
    if kind.startswith("bf16"):
        tiles.append(rosko.make_tile(dense_split_pm=1))
    if kind == "int8":
        qa, _ = quantize_rows_int8(A)
        want = spmm_int(qa, quantize_cols_int8(B)[0])
    else:
        Ar, Br = (A, B) if kind == "fp32" else (bf16_round(A), bf16_round(B))
        ref, D = spmm(Ar, Br)
    for t in tiles:
        C1, C2 = mk(), mk()
        rosko.rosko_spmm(h, Bd, C1, tile=t)
        rosko.rosko_spmm(h2, Bd, C2, tile=t)
        torch.cuda.synchronize()
        if kind == "int8":
            assert torch.equal(C1, C2)          # integer sums: bit for bit
            assert np.array_equal(C2.cpu().numpy().astype(np.int64), want)
        else:
            c1, c2 = C1.cpu().numpy(), C2.cpu().numpy()
            # both handles give oracle results; between them only the rounding
            # order of atomic partial sums (stream-K tile pieces, cut rows)
            # may differ
            assert normalized_error(c1, ref, D) <= 1e-5
            assert normalized_error(c2, ref, D) <= 1e-5
            assert normalized_error(c2, c1.astype(np.float64), D) <= 2e-6
    # unpack of the restored handle reproduces the packed matrix
    dt = {"int8": torch.int8, "fp32": torch.float32}.get(kind, torch.bfloat16)
    U1 = torch.zeros((M, K), dtype=dt, device="cuda")
    U2 = torch.zeros_like(U1)
    rosko.rosko_unpack(h, U1)
    rosko.rosko_unpack(h2, U2)
    assert torch.equal(U1.view(torch.uint8), U2.view(torch.uint8))


@pytest.mark.gpu
def test_damaged_and_foreign_images_are_refused():
    rosko = built()
    A = gen.sparse_weight(200, 300, 0.9, gen.rng_for(93, 1), "uniform")
    h = rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.BF16)
    img = bytearray(rosko.rosko_pack_save(h))
    flipped = bytearray(img)
    flipped[len(img) // 2] ^= 0x40                    # a bit in the device blob
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        rosko.rosko_pack_load(bytes(flipped))
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        rosko.rosko_pack_load(bytes(img[:-9]))        # truncated
    # another format version, with a valid checksum: unsupported, not corrupt
    other = bytearray(img)
    struct.pack_into("<I", other, 8, 2)
    struct.pack_into("<Q", other, len(other) - 8, _fnv1a(bytes(other[:-8])))
    with pytest.raises(RuntimeError, match="UNSUPPORTED"):
        rosko.rosko_pack_load(bytes(other))
    # the intact image still loads
    h2 = rosko.rosko_pack_load(bytes(img))
    assert h2.info() == h.info()
