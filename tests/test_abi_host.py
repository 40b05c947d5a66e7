"""The C-ABI library loads without a GPU, exports every declared symbol and
rejects bad arguments on the host before touching CUDA."""
import ctypes
import os
import re

import pytest

from tests._lib import built, ROOT


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "rosko.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(rosko_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    rosko = built()
    names = _declared_functions()
    assert "rosko_pack" in names and "rosko_spmm" in names and "rosko_free" in names
    raw = ctypes.CDLL(rosko.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_status_strings():
    rosko = built()
    for code, name in enumerate(rosko.STATUS_NAMES):
        assert rosko.rosko_status_string(code) == name
    assert rosko.rosko_status_string(99) == "ROSKO_ERR_UNKNOWN"


def test_host_argument_validation():
    rosko = built()
    L = rosko.lib()
    out = ctypes.c_void_p()
    t = rosko.make_tile()
    nul = None
    # NULL output pointer
    assert L.rosko_pack(nul, rosko.F32, 4, 4, 4, rosko.F32, nul, ctypes.byref(t), nul, nul) == 1
    # negative sizes, short leading dimension, NULL A with nonzero size
    assert L.rosko_pack(nul, rosko.F32, -1, 4, 4, rosko.F32, nul, nul, nul, ctypes.byref(out)) == 1
    assert L.rosko_pack(ctypes.c_void_p(16), rosko.F32, 4, 8, 4, rosko.F32, nul, nul, nul,
                        ctypes.byref(out)) == 1
    assert L.rosko_pack(nul, rosko.F32, 4, 4, 4, rosko.F32, nul, nul, nul, ctypes.byref(out)) == 1
    # unsupported conversion, bad dtype code, bad panel height
    assert L.rosko_pack(ctypes.c_void_p(16), rosko.F64, 4, 4, 4, rosko.BF16, nul, nul, nul,
                        ctypes.byref(out)) == 2
    assert L.rosko_pack(ctypes.c_void_p(16), 9, 4, 4, 4, rosko.F32, nul, nul, nul,
                        ctypes.byref(out)) == 1
    bad = rosko.make_tile(m_r=12)
    assert L.rosko_pack(ctypes.c_void_p(16), rosko.F32, 4, 4, 4, rosko.F32, nul,
                        ctypes.byref(bad), nul, ctypes.byref(out)) == 1
    assert out.value is None
    # bad handles
    assert L.rosko_spmm(nul, nul, rosko.F32, 4, 4, nul, nul, rosko.F32, 4, 0, nul, nul) == 6
    fake = (ctypes.c_uint64 * 64)()
    assert L.rosko_spmm(ctypes.cast(fake, ctypes.c_void_p), nul, rosko.F32, 4, 4, nul, nul,
                        rosko.F32, 4, 0, nul, nul) == 6
    assert L.rosko_unpack(nul, nul, 4, nul) == 6
    assert L.rosko_packed_info(nul, nul, nul, nul, nul, nul, nul, nul) == 6
    assert L.rosko_packed_export(nul, nul, nul, nul, nul, nul) == 6
    L.rosko_free(nul)                       # NULL-safe
    L.rosko_free(ctypes.cast(fake, ctypes.c_void_p))   # foreign pointer ignored
    assert L.rosko_device_status(nul, 0) == 1


@pytest.mark.parametrize("M,K,N,s,dt", [(1024, 1024, 1024, 0.9, 0), (512, 4608, 3136, 0.99, 1),
                                        (11008, 4096, 2048, 0.7, 2), (7, 5, 3, 0.5, 0),
                                        (512, 4608, 3136, 0.998, 0)])
def test_analytic_schedule_fits_gb300(M, K, N, s, dt):
    rosko = built()
    nnz = int(M * K * (1 - s))
    t = rosko.rosko_schedule_analytic(M, K, N, nnz, 0, dt)
    assert t["m_r"] in (8, 16, 32)
    V = t["n_r"] // 32
    assert t["n_r"] % 32 == 0
    # register level: m_r x V accumulators per lane within the 128-register
    # budget for the slab traversals; row-direct (order 4) holds one row of V
    # columns per warp, at most two 16-byte chunks per lane
    rows = 1 if t["order"] == 4 else t["m_r"]
    acc_words = rows * V * (2 if dt == 3 else 1)
    assert acc_words <= 128
    if t["order"] == 4:
        esz = {0: 4, 1: 2, 2: 1, 3: 4}[dt]
        assert V * esz <= 32
    # shared-memory level: the 4-stage B ring leaves room for two CTAs per SM
    esz = {0: 4, 1: 2, 2: 1, 3: 4}[dt]
    assert 1024 + 4 * t["k_c"] * t["n_r"] * esz <= 114 * 1024
    assert t["m_c"] % t["m_r"] == 0 and 1 <= t["m_c"] // t["m_r"] <= 8
    assert 1 <= t["split_k"] <= max(1, (K + t["k_c"] - 1) // t["k_c"] // 8)
    P = -(-M // t["m_r"])
    ctas = -(-P // (t["m_c"] // t["m_r"])) * -(-N // t["n_r"]) * t["split_k"]
    assert ctas >= min(152, -(-P // (t["m_c"] // t["m_r"])) * -(-N // t["n_r"]))


def test_tensor_core_tile_rules():
    # host-only: the analytic schedule's tensor-core tile (GB300, 152 SMs)
    rosko = built()

    def sched(M, K, N, s, dt):
        return rosko.rosko_schedule_analytic(M, K, N, int(M * K * (1 - s)), 0, dt)

    # enough K work per CTA (>= 20 double slabs): 256-row tiles, stream-K
    # over every SM
    t = sched(1024, 4096, 4096, 0.9, rosko.BF16)
    assert (t["dense_m_c"], t["dense_n_r"], t["dense_split_k"]) == (256, 256, 152)
    t = sched(11008, 4096, 2048, 0.7, rosko.BF16)
    assert t["dense_m_c"] == 256
    # INT8 codes drain the accumulator every 1,024 K: 128 rows, so that the
    # second TMEM set overlaps the drains
    t = sched(11008, 4096, 2048, 0.7, rosko.I8)
    assert t["dense_m_c"] == 128
    # 512x4608x3136: 12 double slabs per CTA -> 128-row tiles; its 52 tiles
    # are far from filling the GPU -> split along K over every SM
    t = sched(512, 4608, 3136, 0.9, rosko.BF16)
    assert (t["dense_m_c"], t["dense_n_r"], t["dense_split_k"]) == (128, 256, 152)
    # 2048^3: 128 tiles nearly fill the GPU -> one whole tile per CTA
    t = sched(2048, 2048, 2048, 0.9, rosko.BF16)
    assert (t["dense_m_c"], t["dense_split_k"]) == (128, 128)
    # K < 1024 (fewer than 16 slabs): whole 128-wide tiles, one per CTA up
    # to two per SM
    t = sched(1024, 512, 4096, 0.9, rosko.BF16)
    assert (t["dense_n_r"], t["dense_m_c"], t["dense_split_k"]) == (128, 128, 8 * 32)


def test_split_rule_follows_the_two_time_models():
    # 512x4608x3136: row-direct predicted faster at 99 % (the layer stays
    # sparse), the tensor cores at 90 % (tiles of >= 15 per mille go dense)
    rosko = built()
    t = rosko.rosko_schedule_analytic(512, 4608, 3136, int(512 * 4608 * 0.01), 0, rosko.BF16)
    assert t["dense_split_pm"] == 1001 and t["order"] == 4
    t = rosko.rosko_schedule_analytic(512, 4608, 3136, int(512 * 4608 * 0.1), 0, rosko.BF16)
    assert t["dense_split_pm"] == 15
    # FP32 packs have no tensor-core path
    t = rosko.rosko_schedule_analytic(512, 4608, 3136, int(512 * 4608 * 0.1), 0, rosko.F32)
    assert t["dense_split_pm"] == 1001
