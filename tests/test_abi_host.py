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
