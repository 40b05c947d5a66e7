"""rosko_features_static: the allocation-free variant of rosko_features
(scratch in a static device array).  Collected last so that it also runs
after every other test has used the library."""
import ctypes

import numpy as np
import pytest
import torch

from tests._lib import built
from paper_2307_03930_gb300 import inputs as gen


def test_static_features_rejects_bad_handle_on_host():
    rosko = built()
    # no handle: refused before any CUDA call (runs without a GPU)
    s = rosko.lib().rosko_features_static(None, 10, ctypes.c_void_p(16), None)
    assert rosko.STATUS_NAMES[s] == "ROSKO_ERR_BAD_HANDLE"


def _handle(rosko, M, K, s, seed, pattern="uniform"):
    A = gen.sparse_weight(M, K, s, gen.rng_for(seed, M, K), pattern)
    A[: min(M, 17)] = 0           # empty rows and an empty panel
    return rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.BF16, m_r=16)


@pytest.mark.gpu
def test_static_features_match_allocating_call_twice_in_a_row(monkeypatch):
    rosko = built()
    # a large handle first, then a smaller one: the second call must not see
    # the first call's row counts left in the shared array
    cases = [(_handle(rosko, 3000, 900, 0.9, 81, "powerlaw"), 3136),
             (_handle(rosko, 700, 1500, 0.97, 82, "uniform"), 196)]
    want = [rosko.rosko_features(h, N) for h, N in cases]
    out = torch.zeros((2, 16), dtype=torch.float32, device="cuda")
    # first call on this device: looks up the static array (which loads the
    # library's module data for it, once)
    rosko.rosko_features_static(cases[1][0], 5, out=out[0])
    torch.cuda.synchronize()
    used0 = torch.cuda.memory_allocated()
    # arm the library's allocation-failure hook: the next device allocation
    # made by the library fails, so a hidden allocation would surface here
    monkeypatch.setenv("ROSKO_FAIL_ALLOC", "1")
    for i, (h, N) in enumerate(cases):
        rosko.rosko_features_static(h, N, out=out[i])
    torch.cuda.synchronize()
    assert rosko.rosko_device_status(clear=True) == 0
    # nothing came from torch's allocator either (the armed hook above covers
    # the library's own allocation paths)
    assert torch.cuda.memory_allocated() == used0
    got = out.cpu().numpy().astype(np.float64)
    for g, w in zip(got, want):
        # FP32 arithmetic on the same exact counts as the FP64 definitions
        assert np.allclose(g, w, rtol=1e-5, atol=1e-6), (g, w)
    # the hook is still armed: the allocating variant fails with OOM
    with pytest.raises(RuntimeError, match="OOM"):
        rosko.rosko_features(cases[0][0], 3136)
    monkeypatch.delenv("ROSKO_FAIL_ALLOC")
    # and the pair again, now in the opposite order
    for i, (h, N) in enumerate(reversed(cases)):
        rosko.rosko_features_static(h, N, out=out[i])
    got = out.cpu().numpy().astype(np.float64)
    for g, w in zip(got, reversed(want)):
        assert np.allclose(g, w, rtol=1e-5, atol=1e-6), (g, w)


@pytest.mark.gpu
def test_static_features_rejects_more_rows_than_the_array():
    rosko = built()
    M = (1 << 20) + 1
    A = torch.zeros((M, 8), dtype=torch.float32, device="cuda")
    A[::1000, 3] = 1.0
    h = rosko.rosko_pack(A, rosko.BF16, m_r=32)      # 32-row panels: P < 65536
    out = torch.full((16,), 7.0, device="cuda")
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        rosko.rosko_features_static(h, 64, out=out)
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)         # nothing was enqueued
    # the largest size served
    h2 = rosko.rosko_pack(A[: 1 << 20], rosko.BF16, m_r=32)
    rosko.rosko_features_static(h2, 64, out=out)
    want = rosko.rosko_features(h2, 64)
    assert np.allclose(out.cpu().numpy(), want, rtol=1e-5, atol=1e-6)


@pytest.mark.gpu
def test_feature_calls_refuse_a_handle_of_another_device():
    rosko = built()
    h = _handle(rosko, 300, 400, 0.9, 83)
    # the handle records its device right after its 8-byte tag; pretend it
    # belongs to another GPU (no second GPU is touched: the call is refused
    # on the host before any launch)
    dev_field = ctypes.c_int.from_address(h.handle.value + 8)
    own = dev_field.value
    out = torch.full((16,), 7.0, device="cuda")
    try:
        dev_field.value = own + 1
        with pytest.raises(RuntimeError, match="INVALID_ARG"):
            rosko.rosko_features_static(h, 64, out=out)
        with pytest.raises(RuntimeError, match="INVALID_ARG"):
            rosko.rosko_features(h, 64)
    finally:
        dev_field.value = own
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)
    rosko.rosko_features_static(h, 64, out=out)
    assert np.allclose(out.cpu().numpy(), rosko.rosko_features(h, 64), rtol=1e-5, atol=1e-6)
