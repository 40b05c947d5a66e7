"""Failure detection on the GPU without a fault: a bounded device wait that
runs out sets the timeout bit of the device status word, its kernel returns,
and the context stays usable.  The wait is forced to expire by the library's
diagnostic launch (an mbarrier that nothing completes), with the wait limit
lowered to a few milliseconds."""
import time

import numpy as np
import pytest
import torch

from tests._lib import built
from oracle.spmm import spmm, normalized_error
from oracle.quant import bf16_round
from paper_2307_03930_gb300 import inputs as gen

pytestmark = pytest.mark.gpu


def test_wait_limit_rejects_negative():
    rosko = built()
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        rosko.rosko_set_wait_limit(-1)


def test_expired_wait_sets_timeout_and_context_survives():
    rosko = built()
    assert rosko.rosko_device_status(clear=True) == 0
    rosko.rosko_set_wait_limit(5_000_000)          # 5 ms
    try:
        t0 = time.perf_counter()
        rosko.rosko_probe_bounded_wait()
        bits = rosko.rosko_device_status(clear=True)   # synchronises
        waited = time.perf_counter() - t0
    finally:
        rosko.rosko_set_wait_limit(0)
    assert bits & 1, bits                          # bit 1: a bounded wait ran out
    assert waited < 1.0, waited                    # the short limit, not the 2 s default
    assert rosko.rosko_device_status() == 0        # cleared
    # the context is intact: a pipelined kernel (tensor-core path, with its
    # own bounded waits) and the row-direct path still give oracle results
    A = gen.sparse_weight(384, 1280, 0.9, gen.rng_for(5, 1), "uniform")
    B = gen.relu_normal((1280, 520), gen.rng_for(5, 2))
    h = rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.BF16)
    Bd = torch.from_numpy(B).cuda().to(torch.bfloat16)
    ref, D = spmm(bf16_round(A), bf16_round(B))
    for tile in (rosko.make_tile(dense_split_pm=1), rosko.make_tile(order=4, dense_split_pm=1001)):
        C = torch.full((384, 520), float("nan"), device="cuda")
        rosko.rosko_spmm(h, Bd, C, tile=tile)
        torch.cuda.synchronize()
        assert normalized_error(C.cpu().numpy(), ref, D) <= 1e-5
    assert rosko.rosko_device_status(clear=True) == 0


def test_default_limit_lets_a_normal_wait_complete():
    # with the default limit restored, the pipelined kernels' waits complete
    # normally (no spurious timeout bit over a batch of launches)
    rosko = built()
    A = gen.sparse_weight(512, 2048, 0.8, gen.rng_for(6, 1), "uniform")
    B = gen.relu_normal((2048, 1024), gen.rng_for(6, 2))
    h = rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.BF16)
    Bd = torch.from_numpy(B).cuda().to(torch.bfloat16)
    C = torch.empty((512, 1024), device="cuda")
    for _ in range(20):
        rosko.rosko_spmm(h, Bd, C, tile=rosko.make_tile(dense_split_pm=1))
    torch.cuda.synchronize()
    assert rosko.rosko_device_status(clear=True) == 0
