"""Tensor-core dense-panel path (tcgen05, BF16 in / FP32 accumulate) and the
sparse/dense split, against the FP64 oracle on the BF16-rounded inputs
(normalised error <= 1e-5).  GPU only."""
import numpy as np
import pytest
import torch

from tests._lib import built
from tests.test_gpu_spmm import _ldpad
from oracle.spmm import spmm, normalized_error
from oracle.quant import bf16_round
from paper_2307_03930_gb300 import inputs as gen

pytestmark = pytest.mark.gpu


def _run(rosko, A, B, tile, rows=None, accumulate=False, C0=None, dense_min_pm=0):
    M, K = A.shape
    N = B.shape[1]
    h = rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.BF16, dense_min_pm=dense_min_pm)
    Bd = _ldpad(torch.from_numpy(B).to(torch.bfloat16), 2)
    # C = A.B overwrites C: start from NaN so that an element no kernel
    # writes (or a missed zero fill) fails the comparison
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    if C0 is not None:
        C.copy_(torch.from_numpy(C0))
    # a zero fill of C ahead of a tensor-core launch is one small kernel (the
    # tensor-core launch depends on it programmatically); it is counted apart
    # from the product's launches (without one, the fill is a memset)
    pl = rosko.rosko_spmm_plan(h, Bd, C, tile=tile, accumulate=accumulate)
    fill = 1 if (pl["zero_fill"] and pl["dense_tiles"] > 0) else 0
    l0 = rosko.rosko_kernel_launches()
    rosko.rosko_spmm(h, Bd, C, tile=tile, accumulate=accumulate)
    launches = rosko.rosko_kernel_launches() - l0 - fill
    torch.cuda.synchronize()
    assert rosko.rosko_device_status(clear=True) == 0
    rows = np.arange(M) if rows is None else np.asarray(rows)
    ref, D = spmm(bf16_round(A), bf16_round(B), rows=rows, C0=C0)
    if C0 is not None:
        D = D + np.abs(C0[rows].astype(np.float64))
    err = normalized_error(C.cpu().numpy()[rows], ref, D)
    return err, launches


@pytest.mark.parametrize("M,K,N", [(128, 64, 128), (130, 77, 257), (256, 1000, 300),
                                   (1, 8, 1), (300, 129, 64), (384, 2048, 520)])
@pytest.mark.parametrize("TN,ctas", [(128, 0), (256, 0), (256, 7), (128, 1), (256, 3)])
@pytest.mark.parametrize("MC", [128, 256])
def test_all_dense(M, K, N, TN, ctas, MC):
    # stream-K over `ctas` CTAs (0: one per SM): tiles whose K range is cut
    # between CTAs are added with atomics, whole tiles are stored; MC = 256
    # pairs two 128-row tiles per CTA tile (an odd tile count leaves the
    # second half of the last pair empty)
    rosko = built()
    A = gen.sparse_weight(M, K, 0.5, gen.rng_for(7, M, K), "uniform")
    B = gen.normal((K, N), gen.rng_for(8, K, N))
    t = rosko.make_tile(dense_split_pm=1, dense_n_r=TN, dense_split_k=ctas, dense_m_c=MC)
    err, launches = _run(rosko, A, B, t)
    assert err <= 1e-5, err
    assert launches == 1          # only the tensor-core kernel ran


@pytest.mark.parametrize("MC,order", [(128, 0), (256, 0), (128, 4), (256, 1)])
def test_mixed_split_powerlaw(MC, order):
    # power-law rows give tiles of very different density: some run dense,
    # the others on the sparse kernel (its panel list skips the dense tiles'
    # panels), in one call
    rosko = built()
    A = gen.sparse_weight(1000, 700, 0.97, gen.rng_for(9), "powerlaw")
    B = gen.relu_normal((700, 333), gen.rng_for(10))
    t = rosko.make_tile(dense_split_pm=30, dense_m_c=MC, order=order)
    err, launches = _run(rosko, A, B, t)
    assert err <= 1e-5, err
    dens = [(A[i:i + 128] != 0).mean() for i in range(0, 1000, 128)]
    n_dense = sum(d * 1000 >= 30 for d in dens)
    assert 0 < n_dense < len(dens)
    assert launches == 2


@pytest.mark.parametrize("ctas", [1, 5, 0])
@pytest.mark.parametrize("MC", [128, 256])
def test_dense_accumulate(ctas, MC):
    rosko = built()
    A = gen.sparse_weight(200, 512, 0.8, gen.rng_for(11), "uniform")
    B = gen.normal((512, 200), gen.rng_for(12))
    C0 = np.random.default_rng(3).standard_normal((200, 200)).astype(np.float32)
    t = rosko.make_tile(dense_split_pm=1, dense_split_k=ctas, dense_m_c=MC)
    err, _ = _run(rosko, A, B, t, accumulate=True, C0=C0)
    assert err <= 1e-5, err


def test_bad_dense_m_c_rejected():
    rosko = built()
    A = gen.sparse_weight(256, 64, 0.5, gen.rng_for(15), "uniform")
    h = rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.BF16)
    B = _ldpad(torch.zeros((64, 64), dtype=torch.bfloat16), 2)
    C = torch.zeros((256, 64), device="cuda")
    with pytest.raises(RuntimeError):
        rosko.rosko_spmm(h, B, C, tile=rosko.make_tile(dense_split_pm=1, dense_m_c=192))


def test_no_copy_means_sparse_only():
    rosko = built()
    A = gen.sparse_weight(256, 300, 0.5, gen.rng_for(13), "uniform")
    B = gen.normal((300, 100), gen.rng_for(14))
    t = rosko.make_tile(dense_split_pm=1)
    err, launches = _run(rosko, A, B, t, dense_min_pm=1001)
    assert err <= 1e-5 and launches == 1


@pytest.mark.parametrize("s", [0.5, 0.9, 0.95])
def test_c2_dense_full_size_sampled(s):
    # the bench's launch configuration: analytic schedule (dense split at 5 per mille)
    rosko = built()
    rng = gen.rng_for(1, int(round(s * 1000)))
    A = gen.magnitude_prune(gen.normal((512, 4608), rng), s)
    B = gen.relu_normal((4608, 3136), rng)
    rows = np.random.default_rng(int(s * 1000)).choice(512, 40, replace=False)
    err, launches = _run(rosko, A, B, None, rows=rows)
    assert err <= 1e-5, err
    assert launches == 1


def test_plan_reports_the_split_and_launches_nothing():
    rosko = built()
    A = gen.sparse_weight(1000, 700, 0.97, gen.rng_for(9), "powerlaw")
    h = rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.BF16)
    B = _ldpad(torch.zeros((700, 333), dtype=torch.bfloat16), 2)
    C = torch.full((1000, 333), 3.0, device="cuda")
    t = rosko.make_tile(dense_split_pm=30, order=4)
    l0 = rosko.rosko_kernel_launches()
    pl = rosko.rosko_spmm_plan(h, B, C, tile=t)
    torch.cuda.synchronize()
    assert rosko.rosko_kernel_launches() == l0
    assert torch.all(C == 3.0)                 # nothing written
    dens = [(A[i:i + 128] != 0).mean() for i in range(0, 1000, 128)]
    n_dense = sum(d * 1000 >= 30 for d in dens)
    dense_panels = sum(-(-min(128, 1000 - 128 * j) // 16) for j, d in enumerate(dens)
                       if d * 1000 >= 30)
    assert pl["dense_tiles"] == n_dense
    assert pl["sparse_panels"] == -(-1000 // 16) - dense_panels
    assert pl["order"] == 4
    # sparse only: no dense tile
    pl = rosko.rosko_spmm_plan(h, B, C, tile=rosko.make_tile(dense_split_pm=1001))
    assert pl["dense_tiles"] == 0 and pl["sparse_panels"] == -(-1000 // 16)


@pytest.mark.parametrize("ctas,TN,MC", [(5, 128, 128), (16, 256, 128), (7, 128, 256)])
@pytest.mark.parametrize("accumulate", [False, True])
def test_tile_aligned_split(ctas, TN, MC, accumulate):
    # at least four tiles per CTA: each CTA owns whole tiles (stored, not
    # reduced; C is not zero-filled first)
    rosko = built()
    A = gen.sparse_weight(1000, 300, 0.6, gen.rng_for(17), "uniform")
    B = gen.normal((300, 1000), gen.rng_for(18))
    C0 = np.random.default_rng(4).standard_normal((1000, 1000)).astype(np.float32) \
        if accumulate else None
    t = rosko.make_tile(dense_split_pm=1, dense_n_r=TN, dense_split_k=ctas, dense_m_c=MC)
    err, launches = _run(rosko, A, B, t, accumulate=accumulate, C0=C0)
    assert err <= 1e-5, err
    assert launches == 1
