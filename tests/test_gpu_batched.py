"""Batched SpMM (one persistent tensor-core launch per CTA-tile shape for
every problem's dense tiles, one row-direct launch for the row-direct sparse
remainders, other remainders per problem) against the oracle, and its
capture/replay in a CUDA graph.  GPU only."""
import numpy as np
import pytest
import torch

from tests._lib import built
from tests.test_gpu_spmm import _ldpad
from oracle.spmm import spmm, normalized_error
from oracle.quant import bf16_round
from paper_2307_03930_gb300 import inputs as gen

pytestmark = pytest.mark.gpu


def _problems(seed, shapes):
    out = []
    for j, (M, K, N, s, pat) in enumerate(shapes):
        A = gen.sparse_weight(M, K, s, gen.rng_for(seed, j), pat)
        B = gen.relu_normal((K, N), gen.rng_for(seed, 100 + j))
        out.append((A, B))
    return out


SHAPES = [(300, 500, 257, 0.7, "uniform"), (64, 96, 196, 0.99, "uniform"),
          (513, 1000, 700, 0.95, "powerlaw"), (130, 77, 300, 0.999, "uniform"),
          (256, 640, 128, 0.9, "block4x1"), (1000, 300, 450, 0.985, "powerlaw")]


def _run_batched(rosko, probs, tiles=None, accumulate=False, C0s=None, f32=False):
    code, bt, esz = (rosko.F32, torch.float32, 4) if f32 else (rosko.BF16, torch.bfloat16, 2)
    hs = [rosko.rosko_pack(torch.from_numpy(A).cuda(), code) for A, _ in probs]
    Bs = [_ldpad(torch.from_numpy(B).to(bt), esz) for _, B in probs]
    Cs = [torch.full((A.shape[0], B.shape[1]), float("nan"), device="cuda") for A, B in probs]
    if C0s is not None:
        for C, C0 in zip(Cs, C0s):
            C.copy_(torch.from_numpy(C0))
    l0 = rosko.rosko_kernel_launches()
    rosko.rosko_spmm_batched(hs, Bs, Cs, accumulate=accumulate, tiles=tiles)
    torch.cuda.synchronize()
    assert rosko.rosko_device_status(clear=True) == 0
    return hs, Bs, Cs, rosko.rosko_kernel_launches() - l0


@pytest.mark.parametrize("accumulate", [False, True])
def test_batched_matches_oracle(accumulate):
    rosko = built()
    probs = _problems(71, SHAPES)
    C0s = [np.random.default_rng(j).standard_normal((A.shape[0], B.shape[1])).astype(np.float32)
           for j, (A, B) in enumerate(probs)] if accumulate else None
    hs, Bs, Cs, launches = _run_batched(rosko, probs, accumulate=accumulate, C0s=C0s)
    for j, ((A, B), C) in enumerate(zip(probs, Cs)):
        ref, D = spmm(bf16_round(A), bf16_round(B), C0=C0s[j] if accumulate else None)
        if accumulate:
            D = D + np.abs(C0s[j])
        assert normalized_error(C.cpu().numpy(), ref, D) <= 1e-5, j
    # one dense launch per CTA-tile shape (at most four) + one row-direct
    # launch for every sparse remainder
    assert launches <= 5


@pytest.mark.parametrize("MC", [128, 256])
def test_batched_forced_dense_for_all(MC):
    rosko = built()
    probs = _problems(72, SHAPES)
    tiles = [rosko.make_tile(dense_split_pm=1, dense_m_c=MC) for _ in probs]
    hs, Bs, Cs, launches = _run_batched(rosko, probs, tiles=tiles)
    for (A, B), C in zip(probs, Cs):
        ref, D = spmm(bf16_round(A), bf16_round(B))
        assert normalized_error(C.cpu().numpy(), ref, D) <= 1e-5
    # every tile has density >= 1 per mille except the 99.9% problem's:
    # two tile shapes here (small K: 128 columns) + one row-direct launch
    assert launches <= 3


def test_batched_graph_capture_and_replay():
    rosko = built()
    probs = _problems(73, SHAPES[:4])
    hs, Bs, Cs, _ = _run_batched(rosko, probs)       # first call outside capture
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rosko.rosko_spmm_batched(hs, Bs, Cs)
    # new activations in place, replay
    new_B = [gen.relu_normal(B.shape, gen.rng_for(74, j)) for j, (_, B) in enumerate(probs)]
    for Bd, Bn in zip(Bs, new_B):
        Bd.copy_(torch.from_numpy(Bn).to(torch.bfloat16))
    g.replay()
    torch.cuda.synchronize()
    for (A, _), Bn, C in zip(probs, new_B, Cs):
        ref, D = spmm(bf16_round(A), bf16_round(Bn))
        assert normalized_error(C.cpu().numpy(), ref, D) <= 1e-5


@pytest.mark.parametrize("accumulate", [False, True])
def test_batched_fp32_row_direct_is_one_launch(accumulate):
    # FP32 has no tensor-core path; every problem below 15% density runs
    # row-direct, and all of them share one launch
    rosko = built()
    shapes = [(300, 500, 257, 0.9, "uniform"), (64, 96, 196, 0.99, "uniform"),
              (513, 1000, 700, 0.95, "powerlaw"), (130, 77, 300, 0.999, "uniform"),
              (256, 640, 128, 0.9, "block4x1"), (33, 20, 5, 0.95, "uniform")]
    probs = _problems(75, shapes)
    C0s = [np.random.default_rng(j).standard_normal((A.shape[0], B.shape[1])).astype(np.float32)
           for j, (A, B) in enumerate(probs)] if accumulate else None
    hs, Bs, Cs, launches = _run_batched(rosko, probs, accumulate=accumulate, C0s=C0s, f32=True)
    for j, ((A, B), C) in enumerate(zip(probs, Cs)):
        ref, D = spmm(A, B, C0=C0s[j] if accumulate else None)
        if accumulate:
            D = D + np.abs(C0s[j])
        assert normalized_error(C.cpu().numpy(), ref, D) <= 1e-5, j
    assert launches == 1


def test_c4_full_size_batch_under_graph_replay():
    """The 64 uneven layers the benchmark times (seed 3: M, K log-uniform in
    [64, 4096], N in [196, 12544], sparsity uniform in [0.70, 0.99], BF16,
    uniform masks, post-ReLU B), run by one rosko_spmm_batched call captured
    in a CUDA graph and replayed; every problem's C is compared with the
    oracle on 16 sampled rows (all columns)."""
    rosko = built()
    seed = 3
    shapes = gen.c4_shapes(seed, 64)
    hs, Bs, Cs, probs = [], [], [], []
    for j, (M_, K_, N_, s_) in enumerate(shapes):
        A = gen.sparse_weight(M_, K_, s_, gen.rng_for(seed, 1, j), "uniform")
        B = gen.relu_normal((K_, N_), gen.rng_for(seed, 2, j))
        hs.append(rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.BF16))
        Bs.append(_ldpad(torch.from_numpy(B).to(torch.bfloat16), 2))
        Cs.append(torch.full((M_, N_), float("nan"), device="cuda"))
        probs.append((A, B))
    # first call uncaptured (it resolves and caches what capture must not do)
    rosko.rosko_spmm_batched(hs, Bs, Cs)
    torch.cuda.synchronize()
    for C in Cs:
        C.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rosko.rosko_spmm_batched(hs, Bs, Cs)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert rosko.rosko_device_status(clear=True) == 0
    worst = 0.0
    for j, ((A, B), C) in enumerate(zip(probs, Cs)):
        M_ = A.shape[0]
        rows = np.unique(np.random.default_rng(1000 + j).integers(0, M_, 16))
        ref, D = spmm(bf16_round(A[rows]), bf16_round(B))
        err = normalized_error(C[torch.from_numpy(rows).cuda()].cpu().numpy(), ref, D)
        worst = max(worst, err)
        assert err <= 1e-5, (j, shapes[j], err)
    assert worst <= 1e-5
