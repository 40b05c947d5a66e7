"""INT8 x INT8 -> INT32 through the BF16 tensor pipe: the INT8 codes are
exact in BF16, every K chunk of at most 1024 sums exactly in the FP32
accumulator (1024 * 127^2 < 2^24), and the chunks are converted and added
into INT32 C.  Results must match the integer oracle bit for bit."""
import numpy as np
import pytest
import torch

from tests._lib import built
from tests.test_gpu_spmm import _ldpad
from oracle.spmm import spmm_int
from oracle.quant import quantize_rows_int8, quantize_cols_int8
from paper_2307_03930_gb300 import inputs as gen

pytestmark = pytest.mark.gpu


def _case(M, K, N, s, seed, pattern="uniform", magnitude=False):
    rng = gen.rng_for(seed, M, K)
    A = (gen.magnitude_prune(gen.normal((M, K), rng), s) if magnitude
         else gen.sparse_weight(M, K, s, rng, pattern))
    B = gen.normal((K, N), gen.rng_for(seed, K, N))
    qa, _ = quantize_rows_int8(A)
    qb, _ = quantize_cols_int8(B)
    return A, qa, qb


@pytest.mark.parametrize("M,K,N,s,pattern,accumulate", [
    (300, 2500, 520, 0.7, "uniform", False),     # three K chunks, the last partial
    (300, 2500, 520, 0.7, "uniform", True),
    (129, 1024, 257, 0.5, "uniform", False),     # exactly one chunk, ragged tiles
    (700, 3000, 300, 0.9, "powerlaw", False),    # mixed: dense tiles + sparse rest
    (64, 5000, 96, 0.3, "uniform", False),       # near-dense rows, sums near 2^24 per chunk
])
def test_int8_tensor_core_bit_exact(M, K, N, s, pattern, accumulate):
    rosko = built()
    A, qa, qb = _case(M, K, N, s, 31, pattern)
    h = rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.I8)
    Bd = _ldpad(torch.from_numpy(qb), 1)
    C0 = np.random.default_rng(5).integers(-1000, 1000, (M, N)).astype(np.int32)
    C = torch.from_numpy(C0.copy()).cuda() if accumulate else \
        torch.full((M, N), -7, dtype=torch.int32, device="cuda")
    pm = 1
    if pattern == "powerlaw":
        # a threshold between the tiles' densities: some tiles on the tensor
        # cores, the others on the row-direct kernel
        dens = sorted(np.count_nonzero(qa[r:r + 128]) * 1000.0 / (min(128, M - r) * K)
                      for r in range(0, M, 128))
        pm = int(dens[len(dens) // 2]) + 1
        assert dens[-1] >= pm > dens[0]
    tile = rosko.make_tile(dense_split_pm=pm)
    pl = rosko.rosko_spmm_plan(h, Bd, C, tile=tile)
    assert pl["dense_tiles"] > 0
    if pattern == "powerlaw":
        assert pl["sparse_panels"] > 0 and pl["dense_tiles"] < -(-M // 128)
    rosko.rosko_spmm(h, Bd, C, tile=tile, accumulate=accumulate)
    torch.cuda.synchronize()
    assert rosko.rosko_device_status(clear=True) == 0
    want = spmm_int(qa, qb, C0=C0 if accumulate else None)
    assert np.array_equal(C.cpu().numpy().astype(np.int64), want)


@pytest.mark.parametrize("Mx,Kx", [(11008, 4096), (4096, 11008)])
def test_int8_tensor_core_ffn_sampled(Mx, Kx):
    # the transformer-FFN layers at 70% (magnitude-pruned), 2048 tokens: the
    # analytic rule sends them to the tensor cores; 16 sampled rows against
    # the oracle, bit for bit
    rosko = built()
    A, qa, qb = _case(Mx, Kx, 2048, 0.7, 2, magnitude=True)
    h = rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.I8)
    Bd = _ldpad(torch.from_numpy(qb), 1)
    C = torch.empty((Mx, 2048), dtype=torch.int32, device="cuda")
    pl = rosko.rosko_spmm_plan(h, Bd, C)
    assert pl["dense_tiles"] == -(-Mx // 128) and pl["sparse_panels"] == 0
    rosko.rosko_spmm(h, Bd, C)
    torch.cuda.synchronize()
    assert rosko.rosko_device_status(clear=True) == 0
    rows = np.unique(np.random.default_rng(Mx).integers(0, Mx, 16))
    want = spmm_int(qa[rows], qb)
    got = C[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.int64)
    assert np.array_equal(got, want)


def test_int8_dequant_output_stays_on_cuda_cores():
    # FP32 output with scales (C = s_i t_j sum q_a q_b) keeps the sparse path
    rosko = built()
    A, qa, qb = _case(200, 1500, 130, 0.6, 7)
    h = rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.I8)
    Bd = _ldpad(torch.from_numpy(qb), 1)
    C = torch.empty((200, 130), device="cuda")
    t = torch.ones(130, device="cuda")
    pl = rosko.rosko_spmm_plan(h, Bd, C, col_scale=t)
    assert pl["dense_tiles"] == 0
