"""Consecutive SpMMs on one stream where each call's B is the previous
call's C, issued back to back without synchronising: the row-direct kernel
is launched as a programmatic dependent of the launch before it and must
read nothing before that launch has completed.  Each layer is checked
against the FP64 oracle applied to the input the GPU actually had (the
previous layer's GPU output); outputs start as NaN, so a read of a buffer
not yet written would show.  GPU only."""
import numpy as np
import pytest
import torch

from tests._lib import built
from oracle.spmm import spmm, normalized_error
from paper_2307_03930_gb300 import inputs as gen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("s", [0.9, 0.99])
def test_chained_layers_read_the_previous_output(s):
    rosko = built()
    dims = [(300, 256), (256, 200), (200, 128), (128, 64)]   # (K, M) per layer
    N = 256
    rng = gen.rng_for(21, int(s * 100))
    As = [gen.sparse_weight(M, K, s, gen.rng_for(22, i, int(s * 100)), "uniform")
          for i, (K, M) in enumerate(dims)]
    hs = [rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.F32) for A in As]
    B0 = torch.from_numpy(gen.normal((dims[0][0], N), rng)).cuda()
    for rep in range(3):
        outs = [torch.full((M, N), float("nan"), device="cuda") for _, M in dims]
        x = B0 * (rep + 1)
        for h, C in zip(hs, outs):
            rosko.rosko_spmm(h, x, C)      # no synchronisation in between
            x = C
        torch.cuda.synchronize()
        assert rosko.rosko_device_status(clear=True) == 0
        prev = (B0 * (rep + 1)).cpu().numpy()
        for A, C in zip(As, outs):
            got = C.cpu().numpy()
            assert np.all(np.isfinite(got))
            ref, D = spmm(A, prev.astype(np.float32))
            assert normalized_error(got, ref, D) <= 1e-5
            prev = got
