"""Autotuner and schedule modes (GPU): every candidate of the fixed set is
correct, the autotuner's choice is cached and reused, and the result matches
the oracle whichever schedule runs."""
import numpy as np
import pytest
import torch

from tests._lib import built
from tests.test_gpu_spmm import _problem, run, check, _ldpad

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["bf16", "f32"])
@pytest.mark.parametrize("s", [0.6, 0.99])
def test_every_candidate_is_correct(mode, s):
    rosko = built()
    A, B = _problem(260, 900, 300, s, seed=41)
    dt = rosko.BF16 if mode == "bf16" else rosko.F32
    h = rosko.rosko_pack(torch.from_numpy(A).cuda(), dt)
    n_ok = 0
    for i in range(rosko.rosko_num_candidates()):
        t = rosko.rosko_candidate(h, 300, i)
        if t is None:
            continue
        n_ok += 1
        check(mode, *run(rosko, A, B, mode, m_r=16, tile=t))
    assert n_ok >= (8 if mode == "f32" else 30)


def test_autotune_choice_is_cached_and_correct():
    rosko = built()
    A, B = _problem(384, 1200, 500, 0.97, seed=42)
    Ad = torch.from_numpy(A).cuda()
    h = rosko.rosko_pack(Ad, rosko.BF16)
    Bd = _ldpad(torch.from_numpy(B).to(torch.bfloat16), 2)
    C = torch.empty((384, 500), device="cuda")
    best, times = rosko.rosko_autotune(h, Bd, C)
    assert len(times) == rosko.rosko_num_candidates()
    ok = [t for t in times if t is not None]
    assert ok and all(t > 0 for t in ok)
    # the returned tile is the fastest applicable candidate
    i_best = int(np.argmin([t if t is not None else np.inf for t in times]))
    cand = rosko.rosko_candidate(h, 500, i_best)
    assert cand.as_dict() == best.as_dict()
    # mode AUTOTUNE reuses it without searching again (no extra launches:
    # at most a zero fill, a tensor-core and a sparse launch)
    l0 = rosko.rosko_kernel_launches()
    rosko.rosko_spmm(h, Bd, C, tile=rosko.make_tile(mode=rosko.SCHED_AUTOTUNE))
    assert rosko.rosko_kernel_launches() - l0 <= 3
    check("bf16", *run(rosko, A, B, "bf16", m_r=16, tile=best))
