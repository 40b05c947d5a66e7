"""Host logic of the selector's measurement sweep and training (CPU): the
learned mode's deference rule, the soft training targets, the regret table
and the sweep's problem distributions, each on hand-worked examples."""
import math

import numpy as np

from paper_2307_03930_gb300 import selector as sel

LN2 = math.log(2.0)


def test_choose_defers_within_the_margin():
    # candidate 1 is the analytic rule's; the network's top pick must beat
    # its logit by more than ln 2 to run
    ok = np.ones((4, 3), dtype=bool)
    z = np.array([[0.0, 1.0, 1.0 + 0.9 * LN2],     # within the margin: rule
                  [0.0, 1.0, 1.0 + 1.1 * LN2],     # beyond it: candidate 2
                  [5.0, 1.0, 0.0],                 # clear win: candidate 0
                  [0.0, 3.0, 1.0]])                # the rule is the top: rule
    eq = np.array([1, 1, 1, 1])
    assert sel.choose(z, ok, eq).tolist() == [-1, 2, 0, -1]


def test_choose_without_a_rule_candidate_and_with_inapplicable_ones():
    ok = np.array([[True, False, True], [True, True, True]])
    z = np.array([[1.0, 9.0, 2.0],      # candidate 1 does not apply
                  [1.0, 2.0, 0.0]])
    eq = np.array([-1, -1])             # the rule's schedule is no candidate
    assert sel.choose(z, ok, eq).tolist() == [2, 1]


def test_soft_targets_hand_values():
    t = np.array([[1.0, 2.0, np.nan, 1.5]])
    tau = 0.5
    w = np.array([1.0, math.exp(-1.0 / tau), 0.0, math.exp(-0.5 / tau)])
    got = sel.soft_targets(t, tau)
    assert np.allclose(got[0], w / w.sum(), rtol=1e-6)
    # tau -> 0: all the mass on the fastest candidate
    assert np.allclose(sel.soft_targets(t, 1e-4)[0], [1, 0, 0, 0], atol=1e-6)
    assert got.dtype == np.float32


def test_regret_hand_example():
    times = np.array([[1.0, 2.0], [3.0, 1.5]])
    analytic = np.array([2.0, 3.0])
    choice = np.array([0, -1])          # problem 2 keeps the analytic rule
    r = sel.regret(times, analytic, choice)
    # chosen times 1 and 3 against best 1 and 1.5
    assert math.isclose(r["mlp_regret"], (0.0 + 1.0) / 2)
    assert math.isclose(r["analytic_regret"], (1.0 + 1.0) / 2)
    assert math.isclose(r["mlp_vs_analytic_geomean_speedup"], math.sqrt(2.0 * 1.0))
    assert r["n"] == 2


def test_sweep_problem_distributions():
    for family, (mlo, mhi), (nlo, nhi), (slo, shi) in (
            ("layers", (64, 4096), (196, 12544), (0.70, 0.99)),
            ("conv", (64, 2048), (196, 12544), (0.5, 0.999))):
        a = sel.random_problems(4, 300, family)
        assert a == sel.random_problems(4, 300, family)          # seeded
        assert a != sel.random_problems(5, 300, family)
        M, K, N, s = (np.array([p[i] for p in a]) for i in range(4))
        assert M.min() >= mlo and M.max() <= mhi
        assert N.min() >= nlo and N.max() <= nhi
        assert s.min() >= slo and s.max() <= shi
        if family == "layers":
            assert K.min() >= 64 and K.max() <= 4096
        else:
            assert np.all(K % 9 == 0) and K.min() >= 9 * 32 and K.max() <= 9 * 1024
        assert {p[4] for p in a} == set(sel.PATTERNS)
        assert [p[5] for p in a] == list(range(300))
    # the two families draw from different streams
    assert sel.random_problems(4, 5, "layers") != sel.random_problems(4, 5, "conv")


def _split_sweep(n, rng):
    """Features and a 60-column time grid (ms) whose all-dense and
    row-direct columns follow two known linear models exactly."""
    M = rng.integers(64, 4096, n).astype(float)
    K = rng.integers(64, 4096, n).astype(float)
    N = rng.integers(196, 12544, n).astype(float)
    d = rng.uniform(0.001, 0.3, n)
    nnz = np.round(d * M * K)
    f = np.zeros((n, 16))
    f[:, 0], f[:, 1], f[:, 2] = np.log2(M), np.log2(K), np.log2(N)
    f[:, 3] = nnz / (M * K)
    t = np.full((n, 60), 1.0)                      # every other candidate slow
    dense_us = 12.0 + 2 * M * K * N / 0.6e15 * 1e6
    direct_us = 5.0 + 2 * nnz * N / 11e12 * 1e6
    i_rd = np.where((f[:, 3] < 0.015) & (N >= 1024), 3, 11)
    r = np.arange(n)
    t[r, i_rd * 5 + 1] = dense_us * 1e-3
    t[r, i_rd * 5] = direct_us * 1e-3
    t[r, i_rd * 5 + 3] = dense_us * 1e-3
    return f, t


def test_fit_split_recovers_planted_models():
    f, t = _split_sweep(400, np.random.default_rng(3))
    m = sel.fit_split(f, t)
    assert abs(m["dense_us"] - 12.0) < 1e-6 and abs(m["direct_us"] - 5.0) < 1e-6
    assert abs(m["dense_flops"] / 0.6e15 - 1) < 1e-9 and abs(m["direct_bytes_s"] / 11e12 - 1) < 1e-9
    # exact models choose the faster path every time: no regret
    r = sel.split_regret(f, t, m)
    assert r["vs_best"] == 0.0 and r["vs_better_of_two"] == 0.0
    # swapping the two rates misroutes some layers: positive regret
    bad = dict(m, dense_flops=m["direct_bytes_s"] * 50, direct_bytes_s=m["dense_flops"] / 50)
    assert sel.split_regret(f, t, bad)["vs_better_of_two"] > 0.0
