"""Learned selector kernels against the FP64 oracle (GPU): features of a packed
handle, MLP forward, softmax cross-entropy gradients, Adam, training, and the
LEARNED schedule mode."""
import numpy as np
import pytest
import torch

from tests._lib import built
from tests.test_gpu_spmm import _problem, run, check
from oracle import mlp as omlp
from oracle.features import features as ofeatures
from paper_2307_03930_gb300 import inputs as gen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pattern,M,K,s", [("uniform", 300, 500, 0.9), ("powerlaw", 517, 333, 0.97),
                                           ("block4x1", 256, 640, 0.95), ("uniform", 40, 70, 0.5)])
def test_features_match_oracle(pattern, M, K, s):
    rosko = built()
    A = gen.sparse_weight(M, K, s, gen.rng_for(51, M), pattern)
    A[:17] = 0                     # empty rows and (with m_r = 16) an empty panel
    h = rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.BF16, m_r=16)
    got = rosko.rosko_features(h, 777)
    want = ofeatures(A, 16, 777)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12), (got, want)


def _params(rng, n_in, n_out):
    return omlp.init_params(n_in, n_out, rng)


def _flat(params):
    return np.concatenate([p.ravel() for p in params]).astype(np.float32)


def _unflat(v, n_in, n_out):
    sizes = [n_in, 64, 64, 64, n_out]
    out, off = [], 0
    for l in range(4):
        w = v[off:off + sizes[l] * sizes[l + 1]].reshape(sizes[l + 1], sizes[l])
        off += w.size
        b = v[off:off + sizes[l + 1]]
        off += b.size
        out += [w, b]
    return out


def test_param_layout_and_forward():
    rosko = built()
    n_in, n_out, B = 16, rosko.rosko_num_candidates(), 37
    assert rosko.rosko_mlp_param_count(n_in, n_out) == (16 * 64 + 64) + 2 * (64 * 64 + 64) + (64 * n_out + n_out)
    rng = np.random.default_rng(0)
    P = _params(rng, n_in, n_out)
    X = rng.standard_normal((B, n_in)).astype(np.float32)
    flat = _flat(P)
    z = rosko.rosko_mlp_forward(torch.from_numpy(flat).cuda(), torch.from_numpy(X).cuda(), n_out)
    want, _ = omlp.forward([p.astype(np.float32).astype(np.float64) for p in P], X.astype(np.float64))
    got = z.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-4 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("soft", [False, True])
def test_loss_and_gradients_match_oracle(soft):
    rosko = built()
    n_in, n_out, B = 16, 40, 64
    rng = np.random.default_rng(1)
    P = [p.astype(np.float32).astype(np.float64) for p in _params(rng, n_in, n_out)]
    X = rng.standard_normal((B, n_in)).astype(np.float32)
    if soft:
        Y = rng.random((B, n_out)).astype(np.float32)
        Y /= Y.sum(axis=1, keepdims=True)
    else:
        Y = np.zeros((B, n_out), np.float32)
        Y[np.arange(B), rng.integers(0, n_out, B)] = 1
    loss, grads = rosko.rosko_mlp_loss_grad(torch.from_numpy(_flat(P)).cuda(),
                                            torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda())
    l_ref, g_ref = omlp.loss_and_grad(P, X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss.item() - l_ref) <= 1e-5 * max(1.0, abs(l_ref))
    g = _unflat(grads.cpu().numpy(), n_in, n_out)
    for a, b in zip(g, g_ref):
        assert np.max(np.abs(a - b)) <= 1e-4 * max(1e-3, np.max(np.abs(b))), np.max(np.abs(a - b))


@pytest.mark.parametrize("wd", [0.0, 0.5])
def test_adam_matches_oracle(wd):
    rosko = built()
    rng = np.random.default_rng(2)
    n = 1000
    p = rng.standard_normal(n).astype(np.float32)
    g = rng.standard_normal(n).astype(np.float32)
    m = (rng.standard_normal(n) * 0.1).astype(np.float32)
    v = (rng.random(n) * 0.01).astype(np.float32)
    tp, tg, tm, tv = [torch.from_numpy(x.copy()).cuda() for x in (p, g, m, v)]
    # hyper-parameters exactly representable in FP32, so that both sides use
    # the same beta values (1 - beta is then exact in FP32 as well)
    b1, b2, lr = float(np.float32(0.9)), float(np.float32(0.999)), float(np.float32(3e-3))
    rosko.rosko_mlp_adam(tp, tg, tm, tv, step=7, lr=lr, beta1=b1, beta2=b2, weight_decay=wd)
    (rp,), (rm,), (rv,) = omlp.adam_step([p.astype(np.float64)], [g.astype(np.float64)],
                                         [m.astype(np.float64)], [v.astype(np.float64)], t=7,
                                         lr=lr, beta1=b1, beta2=b2, weight_decay=wd)
    assert np.allclose(tp.cpu().numpy(), rp, rtol=1e-5, atol=1e-6)
    assert np.allclose(tm.cpu().numpy(), rm, rtol=1e-5, atol=1e-7)
    assert np.allclose(tv.cpu().numpy(), rv, rtol=1e-5, atol=1e-9)


def test_training_on_gpu_reduces_loss():
    rosko = built()
    n_in, n_out, B = 16, 40, 256
    rng = np.random.default_rng(3)
    X = rng.standard_normal((B, n_in)).astype(np.float32)
    # labels depend on the features: a learnable rule
    lab = (np.argmax(X[:, :4], axis=1) * 10 + (X[:, 5] > 0)).astype(int) % n_out
    Y = np.zeros((B, n_out), np.float32)
    Y[np.arange(B), lab] = 1
    P = torch.from_numpy(_flat(_params(rng, n_in, n_out))).cuda()
    m, v = torch.zeros_like(P), torch.zeros_like(P)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    l0 = None
    for step in range(1, 301):
        loss, g = rosko.rosko_mlp_loss_grad(P, Xd, Yd)
        if l0 is None:
            l0 = loss.item()
        rosko.rosko_mlp_adam(P, g, m, v, step, lr=3e-3)
    l1, _ = rosko.rosko_mlp_loss_grad(P, Xd, Yd)
    assert l1.item() < 0.3 * l0
    z = rosko.rosko_mlp_forward(P, Xd, n_out).cpu().numpy()
    assert (np.argmax(z, axis=1) == lab).mean() > 0.9


def test_learned_mode_uses_the_network_and_is_correct():
    rosko = built()
    n_out = rosko.rosko_num_candidates()
    A, B = _problem(256, 900, 300, 0.95, seed=61)
    h = rosko.rosko_pack(torch.from_numpy(A).cuda(), rosko.BF16)
    f = rosko.rosko_features(h, 300)
    # a network whose output bias prefers one applicable candidate
    target = next(i for i in range(n_out) if rosko.rosko_candidate(h, 300, i) is not None
                  and rosko.rosko_candidate(h, 300, i).order == 3)
    params = np.zeros(rosko.rosko_mlp_param_count(16, n_out), np.float32)
    params[-n_out + target] = 5.0
    rosko.rosko_selector_set(params, np.zeros(16), np.ones(16), f - 1, f + 1)
    t = rosko.make_tile(mode=rosko.SCHED_LEARNED)
    check("bf16", *run(rosko, A, B, "bf16", m_r=16, tile=t))
    # outside the trained range the analytic rule runs (still correct)
    rosko.rosko_selector_set(params, np.zeros(16), np.ones(16), f + 10, f + 11)
    check("bf16", *run(rosko, A, B, "bf16", m_r=16, tile=t))
